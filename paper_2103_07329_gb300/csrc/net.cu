// net.cu -- the learned initial guess: a 3-D convolutional encoder-decoder
// that maps (right-hand side, log coefficient) on the grid to a first iterate
// X0 of the Krylov solve, trained on the GPU on solutions the solver itself
// produces.  The paper has no learned component; this is the warm-started
// form that is measured against X0 = 0.
//
// Tensors are channels-last BF16 blocks [sample][z][y][x][c] (c = 8 or 16) on
// grids of edge Nl.  Every convolution is 3x3x3, stride 1, zero padding 1, a
// cross-correlation with tap t = 9 (dz+1) + 3 (dy+1) + (dx+1):
//   forward         out[v][co] = b[co] + sum_{t,ci} W[co][t][ci] in[v + off_t][ci]
//   backward-data   gin[v][ci] = sum_{t,co} W[co][t][ci] g[v - off_t][co], which is the
//                   forward form with the taps mirrored (t -> 26 - t) and the
//                   channel roles swapped
//   backward-weight dW[co][t][ci] = sum_v g[v][co] in[v + off_t][ci], db[co] = sum_v g[v][co]
// where g is the output gradient, multiplied by [out > 0] behind a ReLU.
// All three run as implicit GEMMs on the tensor cores (mma.sync m16n8k16,
// BF16 operands, FP32 accumulation) with ldmatrix fragment loads:
//   forward / backward-data: M = voxels, N = output channels, K = 27 CIN
//   backward-weight:         M = output channels, N = 27 CIN, K = voxels.
// A block works on 8x8x8 bricks of output voxels with the 10^3 input brick
// (halo included, zero outside the grid) staged in shared memory; warp w owns
// slice z = w, i.e. four 16-voxel M tiles of 8 voxels in x by 2 in y.
// Weight gradients are summed per block in registers over the block's bricks
// and the per-block partial sums are reduced in a fixed order, so every
// result is a deterministic function of the inputs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/xamg_gpu.h"
#include "launch.h"

namespace xamg {
namespace net {

using bf16 = __nv_bfloat16;
constexpr int kThreads = 256;
constexpr int kWgradGrid = 304;  // blocks of every backward-weight launch (fixed: deterministic sums)

__host__ __device__ constexpr int kpad(int cin) { return (27 * cin + 15) / 16 * 16; }
// Row strides in shared memory, chosen so that the eight 16-byte rows of
// every ldmatrix phase fall into distinct bank groups.
__host__ __device__ constexpr int vstride(int c) { return c == 16 ? 24 : c; }
__host__ __device__ constexpr int kstride(int cin) { return kpad(cin) + 8; }
constexpr int kGStride = 24;  // voxel stride of the staged output gradient

// Two input bricks (the one being multiplied and the next one in flight),
// the weights and a zero row.
template <int CIN, int COUT>
constexpr size_t fwd_smem() {
  return (size_t)(2 * 1000 * vstride(CIN) + COUT * kstride(CIN) + 8) * sizeof(bf16);
}
template <int CIN>
constexpr size_t wgrad_smem() {
  return (size_t)(1000 * vstride(CIN) + 512 * kGStride) * sizeof(bf16) + kThreads * sizeof(float);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t b0,
                                         const uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t &r0, uint32_t &r1, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ int tap_offset(int t) {  // halo-brick voxel offset of tap t
  return (t / 9 - 1) * 100 + ((t / 3) % 3 - 1) * 10 + (t % 3 - 1);
}

struct Brick {
  int64_t sbase;  // first voxel of the sample
  int x0, y0, z0;
};

__device__ __forceinline__ Brick brick_of(int b, int nb, int N) {
  Brick r;
  const int per = nb * nb * nb;
  const int s = b / per, q = b % per;
  r.x0 = (q % nb) * 8;
  r.y0 = ((q / nb) % nb) * 8;
  r.z0 = (q / (nb * nb)) * 8;
  r.sbase = (int64_t)s * N * N * N;
  return r;
}

// Stages the 10^3 input brick (zero outside the grid) around the output brick
// at (x0, y0, z0) with voxel stride VS; with `mask`, an element is kept only
// where the mask element is > 0.
template <int C, int VS>
__device__ __forceinline__ void stage_brick(bf16 *dst, const bf16 *__restrict__ src,
                                            const bf16 *__restrict__ mask, int N, const Brick &bk) {
  constexpr int CH = C / 8;  // 16-byte chunks per voxel
  for (int idx = threadIdx.x; idx < 1000 * CH; idx += kThreads) {
    const int vox = idx / CH, part = idx % CH;
    const int hx = vox % 10, hy = (vox / 10) % 10, hz = vox / 100;
    const int gz = bk.z0 + hz - 1, gy = bk.y0 + hy - 1, gx = bk.x0 + hx - 1;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (gz >= 0 && gz < N && gy >= 0 && gy < N && gx >= 0 && gx < N) {
      const int64_t off = (bk.sbase + ((int64_t)gz * N + gy) * N + gx) * C + part * 8;
      val = __ldg(reinterpret_cast<const uint4 *>(src + off));
      if (mask) {
        const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(mask + off));
        bf16 *v = reinterpret_cast<bf16 *>(&val);
        const bf16 *mm = reinterpret_cast<const bf16 *>(&mk);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (!(__bfloat162float(mm[j]) > 0.0f)) v[j] = __float2bfloat16(0.0f);
      }
    }
    *reinterpret_cast<uint4 *>(dst + vox * VS + part * 8) = val;
  }
}

// The same staging without a mask, as asynchronous 16-byte copies (zero
// filled outside the grid) that complete while the previous brick is
// multiplied; the caller commits and waits.
template <int C, int VS>
__device__ __forceinline__ void stage_brick_async(bf16 *dst, const bf16 *__restrict__ src, int N,
                                                  const Brick &bk) {
  constexpr int CH = C / 8;  // 16-byte chunks per voxel
  for (int idx = threadIdx.x; idx < 1000 * CH; idx += kThreads) {
    const int vox = idx / CH, part = idx % CH;
    const int hx = vox % 10, hy = (vox / 10) % 10, hz = vox / 100;
    const int gz = bk.z0 + hz - 1, gy = bk.y0 + hy - 1, gx = bk.x0 + hx - 1;
    const bool in = gz >= 0 && gz < N && gy >= 0 && gy < N && gx >= 0 && gx < N;
    // outside the grid: no bytes read (src-size 0), the 16 bytes are zeroed
    const int64_t off = in ? (bk.sbase + ((int64_t)gz * N + gy) * N + gx) * C + part * 8 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst + vox * VS + part * 8)),
                 "l"(src + off), "r"(in ? 16 : 0)
                 : "memory");
  }
}

// out = [relu](conv(in [* (mask > 0)]) + bias); wt: BF16 [COUT][kpad(CIN)]
// with k = t CIN + ci and zeros for k >= 27 CIN.  With out0 != NULL only
// output channel 0 is stored, in FP32, to out0[sample][voxel] (out unused).
// Blocks loop over the `total` bricks (samples x nb^3).
template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(kThreads) k_conv3(const bf16 *__restrict__ in,
                                                    const bf16 *__restrict__ mask,
                                                    const bf16 *__restrict__ wt,
                                                    const float *__restrict__ bias,
                                                    bf16 *__restrict__ out, float *__restrict__ out0,
                                                    int N, int nb, int total) {
  constexpr int VS = vstride(CIN), KP = kpad(CIN), KS = kstride(CIN), NT = COUT / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *in_s = reinterpret_cast<bf16 *>(smem_raw);
  bf16 *w_s = in_s + 2 * 1000 * VS;  // after the two input bricks
  bf16 *zero_s = w_s + COUT * KS;
  for (int idx = threadIdx.x; idx < COUT * (KP / 8); idx += kThreads) {
    const int row = idx / (KP / 8), ch = idx % (KP / 8);
    *reinterpret_cast<uint4 *>(w_s + row * KS + ch * 8) = __ldg(reinterpret_cast<const uint4 *>(wt) + idx);
  }
  if (threadIdx.x == 0) *reinterpret_cast<uint4 *>(zero_s) = make_uint4(0, 0, 0, 0);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int mi = lane >> 3, r = lane & 7;  // ldmatrix: matrix and row this lane addresses
  const int z = warp;
  const uint32_t in_a = smem_addr(in_s), w_a = smem_addr(w_s), zero_a = smem_addr(zero_s);
  // B (weights [n][k]): matrix mi covers n = (mi >> 1) * 8 + r (two N tiles)
  // or n = r (one N tile; lanes 16..31 are then ignored), k half (mi & 1).
  const int bn = (NT == 2 ? (mi >> 1) * 8 : 0) + r;
  const uint32_t b_row = w_a + (uint32_t)(bn * KS + (mi & 1) * 8) * 2u;
  float bv[NT][2];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    bv[nt][0] = bias ? __ldg(bias + nt * 8 + 2 * tq) : 0.0f;
    bv[nt][1] = bias ? __ldg(bias + nt * 8 + 2 * tq + 1) : 0.0f;
  }

  // without a mask the input bricks are double-buffered: brick b + gridDim.x
  // is copied asynchronously while brick b is multiplied
  int buf = 0;
  if (!mask && blockIdx.x < total) {
    stage_brick_async<CIN, VS>(in_s, in, N, brick_of(blockIdx.x, nb, N));
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int b = blockIdx.x; b < total; b += gridDim.x) {
    const Brick bk = brick_of(b, nb, N);
    if (mask) {
      __syncthreads();  // the previous brick's fragments are consumed
      stage_brick<CIN, VS>(in_s, in, mask, N, bk);
    } else {
      // the other buffer was last read by the previous brick's fragments
      __syncthreads();
      if (b + (int)gridDim.x < total)
        stage_brick_async<CIN, VS>(in_s + (buf ^ 1) * 1000 * VS, in, N, brick_of(b + gridDim.x, nb, N));
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this brick's copies
    }
    __syncthreads();
    const uint32_t in_b = in_a + (uint32_t)(buf * 1000 * VS) * 2u;
    float acc[4][NT][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.0f;
    // A row of this lane in M tile mt: voxel (x = r, y = 2 mt + (mi & 1), z);
    // matrix mi covers k half (mi >> 1)
    const int a_base = ((z + 1) * 10 + 1 + (mi & 1)) * 10 + 1 + r;
#pragma unroll 2
    for (int ks = 0; ks < KP / 16; ++ks) {
      uint32_t bf[NT][2];
      if constexpr (NT == 2) {
        uint32_t q[4];
        ldsm_x4(q, b_row + ks * 32u);
        bf[0][0] = q[0];
        bf[0][1] = q[1];
        bf[NT - 1][0] = q[2];
        bf[NT - 1][1] = q[3];
      } else {
        ldsm_x2(bf[0][0], bf[0][1], b_row + ks * 32u);
      }
      const int kq = ks * 16 + (mi >> 1) * 8;  // first k of this lane's 8-wide chunk
      const int t = kq / CIN, c0 = kq % CIN;
      const bool real = t < 27;
      const int toff = real ? tap_offset(t) : 0;
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int hv = a_base + mt * 20 + toff;
        const uint32_t addr = real ? in_b + (uint32_t)(hv * VS + c0) * 2u : zero_a;
        uint32_t a[4];
        ldsm_x4(a, addr);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) mma16816(acc[mt][nt], a, bf[nt][0], bf[nt][1]);
      }
    }
    const int gz = bk.z0 + z, gx = bk.x0 + g;
    if (gz < N && gx < N) {
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int gy = bk.y0 + 2 * mt + h;
          if (gy >= N) continue;
          const int64_t vox = bk.sbase + ((int64_t)gz * N + gy) * N + gx;
          if (out0) {
            if (tq == 0) {
              const float v0 = acc[mt][0][2 * h] + bv[0][0];
              out0[vox] = RELU ? fmaxf(v0, 0.0f) : v0;
            }
            continue;
          }
          const int64_t o = vox * COUT + 2 * tq;
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            float v0 = acc[mt][nt][2 * h] + bv[nt][0], v1 = acc[mt][nt][2 * h + 1] + bv[nt][1];
            if (RELU) {
              v0 = fmaxf(v0, 0.0f);
              v1 = fmaxf(v1, 0.0f);
            }
            *reinterpret_cast<uint32_t *>(out + o + nt * 8) = pack2(v0, v1);
          }
        }
    }
    if (!mask) buf ^= 1;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");  // no copy left in flight at exit
}

// Per-block partial sums of one layer's weight and bias gradients over the
// bricks b = blockIdx.x, blockIdx.x + gridDim.x, ...:
//   part[block][co][k] = sum_v gz[v][co] in[v + off_t][ci]   (k = t CIN + ci < kpad)
//   bpart[block][co]   = sum_v gz[v][co]
// with gz = gout * (act > 0) when act is given.
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) k_conv3_wgrad(const bf16 *__restrict__ in,
                                                          const bf16 *__restrict__ gout,
                                                          const bf16 *__restrict__ act,
                                                          float *__restrict__ part,
                                                          float *__restrict__ bpart, int N, int nb,
                                                          int total) {
  constexpr int VS = vstride(CIN), KP = kpad(CIN), NTILES = KP / 8;
  constexpr int NPW = (NTILES + 7) / 8;  // N tiles per warp
  constexpr int CHO = COUT / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *in_s = reinterpret_cast<bf16 *>(smem_raw);
  bf16 *g_s = in_s + 1000 * VS;
  float *bred = reinterpret_cast<float *>(g_s + 512 * kGStride);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int mi = lane >> 3, r = lane & 7;
  const uint32_t in_a = smem_addr(in_s), g_a = smem_addr(g_s);
  // this warp's N tiles: tile = warp * NPW + j covers k = 8 tile .. 8 tile + 7,
  // all in one tap because CIN is a multiple of 8
  int toff[NPW], cofs[NPW];
  bool real[NPW];
#pragma unroll
  for (int j = 0; j < NPW; ++j) {
    const int tile = warp * NPW + j;
    const int t = tile * 8 / CIN;
    real[j] = tile < NTILES && t < 27;
    toff[j] = real[j] ? tap_offset(t) : 0;
    cofs[j] = (tile * 8) % CIN;
  }
  float acc[NPW][4];
#pragma unroll
  for (int j = 0; j < NPW; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
  float bsum = 0.0f;  // bias partial of channel (threadIdx.x & 15)

  for (int b = blockIdx.x; b < total; b += gridDim.x) {
    const Brick bk = brick_of(b, nb, N);
    __syncthreads();
    stage_brick<CIN, VS>(in_s, in, nullptr, N, bk);
    for (int idx = threadIdx.x; idx < 512 * 2; idx += kThreads) {
      const int v = idx >> 1, part_i = idx & 1;
      uint4 val = make_uint4(0, 0, 0, 0);
      const int x = v & 7, y = (v >> 3) & 7, zz = v >> 6;
      const int gx = bk.x0 + x, gy = bk.y0 + y, gz = bk.z0 + zz;
      if (part_i < CHO && gx < N && gy < N && gz < N) {
        const int64_t o = (bk.sbase + ((int64_t)gz * N + gy) * N + gx) * COUT + part_i * 8;
        val = __ldg(reinterpret_cast<const uint4 *>(gout + o));
        if (act) {
          const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(act + o));
          bf16 *vv = reinterpret_cast<bf16 *>(&val);
          const bf16 *mm = reinterpret_cast<const bf16 *>(&mk);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (!(__bfloat162float(mm[j]) > 0.0f)) vv[j] = __float2bfloat16(0.0f);
        }
      }
      *reinterpret_cast<uint4 *>(g_s + v * kGStride + part_i * 8) = val;
    }
    __syncthreads();
    for (int v = threadIdx.x >> 4; v < 512; v += kThreads / 16)
      bsum += __bfloat162float(g_s[v * kGStride + (threadIdx.x & 15)]);
#pragma unroll 2
    for (int ks = 0; ks < 32; ++ks) {
      // A = gz^T: matrix mi holds voxels ks*16 + (mi >> 1)*8 + r, channels (mi & 1)*8 ..
      uint32_t a[4];
      ldsm_x4_t(a, g_a + (uint32_t)((ks * 16 + (mi >> 1) * 8 + r) * kGStride + (mi & 1) * 8) * 2u);
      // B rows: voxel ks*16 + h*8 + r = (x r, y (2 ks + h) & 7, z (2 ks + h) >> 3),
      // h = (mi & 1) for the lanes that address rows (0..15)
      const int yy = 2 * ks + (mi & 1);
      const int b_base = (((yy >> 3) + 1) * 10 + (yy & 7) + 1) * 10 + r + 1;
#pragma unroll
      for (int j = 0; j < NPW; ++j) {
        if (!real[j]) continue;
        uint32_t b0, b1;
        ldsm_x2_t(b0, b1, in_a + (uint32_t)((b_base + toff[j]) * VS + cofs[j]) * 2u);
        mma16816(acc[j], a, b0, b1);
      }
    }
  }
  const size_t pbase = (size_t)blockIdx.x * COUT * KP;
#pragma unroll
  for (int j = 0; j < NPW; ++j) {
    const int tile = warp * NPW + j;
    if (tile >= NTILES) continue;
    const int c = tile * 8 + 2 * tq;
    if (g < COUT)
      *reinterpret_cast<float2 *>(part + pbase + (size_t)g * KP + c) = make_float2(acc[j][0], acc[j][1]);
    if (g + 8 < COUT)
      *reinterpret_cast<float2 *>(part + pbase + (size_t)(g + 8) * KP + c) = make_float2(acc[j][2], acc[j][3]);
  }
  __syncthreads();
  bred[threadIdx.x] = bsum;
  __syncthreads();
  if (threadIdx.x < COUT) {
    float s = 0.0f;
    for (int q = 0; q < kThreads / 16; ++q) s += bred[q * 16 + threadIdx.x];
    bpart[(size_t)blockIdx.x * COUT + threadIdx.x] = s;
  }
}

// gW[co][k] (k < 27 cin, unpadded) = sum over blocks of part[b][co][k] (rows
// of kp), in block order.
__global__ void k_reduce_wgrad(const float *__restrict__ part, int nblk, int cout, int cin, int kp,
                               float *__restrict__ gw) {
  const int kk = 27 * cin;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cout * kk) return;
  const int co = i / kk, k = i % kk;
  float s = 0.0f;
  for (int b = 0; b < nblk; ++b) s += part[((size_t)b * cout + co) * kp + k];
  gw[i] = s;
}

// out[i] = sum over blocks of part[b][i], in block order.
__global__ void k_reduce_parts(const float *__restrict__ part, int nblk, int len, float *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  float s = 0.0f;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * len + i];
  out[i] = s;
}

// ---- grid transfers on channels-last BF16 tensors, 8 channels per thread ----
// coarse (Nc^3) = mean of the 2x2x2 fine children
__global__ void k_pool2(const bf16 *__restrict__ in, bf16 *__restrict__ out, int Nc, int C, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int CH = C / 8;
  const int part = (int)(i % CH);
  const int64_t v = i / CH;
  const int x = (int)(v % Nc), y = (int)((v / Nc) % Nc), z = (int)((v / Nc / Nc) % Nc);
  const int64_t s = v / ((int64_t)Nc * Nc * Nc);
  const int Nf = 2 * Nc;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int d = 0; d < 8; ++d) {
    const int fz = 2 * z + (d >> 2), fy = 2 * y + ((d >> 1) & 1), fx = 2 * x + (d & 1);
    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(in + ((((s * Nf + fz) * Nf + fy) * Nf + fx) * C + part * 8)));
    const bf16 *e = reinterpret_cast<const bf16 *>(&q);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(e[j]);
  }
  uint4 o;
  uint32_t *ow = reinterpret_cast<uint32_t *>(&o);
#pragma unroll
  for (int j = 0; j < 4; ++j) ow[j] = pack2(0.125f * acc[2 * j], 0.125f * acc[2 * j + 1]);
  *reinterpret_cast<uint4 *>(out + v * C + part * 8) = o;
}

// fine (Nf^3): out = scale * coarse[parent] + skip (skip may be NULL).
// Forward: nearest upsampling plus the skip connection (scale 1); backward of
// the pooling: the coarse gradient / 8 added to the skip path's gradient.
__global__ void k_up2_add(const bf16 *__restrict__ coarse, const bf16 *__restrict__ skip,
                          bf16 *__restrict__ out, int Nf, int C, float scale, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int CH = C / 8;
  const int part = (int)(i % CH);
  const int64_t v = i / CH;
  const int x = (int)(v % Nf), y = (int)((v / Nf) % Nf), z = (int)((v / Nf / Nf) % Nf);
  const int64_t s = v / ((int64_t)Nf * Nf * Nf);
  const int Nc = Nf / 2;
  const uint4 q = __ldg(reinterpret_cast<const uint4 *>(
      coarse + ((((s * Nc + z / 2) * Nc + y / 2) * Nc + x / 2) * C + part * 8)));
  const bf16 *e = reinterpret_cast<const bf16 *>(&q);
  float sk[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (skip) {
    const uint4 p = __ldg(reinterpret_cast<const uint4 *>(skip + v * C + part * 8));
    const bf16 *f = reinterpret_cast<const bf16 *>(&p);
#pragma unroll
    for (int j = 0; j < 8; ++j) sk[j] = __bfloat162float(f[j]);
  }
  uint4 o;
  uint32_t *ow = reinterpret_cast<uint32_t *>(&o);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    ow[j] = pack2(fmaf(scale, __bfloat162float(e[2 * j]), sk[2 * j]),
                  fmaf(scale, __bfloat162float(e[2 * j + 1]), sk[2 * j + 1]));
  *reinterpret_cast<uint4 *>(out + v * C + part * 8) = o;
}

// backward of the nearest upsampling: coarse gradient = sum of the 8 children
__global__ void k_up2_bwd(const bf16 *__restrict__ gfine, bf16 *__restrict__ out, int Nc, int C, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int CH = C / 8;
  const int part = (int)(i % CH);
  const int64_t v = i / CH;
  const int x = (int)(v % Nc), y = (int)((v / Nc) % Nc), z = (int)((v / Nc / Nc) % Nc);
  const int64_t s = v / ((int64_t)Nc * Nc * Nc);
  const int Nf = 2 * Nc;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int d = 0; d < 8; ++d) {
    const int fz = 2 * z + (d >> 2), fy = 2 * y + ((d >> 1) & 1), fx = 2 * x + (d & 1);
    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(gfine + ((((s * Nf + fz) * Nf + fy) * Nf + fx) * C + part * 8)));
    const bf16 *e = reinterpret_cast<const bf16 *>(&q);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(e[j]);
  }
  uint4 o;
  uint32_t *ow = reinterpret_cast<uint32_t *>(&o);
#pragma unroll
  for (int j = 0; j < 4; ++j) ow[j] = pack2(acc[2 * j], acc[2 * j + 1]);
  *reinterpret_cast<uint4 *>(out + v * C + part * 8) = o;
}

// network input of sample b: channels (inp[src][v][0], inp[src][v][1], 0 x 6)
// with src = idx ? idx[b] : b
__global__ void k_pack_input(const float *__restrict__ inp, const int32_t *__restrict__ idx, int64_t V,
                             int batch, bf16 *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * batch) return;
  const int b = (int)(i / V);
  const int64_t v = i % V;
  const int64_t src = (idx ? (int64_t)idx[b] : (int64_t)b) * V + v;
  const float2 q = __ldg(reinterpret_cast<const float2 *>(inp) + src);
  *reinterpret_cast<uint4 *>(out + i * 8) = make_uint4(pack2(q.x, q.y), 0u, 0u, 0u);
}

// Transposes between the solver's n x m row-major blocks and the network's
// sample-major tensors, through a 32-voxel x 32-column tile in shared memory
// so that both sides are read and written in whole rows.  Block (32, 8).
//
// Network input from B: channel 0 of sample j = B[v][j] / s_j (s_j the
// column's root mean square; 0 for a zero column), channel 1 = logk[v].
__global__ void __launch_bounds__(256) k_pack_rhs(const double *__restrict__ B, int m,
                                                  const double *__restrict__ ss, int64_t n,
                                                  const float *__restrict__ logk, bf16 *__restrict__ out) {
  __shared__ float tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t v0 = (int64_t)blockIdx.x * 32;
  for (int r = ty; r < 32; r += 8) {
    const int64_t v = v0 + r;
    float val = 0.0f;
    if (tx < m && v < n) {
      const double s = sqrt(ss[tx] / (double)n);
      val = s > 0.0 ? (float)(B[v * m + tx] / s) : 0.0f;
    }
    tile[r][tx] = val;
  }
  __syncthreads();
  const int64_t v = v0 + tx;
  if (v >= n) return;
  const float lk = __ldg(logk + v);
  for (int j = ty; j < m; j += 8)
    *reinterpret_cast<uint4 *>(out + ((int64_t)j * n + v) * 8) = make_uint4(pack2(tile[tx][j], lk), 0u, 0u, 0u);
}

// X0[v][j] = y[j][v] * s_j * scale
__global__ void __launch_bounds__(256) k_unpack_x0(const float *__restrict__ y, int m,
                                                   const double *__restrict__ ss, int64_t n, double scale,
                                                   double *__restrict__ X0) {
  __shared__ float tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t v0 = (int64_t)blockIdx.x * 32;
  for (int j = ty; j < m; j += 8) tile[j][tx] = v0 + tx < n ? y[(int64_t)j * n + v0 + tx] : 0.0f;
  __syncthreads();
  if (tx >= m) return;
  const double f = sqrt(ss[tx] / (double)n) * scale;
  for (int r = ty; r < 32; r += 8) {
    const int64_t v = v0 + r;
    if (v < n) X0[v * m + tx] = (double)tile[tx][r] * f;
  }
}

__device__ __forceinline__ int64_t sample_row(const int32_t *idx, int b) {
  return idx ? (int64_t)idx[b] : (int64_t)b;
}

__device__ __forceinline__ float block_sum(float s, float *red) {
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  return red[0];
}

// Mean squared error: lpart[block] = inv * sum over its voxels of
// w_b (y - t)^2 and the output gradient gy = (2 inv w_b (y - t), 0 x 7), with
// inv = 1 / (batch N^3), w_b = wsample[src] (1 if NULL), src = idx[b] or b.
__global__ void __launch_bounds__(kThreads) k_mse(const float *__restrict__ y, const float *__restrict__ target,
                                                  const int32_t *__restrict__ idx,
                                                  const float *__restrict__ wsample, int64_t V, int batch,
                                                  float inv, bf16 *__restrict__ gy, float *__restrict__ lpart) {
  __shared__ float red[kThreads];
  float s = 0.0f;
  const int64_t total = V * batch;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / V);
    const int64_t src = sample_row(idx, b);
    const float w = wsample ? __ldg(wsample + src) : 1.0f;
    const float d = y[i] - __ldg(target + src * V + i % V);
    s = fmaf(w * d, d, s);
    *reinterpret_cast<uint4 *>(gy + 8 * i) = make_uint4(pack2(2.0f * inv * w * d, 0.0f), 0u, 0u, 0u);
  }
  const float t = block_sum(s, red);
  if (threadIdx.x == 0) lpart[blockIdx.x] = t * inv;
}

// Energy-norm loss of the cell-centred diffusion operator A_b whose log
// coefficient is channel 1 of the sample's input (inp[src][v][1]), the
// operator of problems.diffusion7 (face transmissibility 2 k_a k_c / (k_a +
// k_c) between cells, 2 k_c on a boundary face):
//   L = (1 / batch) sum_b w_b e_b^T A_b e_b,  e_b = y_b - t_b,
//   dL/dy_b = (2 / batch) w_b A_b e_b.
// lpart[block] = the block's share of L; gy = (dL/dy, 0 x 7).
__global__ void __launch_bounds__(kThreads) k_energy(const float *__restrict__ y, const float *__restrict__ target,
                                                     const float *__restrict__ inp, const int32_t *__restrict__ idx,
                                                     const float *__restrict__ wsample, int N, int batch,
                                                     float invb, bf16 *__restrict__ gy, float *__restrict__ lpart) {
  __shared__ float red[kThreads];
  const int64_t V = (int64_t)N * N * N;
  float s = 0.0f;
  const int64_t total = V * batch;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / V);
    const int64_t v = i % V;
    const int64_t src = sample_row(idx, b);
    const float w = wsample ? __ldg(wsample + src) : 1.0f;
    const float *lk = inp + src * V * 2 + 1;  // log k, stride 2
    const float *tg = target + src * V;
    const float *yb = y + (int64_t)b * V;
    const int x = (int)(v % N), yy = (int)((v / N) % N), z = (int)(v / ((int64_t)N * N));
    const float kc = expf(__ldg(lk + 2 * v));
    const float ec = yb[v] - __ldg(tg + v);
    float ae = 0.0f;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int d = (f & 1) ? 1 : -1;
      const int ax = f >> 1;  // 0: x, 1: y, 2: z
      const int c = ax == 0 ? x : (ax == 1 ? yy : z);
      if (c + d < 0 || c + d >= N) {
        ae = fmaf(2.0f * kc, ec, ae);
        continue;
      }
      const int64_t nb = v + (int64_t)d * (ax == 0 ? 1 : (ax == 1 ? (int64_t)N : (int64_t)N * N));
      const float kn = expf(__ldg(lk + 2 * nb));
      const float T = 2.0f * kc * kn / (kc + kn);
      ae = fmaf(T, ec - (yb[nb] - __ldg(tg + nb)), ae);
    }
    s = fmaf(w * ec, ae, s);
    *reinterpret_cast<uint4 *>(gy + 8 * i) = make_uint4(pack2(2.0f * invb * w * ae, 0.0f), 0u, 0u, 0u);
  }
  const float t = block_sum(s, red);
  if (threadIdx.x == 0) lpart[blockIdx.x] = t * invb;
}

// Adam (Kingma & Ba 2015) on the FP32 parameters; c1 = 1 - b1^t, c2 = 1 - b2^t
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi;
  const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// BF16 operands of one layer from its FP32 weights W[co][t][ci]:
// forward wt[co][k] (k = t cin + ci, zero for k >= 27 cin, rows of kpad(cin)),
// backward-data wb[ci][k'] = W[co][26 - t'][ci] (k' = t' cout + co, rows of kpad(cout))
__global__ void k_prep_weights(const float *__restrict__ W, bf16 *__restrict__ wt, bf16 *__restrict__ wb,
                               int cin, int cout) {
  const int kp = kpad(cin), kpb = kpad(cout);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (wt && i < cout * kp) {
    const int co = i / kp, k = i % kp;
    wt[i] = __float2bfloat16(k < 27 * cin ? W[co * 27 * cin + k] : 0.0f);
  }
  if (wb && i < cin * kpb) {
    const int ci = i / kpb, k = i % kpb;
    const int t = k / cout, co = k % cout;
    wb[i] = __float2bfloat16(t < 27 ? W[(co * 27 + (26 - t)) * cin + ci] : 0.0f);
  }
}

// ------------------------------------------------------------------ launchers
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <int CIN, int COUT, bool RELU>
cudaError_t conv_t(const bf16 *in, const bf16 *mask, const bf16 *wt, const float *bias, bf16 *out, float *out0,
                   int batch, int N, cudaStream_t st) {
  constexpr size_t sm = fwd_smem<CIN, COUT>();
  static int per_sm = 0;  // resident blocks per SM
  if (!per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3<CIN, COUT, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3<CIN, COUT, RELU>, kThreads, sm);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
  }
  const int nb = (N + 7) / 8;
  const int total = nb * nb * nb * batch;
  const int grid = (int)std::min<int64_t>(total, (int64_t)device_sm_count() * per_sm);
  k_conv3<CIN, COUT, RELU><<<grid, kThreads, sm, st>>>(in, mask, wt, bias, out, out0, N, nb, total);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t conv(int cin, int cout, bool relu, const bf16 *in, const bf16 *mask, const bf16 *wt,
                 const float *bias, bf16 *out, int batch, int N, cudaStream_t st, float *out0 = nullptr) {
#define XAMG_CONV_CASE(CI, CO)                                                \
  if (cin == CI && cout == CO)                                                \
    return relu ? conv_t<CI, CO, true>(in, mask, wt, bias, out, out0, batch, N, st) \
                : conv_t<CI, CO, false>(in, mask, wt, bias, out, out0, batch, N, st);
  XAMG_CONV_CASE(8, 8)
  XAMG_CONV_CASE(8, 16)
  XAMG_CONV_CASE(16, 8)
  XAMG_CONV_CASE(16, 16)
#undef XAMG_CONV_CASE
  return cudaErrorInvalidValue;
}

template <int CIN, int COUT>
cudaError_t wgrad_t(const bf16 *in, const bf16 *gout, const bf16 *act, float *part, float *bpart, int batch,
                    int N, int *grid_out, cudaStream_t st) {
  constexpr size_t sm = wgrad_smem<CIN>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nb = (N + 7) / 8;
  const int total = nb * nb * nb * batch;
  const int grid = std::min(total, kWgradGrid);
  k_conv3_wgrad<CIN, COUT><<<grid, kThreads, sm, st>>>(in, gout, act, part, bpart, N, nb, total);
  ++g_launches;
  *grid_out = grid;
  return cudaGetLastError();
}

// dW (unpadded [cout][27][cin]) and db of one layer; part must hold
// kWgradGrid * cout * kpad(cin) floats, bpart kWgradGrid * cout.
cudaError_t wgrad(int cin, int cout, const bf16 *in, const bf16 *gout, const bf16 *act, float *part, float *bpart,
                  float *dw, float *db, int batch, int N, cudaStream_t st) {
  int grid = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (cin == 8 && cout == 8) e = wgrad_t<8, 8>(in, gout, act, part, bpart, batch, N, &grid, st);
  if (cin == 8 && cout == 16) e = wgrad_t<8, 16>(in, gout, act, part, bpart, batch, N, &grid, st);
  if (cin == 16 && cout == 8) e = wgrad_t<16, 8>(in, gout, act, part, bpart, batch, N, &grid, st);
  if (cin == 16 && cout == 16) e = wgrad_t<16, 16>(in, gout, act, part, bpart, batch, N, &grid, st);
  if (e != cudaSuccess) return e;
  const int len = cout * 27 * cin;
  k_reduce_wgrad<<<(int)cdiv(len, 256), 256, 0, st>>>(part, grid, cout, cin, kpad(cin), dw);
  k_reduce_parts<<<1, 32, 0, st>>>(bpart, grid, cout, db);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t prep_weights(const float *W, bf16 *wt, bf16 *wb, int cin, int cout, cudaStream_t st) {
  const int len = std::max(cout * kpad(cin), cin * kpad(cout));
  k_prep_weights<<<(int)cdiv(len, 256), 256, 0, st>>>(W, wt, wb, cin, cout);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t pool(const bf16 *in, bf16 *out, int batch, int Nc, int C, cudaStream_t st) {
  const int64_t total = (int64_t)batch * Nc * Nc * Nc * (C / 8);
  k_pool2<<<(int)cdiv(total, 256), 256, 0, st>>>(in, out, Nc, C, total);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t up_add(const bf16 *coarse, const bf16 *skip, bf16 *out, int batch, int Nf, int C, float scale,
                   cudaStream_t st) {
  const int64_t total = (int64_t)batch * Nf * Nf * Nf * (C / 8);
  k_up2_add<<<(int)cdiv(total, 256), 256, 0, st>>>(coarse, skip, out, Nf, C, scale, total);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t up_bwd(const bf16 *gfine, bf16 *out, int batch, int Nc, int C, cudaStream_t st) {
  const int64_t total = (int64_t)batch * Nc * Nc * Nc * (C / 8);
  k_up2_bwd<<<(int)cdiv(total, 256), 256, 0, st>>>(gfine, out, Nc, C, total);
  ++g_launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ network
// Encoder-decoder with four grid levels (edges N, N/2, N/4, N/8):
//   e0a 2(8)->8, e0b 8->8                      level 0 -> s0
//   pool, e1a 8->16, e1b 16->16                level 1 -> s1
//   pool, e2a 16->16, e2b 16->16               level 2 -> s2
//   pool, e3a 16->16, e3b 16->16               level 3
//   up + s2, d2 16->16                         level 2
//   up + s1, d1a 16->16, d1b 16->8             level 1
//   up + s0, d0a 8->8, d0b 8->8 (linear)       level 0 -> channel 0 = output
// ReLU after every convolution but the last.
enum Act {
  T_X, T_E0A, T_S0, T_P0, T_E1A, T_S1, T_P1, T_E2A, T_S2, T_P2, T_E3A, T_E3B,
  T_U2, T_D2, T_U1, T_D1A, T_D1B, T_U0, T_D0A, T_Y, T_COUNT
};
struct TensorDef {
  int level, channels;
};
constexpr TensorDef kTensors[T_COUNT] = {
    {0, 8}, {0, 8}, {0, 8}, {1, 8}, {1, 16}, {1, 16}, {2, 16}, {2, 16}, {2, 16}, {3, 16},
    {3, 16}, {3, 16}, {2, 16}, {2, 16}, {1, 16}, {1, 16}, {1, 8}, {0, 8}, {0, 8}, {0, 8}};
struct LayerDef {
  int cin, cout, relu, in, out;
};
constexpr int kLayers = 13;
constexpr LayerDef kLayerDefs[kLayers] = {
    {8, 8, 1, T_X, T_E0A},     {8, 8, 1, T_E0A, T_S0},    {8, 16, 1, T_P0, T_E1A},
    {16, 16, 1, T_E1A, T_S1},  {16, 16, 1, T_P1, T_E2A},  {16, 16, 1, T_E2A, T_S2},
    {16, 16, 1, T_P2, T_E3A},  {16, 16, 1, T_E3A, T_E3B}, {16, 16, 1, T_U2, T_D2},
    {16, 16, 1, T_U1, T_D1A},  {16, 8, 1, T_D1A, T_D1B},  {8, 8, 1, T_U0, T_D0A},
    {8, 8, 0, T_D0A, T_Y}};

int64_t param_count() {
  int64_t n = 0;
  for (const LayerDef &L : kLayerDefs) n += (int64_t)L.cout * 27 * L.cin + L.cout;
  return n;
}

}  // namespace net
}  // namespace xamg

using namespace xamg;
using namespace xamg::net;

struct xamg_net {
  int N = 0, max_batch = 0, device = 0;
  int64_t np = 0;
  int64_t woff[kLayers] = {}, boff[kLayers] = {};
  float *W = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr;  // flat parameters, gradients, moments
  bf16 *wt[kLayers] = {}, *wb[kLayers] = {};
  bf16 *act[T_COUNT] = {}, *grad[T_COUNT] = {};
  float *part = nullptr, *bpart = nullptr, *lpart = nullptr, *loss_d = nullptr;
  float *y32 = nullptr;       // FP32 network output [max_batch][N^3]
  double *ss = nullptr;       // column sums of squares of the last predicted block
  double *ss_part = nullptr;
  int steps = 0;
  bool weights_fresh = false;
  std::vector<void *> owned;
};

namespace {

constexpr int kLossGrid = 512;

#define NCK(call)                                                             \
  do {                                                                        \
    cudaError_t e__ = (call);                                                 \
    if (e__ != cudaSuccess)                                                   \
      return e__ == cudaErrorMemoryAllocation ? XAMG_ERR_OOM : XAMG_ERR_CUDA; \
  } while (0)

#define NRET(expr)                  \
  do {                              \
    const int r__ = (expr);         \
    if (r__ != XAMG_OK) return r__; \
  } while (0)

int64_t level_vox(const xamg_net *net, int level) {
  const int64_t e = net->N >> level;
  return e * e * e;
}

template <class T>
int net_alloc(xamg_net *net, T **p, size_t count) {
  void *q = nullptr;
  NCK(cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
  net->owned.push_back(q);
  *p = (T *)q;
  return XAMG_OK;
}

int refresh_weights(xamg_net *net, cudaStream_t st) {
  if (net->weights_fresh) return XAMG_OK;
  for (int l = 0; l < kLayers; ++l)
    NCK(prep_weights(net->W + net->woff[l], net->wt[l], net->wb[l], kLayerDefs[l].cin, kLayerDefs[l].cout, st));
  net->weights_fresh = true;
  return XAMG_OK;
}

// Forward pass of `batch` packed samples in act[T_X]; the output (channel 0
// of the last layer, FP32) goes to y[batch][N^3].
int forward(xamg_net *net, int batch, float *y, cudaStream_t st) {
  const int N = net->N;
  auto edge = [&](int t) { return N >> kTensors[t].level; };
  auto L = [&](int l) -> cudaError_t {
    const LayerDef &d = kLayerDefs[l];
    return conv(d.cin, d.cout, d.relu != 0, net->act[d.in], nullptr, net->wt[l], net->W + net->boff[l],
                net->act[d.out], batch, edge(d.out), st, l == kLayers - 1 ? y : nullptr);
  };
  NCK(L(0));
  NCK(L(1));
  NCK(pool(net->act[T_S0], net->act[T_P0], batch, edge(T_P0), 8, st));
  NCK(L(2));
  NCK(L(3));
  NCK(pool(net->act[T_S1], net->act[T_P1], batch, edge(T_P1), 16, st));
  NCK(L(4));
  NCK(L(5));
  NCK(pool(net->act[T_S2], net->act[T_P2], batch, edge(T_P2), 16, st));
  NCK(L(6));
  NCK(L(7));
  NCK(up_add(net->act[T_E3B], net->act[T_S2], net->act[T_U2], batch, edge(T_U2), 16, 1.0f, st));
  NCK(L(8));
  NCK(up_add(net->act[T_D2], net->act[T_S1], net->act[T_U1], batch, edge(T_U1), 16, 1.0f, st));
  NCK(L(9));
  NCK(L(10));
  NCK(up_add(net->act[T_D1B], net->act[T_S0], net->act[T_U0], batch, edge(T_U0), 8, 1.0f, st));
  NCK(L(11));
  NCK(L(12));
  return XAMG_OK;
}

// Gradients of the loss into net->G, given net->grad[T_Y] (the output gradient).
int backward(xamg_net *net, int batch, cudaStream_t st) {
  const int N = net->N;
  auto edge = [&](int t) { return N >> kTensors[t].level; };
  bf16 **A = net->act, **Gd = net->grad;
  // weight gradient of layer l from the gradient of its output (post-activation)
  auto WG = [&](int l) -> cudaError_t {
    const LayerDef &d = kLayerDefs[l];
    return wgrad(d.cin, d.cout, A[d.in], Gd[d.out], d.relu ? A[d.out] : nullptr, net->part, net->bpart,
                 net->G + net->woff[l], net->G + net->boff[l], batch, edge(d.out), st);
  };
  // gradient of layer l's input from the gradient of its output
  auto DG = [&](int l) -> cudaError_t {
    const LayerDef &d = kLayerDefs[l];
    return conv(d.cout, d.cin, false, Gd[d.out], d.relu ? A[d.out] : nullptr, net->wb[l], nullptr, Gd[d.in],
                batch, edge(d.in), st);
  };
  NCK(WG(12));
  NCK(DG(12));  // -> D0A
  NCK(WG(11));
  NCK(DG(11));  // -> U0
  NCK(up_bwd(Gd[T_U0], Gd[T_D1B], batch, edge(T_D1B), 8, st));
  NCK(WG(10));
  NCK(DG(10));  // -> D1A
  NCK(WG(9));
  NCK(DG(9));  // -> U1
  NCK(up_bwd(Gd[T_U1], Gd[T_D2], batch, edge(T_D2), 16, st));
  NCK(WG(8));
  NCK(DG(8));  // -> U2
  NCK(up_bwd(Gd[T_U2], Gd[T_E3B], batch, edge(T_E3B), 16, st));
  NCK(WG(7));
  NCK(DG(7));  // -> E3A
  NCK(WG(6));
  NCK(DG(6));  // -> P2
  NCK(up_add(Gd[T_P2], Gd[T_U2], Gd[T_S2], batch, edge(T_S2), 16, 0.125f, st));
  NCK(WG(5));
  NCK(DG(5));  // -> E2A
  NCK(WG(4));
  NCK(DG(4));  // -> P1
  NCK(up_add(Gd[T_P1], Gd[T_U1], Gd[T_S1], batch, edge(T_S1), 16, 0.125f, st));
  NCK(WG(3));
  NCK(DG(3));  // -> E1A
  NCK(WG(2));
  NCK(DG(2));  // -> P0
  NCK(up_add(Gd[T_P0], Gd[T_U0], Gd[T_S0], batch, edge(T_S0), 8, 0.125f, st));
  NCK(WG(1));
  NCK(DG(1));  // -> E0A
  NCK(WG(0));
  return XAMG_OK;
}

int loss_and_output_grad(xamg_net *net, const float *inp, const float *target, const int32_t *idx,
                         const float *wsample, int kind, int batch, cudaStream_t st) {
  const int64_t V = level_vox(net, 0);
  const int grid = (int)std::min<int64_t>(kLossGrid, cdiv(V * batch, kThreads));
  if (kind == XAMG_NET_LOSS_ENERGY)
    k_energy<<<grid, kThreads, 0, st>>>(net->y32, target, inp, idx, wsample, net->N, batch, 1.0f / batch,
                                        net->grad[T_Y], net->lpart);
  else
    k_mse<<<grid, kThreads, 0, st>>>(net->y32, target, idx, wsample, V, batch, (float)(1.0 / ((double)V * batch)),
                                     net->grad[T_Y], net->lpart);
  k_reduce_parts<<<1, 32, 0, st>>>(net->lpart, grid, 1, net->loss_d);
  g_launches += 2;
  NCK(cudaGetLastError());
  return XAMG_OK;
}

int check_net(const xamg_net *net, int batch) {
  if (!net || batch < 1 || batch > net->max_batch) return XAMG_ERR_INVALID_ARG;
  return XAMG_OK;
}

int pack_input(xamg_net *net, const float *inp, const int32_t *idx, int batch, cudaStream_t st) {
  const int64_t V = level_vox(net, 0);
  k_pack_input<<<(int)cdiv(V * batch, 256), 256, 0, st>>>(inp, idx, V, batch, net->act[T_X]);
  ++g_launches;
  NCK(cudaGetLastError());
  return XAMG_OK;
}

int read_loss(xamg_net *net, float *loss, cudaStream_t st) {
  float l = 0.0f;
  NCK(cudaMemcpyAsync(&l, net->loss_d, sizeof(float), cudaMemcpyDeviceToHost, st));
  NCK(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return std::isfinite(l) ? XAMG_OK : XAMG_ERR_NONFINITE;
}

}  // namespace

extern "C" {

int64_t xamg_net_param_count(void) { return param_count(); }

int xamg_net_create(int32_t N, int32_t max_batch, xamg_net **out) {
  if (!out) return XAMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (N < 8 || N % 8 != 0 || N > 1024 || max_batch < 1 || max_batch > 4096) return XAMG_ERR_INVALID_ARG;
  xamg_net *net = new (std::nothrow) xamg_net();
  if (!net) return XAMG_ERR_OOM;
  net->N = N;
  net->max_batch = max_batch;
  if (cudaGetDevice(&net->device) != cudaSuccess) {
    delete net;
    return XAMG_ERR_CUDA;
  }
  int64_t off = 0;
  for (int l = 0; l < kLayers; ++l) {
    net->woff[l] = off;
    off += (int64_t)kLayerDefs[l].cout * 27 * kLayerDefs[l].cin;
    net->boff[l] = off;
    off += kLayerDefs[l].cout;
  }
  net->np = off;
  int rc = XAMG_OK;
  auto A = [&](auto **p, size_t count) {
    if (rc == XAMG_OK) rc = net_alloc(net, p, count);
  };
  A(&net->W, net->np);
  A(&net->G, net->np);
  A(&net->M1, net->np);
  A(&net->M2, net->np);
  for (int l = 0; l < kLayers; ++l) {
    A(&net->wt[l], (size_t)kLayerDefs[l].cout * kpad(kLayerDefs[l].cin));
    A(&net->wb[l], (size_t)kLayerDefs[l].cin * kpad(kLayerDefs[l].cout));
  }
  for (int t = 0; t < T_COUNT; ++t) {
    const size_t count = (size_t)level_vox(net, kTensors[t].level) * max_batch * kTensors[t].channels;
    A(&net->act[t], count);
    A(&net->grad[t], count);
  }
  A(&net->part, (size_t)kWgradGrid * 16 * kpad(16));
  A(&net->bpart, (size_t)kWgradGrid * 16);
  A(&net->lpart, (size_t)kLossGrid);
  A(&net->y32, (size_t)level_vox(net, 0) * max_batch);
  A(&net->loss_d, 1);
  A(&net->ss, XAMG_MAX_RHS);
  A(&net->ss_part, (size_t)kMaxGrid * XAMG_MAX_RHS);
  if (rc == XAMG_OK && cudaMemset(net->W, 0, net->np * sizeof(float)) != cudaSuccess) rc = XAMG_ERR_CUDA;
  if (rc == XAMG_OK && cudaMemset(net->M1, 0, net->np * sizeof(float)) != cudaSuccess) rc = XAMG_ERR_CUDA;
  if (rc == XAMG_OK && cudaMemset(net->M2, 0, net->np * sizeof(float)) != cudaSuccess) rc = XAMG_ERR_CUDA;
  if (rc != XAMG_OK) {
    xamg_net_destroy(net);
    return rc;
  }
  *out = net;
  return XAMG_OK;
}

void xamg_net_destroy(xamg_net *net) {
  if (!net) return;
  for (void *p : net->owned) cudaFree(p);
  delete net;
}

int xamg_net_set_params(xamg_net *net, const float *params) {
  if (!net || !params) return XAMG_ERR_INVALID_ARG;
  NCK(cudaSetDevice(net->device));
  NCK(cudaMemcpy(net->W, params, net->np * sizeof(float), cudaMemcpyHostToDevice));
  NCK(cudaMemset(net->M1, 0, net->np * sizeof(float)));
  NCK(cudaMemset(net->M2, 0, net->np * sizeof(float)));
  net->steps = 0;
  net->weights_fresh = false;
  return XAMG_OK;
}

int xamg_net_get_params(const xamg_net *net, float *params) {
  if (!net || !params) return XAMG_ERR_INVALID_ARG;
  NCK(cudaSetDevice(net->device));
  NCK(cudaMemcpy(params, net->W, net->np * sizeof(float), cudaMemcpyDeviceToHost));
  return XAMG_OK;
}

int xamg_net_forward(xamg_net *net, const float *inp, float *out, int32_t batch, void *stream) {
  NRET(check_net(net, batch));
  if (!inp || !out) return XAMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  NCK(cudaSetDevice(net->device));
  NRET(refresh_weights(net, st));
  NRET(pack_input(net, inp, nullptr, batch, st));
  NRET(forward(net, batch, out, st));
  NCK(cudaStreamSynchronize(st));
  return XAMG_OK;
}

namespace {
int check_loss(const xamg_net_loss *lo) {
  if (lo && lo->kind != XAMG_NET_LOSS_MSE && lo->kind != XAMG_NET_LOSS_ENERGY) return XAMG_ERR_INVALID_ARG;
  return XAMG_OK;
}
}  // namespace

int xamg_net_loss_grad(xamg_net *net, const float *inp, const float *target, int32_t batch,
                       const xamg_net_loss *lo, float *loss, float *grad, void *stream) {
  NRET(check_net(net, batch));
  NRET(check_loss(lo));
  if (!inp || !target) return XAMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  NCK(cudaSetDevice(net->device));
  NRET(refresh_weights(net, st));
  NRET(pack_input(net, inp, nullptr, batch, st));
  NRET(forward(net, batch, net->y32, st));
  NRET(loss_and_output_grad(net, inp, target, nullptr, lo ? lo->sample_weight : nullptr,
                            lo ? lo->kind : XAMG_NET_LOSS_MSE, batch, st));
  NRET(backward(net, batch, st));
  if (grad) NCK(cudaMemcpyAsync(grad, net->G, net->np * sizeof(float), cudaMemcpyDeviceToHost, st));
  return read_loss(net, loss, st);
}

int xamg_net_train_step(xamg_net *net, const float *inp, const float *target, int64_t nsamples, const int32_t *idx,
                        int32_t batch, const xamg_net_loss *lo, const xamg_adam *opt, float *loss, void *stream) {
  NRET(check_net(net, batch));
  NRET(check_loss(lo));
  if (!inp || !target || !idx || !opt || nsamples < 1 || !(opt->lr > 0.0f) ||
      !(opt->beta1 >= 0.0f && opt->beta1 < 1.0f) || !(opt->beta2 >= 0.0f && opt->beta2 < 1.0f) ||
      !(opt->eps > 0.0f))
    return XAMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  NCK(cudaSetDevice(net->device));
  {  // the kernels gather through idx: check every index before any launch
    std::vector<int32_t> hidx(batch);
    NCK(cudaMemcpyAsync(hidx.data(), idx, batch * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NCK(cudaStreamSynchronize(st));
    for (int32_t v : hidx)
      if (v < 0 || v >= nsamples) return XAMG_ERR_INVALID_ARG;
  }
  NRET(refresh_weights(net, st));
  NRET(pack_input(net, inp, idx, batch, st));
  NRET(forward(net, batch, net->y32, st));
  NRET(loss_and_output_grad(net, inp, target, idx, lo ? lo->sample_weight : nullptr,
                            lo ? lo->kind : XAMG_NET_LOSS_MSE, batch, st));
  NRET(backward(net, batch, st));
  const int t = net->steps + 1;
  const float c1 = 1.0f - std::pow(opt->beta1, (float)t), c2 = 1.0f - std::pow(opt->beta2, (float)t);
  k_adam<<<(int)cdiv(net->np, 256), 256, 0, st>>>(net->W, net->G, net->M1, net->M2, net->np, opt->lr, opt->beta1,
                                                   opt->beta2, opt->eps, c1, c2);
  ++g_launches;
  NCK(cudaGetLastError());
  net->steps = t;
  net->weights_fresh = false;
  return loss ? read_loss(net, loss, st) : XAMG_OK;
}

int xamg_net_predict_x0(xamg_net *net, const double *B, const float *logk, double out_scale, double *X0,
                        int32_t m, void *stream) {
  NRET(check_net(net, m));
  if (!B || !logk || !X0 || m > XAMG_MAX_RHS || !std::isfinite(out_scale)) return XAMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  NCK(cudaSetDevice(net->device));
  const int64_t n = level_vox(net, 0);
  const int grid = coldot_rt_grid(n, m);
  if (grid > kMaxGrid) return XAMG_ERR_INVALID_ARG;
  launch_coldot_rt(n, m, B, B, net->ss_part, grid, st);
  launch_reduce_rt(m, net->ss_part, grid, net->ss, st);
  NRET(refresh_weights(net, st));
  k_pack_rhs<<<(int)cdiv(n, 32), dim3(32, 8), 0, st>>>(B, m, net->ss, n, logk, net->act[T_X]);
  ++g_launches;
  NCK(cudaGetLastError());
  NRET(forward(net, m, net->y32, st));
  k_unpack_x0<<<(int)cdiv(n, 32), dim3(32, 8), 0, st>>>(net->y32, m, net->ss, n, out_scale, X0);
  ++g_launches;
  NCK(cudaGetLastError());
  return XAMG_OK;
}

// ---- single layers (device buffers; temporaries are allocated per call) ----
int xamg_conv3d_bf16(const uint16_t *in, const uint16_t *mask, const float *w, const float *bias, uint16_t *out,
                     int32_t batch, int32_t N, int32_t cin, int32_t cout, int32_t relu, int32_t adjoint,
                     void *stream) {
  const bool ok_c = (cin == 8 || cin == 16) && (cout == 8 || cout == 16);
  if (!in || !w || !out || !ok_c || batch < 1 || N < 1 || N > 1024 || (adjoint && bias))
    return XAMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  bf16 *wk = nullptr;
  const size_t wlen = adjoint ? (size_t)cin * kpad(cout) : (size_t)cout * kpad(cin);
  NCK(cudaMallocAsync((void **)&wk, wlen * sizeof(bf16), st));
  cudaError_t e = prep_weights(w, adjoint ? nullptr : wk, adjoint ? wk : nullptr, cin, cout, st);
  if (e == cudaSuccess) {
    if (adjoint)
      e = conv(cout, cin, relu != 0, (const bf16 *)in, (const bf16 *)mask, wk, nullptr, (bf16 *)out, batch, N, st);
    else
      e = conv(cin, cout, relu != 0, (const bf16 *)in, (const bf16 *)mask, wk, bias, (bf16 *)out, batch, N, st);
  }
  cudaError_t e2 = cudaFreeAsync(wk, st);
  cudaError_t e3 = cudaStreamSynchronize(st);
  if (e != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return XAMG_ERR_CUDA;
  return XAMG_OK;
}

int xamg_conv3d_bf16_wgrad(const uint16_t *in, const uint16_t *gout, const uint16_t *act, float *dw, float *db,
                           int32_t batch, int32_t N, int32_t cin, int32_t cout, void *stream) {
  const bool ok_c = (cin == 8 || cin == 16) && (cout == 8 || cout == 16);
  if (!in || !gout || !dw || !db || !ok_c || batch < 1 || N < 1 || N > 1024) return XAMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float *part = nullptr, *bpart = nullptr;
  NCK(cudaMallocAsync((void **)&part, (size_t)kWgradGrid * cout * kpad(cin) * sizeof(float), st));
  cudaError_t e = cudaMallocAsync((void **)&bpart, (size_t)kWgradGrid * cout * sizeof(float), st);
  if (e == cudaSuccess)
    e = wgrad(cin, cout, (const bf16 *)in, (const bf16 *)gout, (const bf16 *)act, part, bpart, dw, db, batch, N, st);
  cudaError_t e2 = cudaFreeAsync(part, st);
  if (bpart) cudaFreeAsync(bpart, st);
  cudaError_t e3 = cudaStreamSynchronize(st);
  if (e != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return XAMG_ERR_CUDA;
  return XAMG_OK;
}

}  // extern "C"
