// kernels.cuh -- device kernels of the solve phase (sm_103a).
//
// Blocks of NV columns are n x NV row-major (element (i, c) at i*NV + c); NV
// is a compile-time power of two in {1, 2, 4, 8, 16, 32}, the counterpart of
// the paper's compile-time RHS count (Sec. 2.3: "The number of RHSs is also
// given as a template parameter").  The block scalar TB is double (the FP64
// solve) or float (the reduced-precision preconditioner of paper Sec. 2.3,
// "mixed-precision"); the matrix values TV are double, float, or bf16 with a
// per-row FP32 scale.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace xamg {

constexpr int kBlock = 256;  // threads per block of the row and element kernels
constexpr int kWarps = kBlock / 32;
// `slices` codes of the row launchers for FP64 blocks of 8 or more columns
// (k_rows, rows_vec): the narrow split with its row loop software-pipelined
// (kPipeNarrow), and the narrow split and its pipelined form with two
// adjacent columns per lane, so that a warp holds two rows (kNarrow2,
// kPipeNarrow2)
constexpr int kPipeNarrow = 300, kNarrow2 = 310, kPipeNarrow2 = 311;

// One fused row operation (paper Sec. 2.2-2.3: the "blas2" SpMV-like group,
// here with m columns at once).  For every row i of the sparse matrix M and
// column c:
//   v      = init[i,c] (or 0)  +/-  sum_k M_ik * src[k,c]      (sign: template NEG)
//   y[i,c] = v                                                 (if y)
//   dn     = c1 * dp[i,c] + w[i] * v
//   dnext[i,c] = dn
//   x[i,c] += dp[i,c] and/or dn
//   partial dots over the block's rows, written to partials[block*NV + c]
// which of these apply is the kernel's compile-time epilogue (enum Epi).
// All pointers except rowptr/col/val/src may alias each other only at the
// same element (own-row reads before own-row writes); src never aliases an
// output.  Dots are always accumulated in FP64 (dot_u, dot_u2 are FP64
// blocks).
template <class TB>
struct RowOpT {
  int n;
  const int32_t *rowptr;
  const int32_t *col;
  const void *val;       // matrix values (TV)
  const float *rscale;   // per-row scale of bf16 values
  const uint16_t *colw;     // 16-bit column offsets (Bf16Idx16, F32Idx16; see Seg16)
  const uint32_t *rowmeta;  // per row: segment boundaries (Seg16)
  const int32_t *tbase;     // per tile of kSegTile rows: kSegs segment bases (Seg16)
  const TB *src;
  const TB *init;
  TB *y;
  const TB *dp;
  const TB *w;
  TB c1;
  TB *dnext;
  TB *x;
  const double *dot_u;
  const double *dot_u2;
  double *partials;
  double *partials2;  // second reduction (EPI_Y_DOT2: v . v; EPI_XLAST_DOT2: dot_u2 . x)
};
using RowOp = RowOpT<double>;
using RowOpF = RowOpT<float>;

// Sum over the lanes of a warp that hold the same column c = lane % NV, in a
// fixed xor-tree order; the result is valid in every lane.
template <int NV>
__device__ __forceinline__ double warp_colsum(double v) {
#pragma unroll
  for (int o = NV; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-level per-column reduction of `v` (each thread's column is
// threadIdx.x % NV); thread c < NV of the block writes out[blockIdx.x*NV + c].
template <int NV>
__device__ __forceinline__ void block_colsum_store(double v, double *out) {
  __shared__ double red[kWarps][32];
  v = warp_colsum<NV>(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < NV) red[warp][lane] = v;
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
    out[(size_t)blockIdx.x * NV + threadIdx.x] = s;
  }
}

// Block-level per-column reduction when lane g of each group of G = NV/VEC
// lanes holds the partial sums of columns g*VEC .. g*VEC+VEC-1: a fixed
// xor tree over the groups of a warp, then thread c < NV adds the warps in
// order and writes out[blockIdx.x*NV + c].
template <int NV, int VEC>
__device__ __forceinline__ void block_colsum_store_vec(const double (&v)[VEC], double *out) {
  if constexpr (VEC == 1) {
    block_colsum_store<NV>(v[0], out);
  } else {
    constexpr int G = NV / VEC;
    __shared__ double red[kWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      s[k] = v[k];
#pragma unroll
      for (int o = G; o < 32; o <<= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    }
    if (lane < G) {
#pragma unroll
      for (int k = 0; k < VEC; ++k) red[warp][lane * VEC + k] = s[k];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) t += red[w][threadIdx.x];
      out[(size_t)blockIdx.x * NV + threadIdx.x] = t;
    }
  }
}

// Epilogue arithmetic.  FP64 blocks fuse it into FMAs (their bound is the
// FP64 issue rate).  FP32 blocks round once per operation in the order the
// Chebyshev recurrence is written -- t = sum_k m_ik x_k (a fused multiply-add
// chain from zero in storage order), v = init +/- t, d = c1 d + w v,
// x = x + d -- so that the reduced-precision cycle rounds at the points of its
// definition, not at points the fusion would choose; the FP32 path is bound
// by memory, so the extra operations cost nothing.
template <class TB>
__device__ __forceinline__ TB ep_add(TB a, TB b) {
  if constexpr (sizeof(TB) == 4) return __fadd_rn(a, b);
  else return a + b;
}
template <class TB>
__device__ __forceinline__ TB ep_mul(TB a, TB b) {
  if constexpr (sizeof(TB) == 4) return __fmul_rn(a, b);
  else return a * b;
}
// c1 d + w v
template <class TB>
__device__ __forceinline__ TB ep_dn(TB c1, TB d, TB w, TB v) {
  if constexpr (sizeof(TB) == 4) return __fadd_rn(__fmul_rn(c1, d), __fmul_rn(w, v));
  else return fma(c1, d, w * v);
}
// x + d + (c1 d + w v): FP32 as (x + d) + (c1 d + w v); FP64 as
// (x + (1 + c1) d) + w v, two FMAs (1 + c1 is the same for every element)
template <class TB>
__device__ __forceinline__ TB ep_xlast(TB x, TB c1, TB d, TB w, TB v) {
  if constexpr (sizeof(TB) == 4) return __fadd_rn(__fadd_rn(x, d), ep_dn(c1, d, w, v));
  else return fma(w, v, fma(c1 + (TB)1, d, x));
}
// The row's value from its product sum t (accumulated from zero, with the
// sign of NEG already applied) and, when has_init, its init value `in`:
// in + s t with the row scale s of scaled values, else in + t.  FP64 blocks
// with unscaled values start their sums from the init value instead.
template <class TB, bool SCALED>
__device__ __forceinline__ TB ep_combine(TB t, TB s, bool has_init, TB in) {
  if constexpr (SCALED) {
    if constexpr (sizeof(TB) == 4) {
      const TB st = __fmul_rn(s, t);
      return has_init ? __fadd_rn(in, st) : st;
    } else {
      return fma(s, t, has_init ? in : (TB)0);
    }
  } else {
    return has_init ? ep_add(in, t) : t;
  }
}
// FP64 blocks with unscaled values begin the product sum at the init value.
template <class TB, bool SCALED>
__device__ __forceinline__ constexpr bool sum_from_init() {
  return !SCALED && sizeof(TB) == 8;
}

// Epilogue of a row kernel, fixed at compile time so that no floating-point
// operation of an unused branch is executed (v is the row's product sum):
enum Epi : int {
  EPI_Y = 0,       // y = v
  EPI_Y_D0,        // y = v ; dnext = w v                         (first smoother step)
  EPI_Y_DN,        // y = v ; dnext = c1 dp + w v                 (Chebyshev step, x untouched)
  EPI_Y_XDP,       // y = v ; x += dp                             (last pre-smoothing step)
  EPI_MID,         // y = v ; dnext = c1 dp + w v ; x += dp       (middle Chebyshev step)
  EPI_XLAST,       // x += dp + (c1 dp + w v), as (x + (1+c1) dp) + w v  (last post-smoothing step)
  EPI_XLAST_DOT,   // EPI_XLAST and partial dot_u . x_new
  EPI_Y_DOT,       // y = v ; partial dot_u . v
  EPI_Y_DOT2,      // y = v ; partial dot_u . v (if dot_u) and v . v
  EPI_XLAST_DOT2,  // EPI_XLAST and partials dot_u . x_new, dot_u2 . x_new
  EPI_COUNT
};

// dpv, wv, xv, du, du2 are the own-row operands loaded before the product loop.
template <class TB, int NV, int EPI>
__device__ __forceinline__ void row_epilogue(const RowOpT<TB> &op, int64_t i, int c, TB acc,
                                             TB dpv, TB wv, TB xv, double du, double du2,
                                             double &dsum, double &dsum2) {
  const int64_t e = i * NV + c;
  if constexpr (EPI != EPI_XLAST && EPI != EPI_XLAST_DOT && EPI != EPI_XLAST_DOT2) {
    if (op.y) op.y[e] = acc;
  }
  if constexpr (EPI == EPI_Y_D0) op.dnext[e] = ep_mul(wv, acc);
  if constexpr (EPI == EPI_Y_DN) op.dnext[e] = ep_dn(op.c1, dpv, wv, acc);
  if constexpr (EPI == EPI_Y_XDP) op.x[e] = ep_add(xv, dpv);
  if constexpr (EPI == EPI_MID) {
    op.dnext[e] = ep_dn(op.c1, dpv, wv, acc);
    op.x[e] = ep_add(xv, dpv);
  }
  if constexpr (EPI == EPI_XLAST || EPI == EPI_XLAST_DOT || EPI == EPI_XLAST_DOT2) {
    const TB xn = ep_xlast(xv, op.c1, dpv, wv, acc);
    op.x[e] = xn;
    if constexpr (EPI == EPI_XLAST_DOT || EPI == EPI_XLAST_DOT2) dsum = fma(du, (double)xn, dsum);
    if constexpr (EPI == EPI_XLAST_DOT2) dsum2 = fma(du2, (double)xn, dsum2);
  }
  if constexpr (EPI == EPI_Y_DOT) dsum = fma(du, (double)acc, dsum);
  if constexpr (EPI == EPI_Y_DOT2) {
    if (op.dot_u) dsum = fma(du, (double)acc, dsum);
    dsum2 = fma((double)acc, (double)acc, dsum2);
  }
}

template <int EPI>
__device__ __forceinline__ constexpr bool epi_has_dot() {
  return EPI == EPI_XLAST_DOT || EPI == EPI_Y_DOT || EPI == EPI_Y_DOT2 || EPI == EPI_XLAST_DOT2;
}

// Own-row operands of the epilogue.
template <class TB, int NV, int EPI>
__device__ __forceinline__ void row_operands(const RowOpT<TB> &op, int64_t i, int c, TB &dpv,
                                             TB &wv, TB &xv, double &du, double &du2) {
  const int64_t e = i * NV + c;
  constexpr bool xlast = EPI == EPI_XLAST || EPI == EPI_XLAST_DOT || EPI == EPI_XLAST_DOT2;
  if constexpr (EPI == EPI_Y_DN || EPI == EPI_Y_XDP || EPI == EPI_MID || xlast) dpv = op.dp[e];
  if constexpr (EPI == EPI_Y_D0 || EPI == EPI_Y_DN || EPI == EPI_MID || xlast) wv = op.w[i];
  if constexpr (EPI == EPI_Y_XDP || EPI == EPI_MID || xlast) xv = op.x[e];
  if constexpr (EPI == EPI_XLAST_DOT || EPI == EPI_Y_DOT || EPI == EPI_XLAST_DOT2) du = op.dot_u[e];
  if constexpr (EPI == EPI_XLAST_DOT2) du2 = op.dot_u2[e];
  if constexpr (EPI == EPI_Y_DOT2) du = op.dot_u ? op.dot_u[e] : 0.0;
}

// Matrix value storage: TV = double / float (value as stored) or bf16 (value
// relative to the row's FP32 scale, applied once per row).
template <class TV> struct ValueLoad;
template <> struct ValueLoad<double> {
  using T = double;  // storage type
  static constexpr bool scaled = false;
  static constexpr bool idx16 = false;
  __device__ __forceinline__ static double get(const void *v, int k) {
    return __ldg(static_cast<const double *>(v) + k);
  }
};
template <> struct ValueLoad<float> {
  using T = float;
  static constexpr bool scaled = false;
  static constexpr bool idx16 = false;
  __device__ __forceinline__ static float get(const void *v, int k) {
    return __ldg(static_cast<const float *>(v) + k);
  }
};
template <> struct ValueLoad<__nv_bfloat16> {
  using T = __nv_bfloat16;
  static constexpr bool scaled = true;
  static constexpr bool idx16 = false;
  __device__ __forceinline__ static float get(const void *v, int k) {
    return __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(v) + k));
  }
};
// 16-bit column indices (paper Sec. 2.3: CSR index types reduced to
// uint16_t), in a segmented form that 3-D stencil rows (three planes far
// apart) and Galerkin rows fit: the rows are cut into tiles of kSegTile
// consecutive rows, and each tile has up to kSegs segment bases b_s such that
// every column of its rows lies in [b_s, b_s + 65535] for the segment s of
// that entry.  Entry k of row i stores col - b_s as uint16; rowmeta[i] packs
// the row's segment boundaries e1 | e2 << 10 | e3 << 20 (entries before e1
// are in segment 0, before e2 in segment 1, before e3 in segment 2, the rest
// in segment 3; a field of 1023 means no boundary), and tbase[t * kSegs + s]
// is b_s of tile t.  Decoding is exact.
constexpr int kSegTile = 32, kSegs = 4, kSegNone = 1023;
__device__ __forceinline__ int seg16_col(const int4 &b, uint32_t meta, int k, uint16_t off) {
  const int e1 = (int)(meta & 1023u), e2 = (int)((meta >> 10) & 1023u), e3 = (int)((meta >> 20) & 1023u);
  const int base = k < e1 ? b.x : k < e2 ? b.y : k < e3 ? b.z : b.w;
  return base + (int)off;
}
// bf16 values with 16-bit column indices.
struct Bf16Idx16 {};
template <> struct ValueLoad<Bf16Idx16> {
  using T = __nv_bfloat16;
  static constexpr bool scaled = true;
  static constexpr bool idx16 = true;
  __device__ __forceinline__ static float get(const void *v, int k) {
    return __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(v) + k));
  }
};
// FP32 values with the same 16-bit column indices.
struct F32Idx16 {};
template <> struct ValueLoad<F32Idx16> {
  using T = float;
  static constexpr bool scaled = false;
  static constexpr bool idx16 = true;
  __device__ __forceinline__ static float get(const void *v, int k) {
    return __ldg(static_cast<const float *>(v) + k);
  }
};

template <bool NEG, class TB>
__device__ __forceinline__ TB fmadd(TB a, TB x, TB acc) {
  return NEG ? fma(-a, x, acc) : fma(a, x, acc);
}


// Exactly `rem` (1..7) further products of one chunk, in order.
template <bool NEG, class TB>
__device__ __forceinline__ TB tail_fma(int rem, const TB (&as)[8], const TB (&xs)[8], TB acc) {
  switch (rem) {
    case 7: acc = fmadd<NEG>(as[0], xs[0], acc); acc = fmadd<NEG>(as[1], xs[1], acc);
            acc = fmadd<NEG>(as[2], xs[2], acc); acc = fmadd<NEG>(as[3], xs[3], acc);
            acc = fmadd<NEG>(as[4], xs[4], acc); acc = fmadd<NEG>(as[5], xs[5], acc);
            acc = fmadd<NEG>(as[6], xs[6], acc); break;
    case 6: acc = fmadd<NEG>(as[0], xs[0], acc); acc = fmadd<NEG>(as[1], xs[1], acc);
            acc = fmadd<NEG>(as[2], xs[2], acc); acc = fmadd<NEG>(as[3], xs[3], acc);
            acc = fmadd<NEG>(as[4], xs[4], acc); acc = fmadd<NEG>(as[5], xs[5], acc); break;
    case 5: acc = fmadd<NEG>(as[0], xs[0], acc); acc = fmadd<NEG>(as[1], xs[1], acc);
            acc = fmadd<NEG>(as[2], xs[2], acc); acc = fmadd<NEG>(as[3], xs[3], acc);
            acc = fmadd<NEG>(as[4], xs[4], acc); break;
    case 4: acc = fmadd<NEG>(as[0], xs[0], acc); acc = fmadd<NEG>(as[1], xs[1], acc);
            acc = fmadd<NEG>(as[2], xs[2], acc); acc = fmadd<NEG>(as[3], xs[3], acc); break;
    case 3: acc = fmadd<NEG>(as[0], xs[0], acc); acc = fmadd<NEG>(as[1], xs[1], acc);
            acc = fmadd<NEG>(as[2], xs[2], acc); break;
    case 2: acc = fmadd<NEG>(as[0], xs[0], acc); acc = fmadd<NEG>(as[1], xs[1], acc); break;
    case 1: acc = fmadd<NEG>(as[0], xs[0], acc); break;
    default: break;
  }
  return acc;
}

// Small vectors of VEC consecutive block columns held by one lane, loaded and
// stored with one 8/16-byte access (VEC = 1, 2, 4).
template <class T, int VEC>
struct Vec {
  T v[VEC];
};
template <class T, int VEC>
__device__ __forceinline__ Vec<T, VEC> vload(const T *p) {
  Vec<T, VEC> r;
  if constexpr (VEC == 1) {
    r.v[0] = *p;
  } else if constexpr (sizeof(T) * VEC == 32) {
    // two 16-byte halves
    const Vec<T, VEC / 2> lo = vload<T, VEC / 2>(p), hi = vload<T, VEC / 2>(p + VEC / 2);
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) {
      r.v[k] = lo.v[k];
      r.v[k + VEC / 2] = hi.v[k];
    }
  } else if constexpr (sizeof(T) * VEC == 16) {
    if constexpr (sizeof(T) == 4) {
      const float4 q = *reinterpret_cast<const float4 *>(p);
      r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
    } else {
      const double2 q = *reinterpret_cast<const double2 *>(p);
      r.v[0] = q.x; r.v[1] = q.y;
    }
  } else {
    static_assert(sizeof(T) * VEC == 8, "8- or 16-byte vectors");
    const float2 q = *reinterpret_cast<const float2 *>(p);
    r.v[0] = q.x; r.v[1] = q.y;
  }
  return r;
}
template <class T, int VEC>
__device__ __forceinline__ Vec<T, VEC> vldg(const T *p) {
  Vec<T, VEC> r;
  if constexpr (VEC == 1) {
    r.v[0] = __ldg(p);
  } else if constexpr (sizeof(T) * VEC == 32) {
    const Vec<T, VEC / 2> lo = vldg<T, VEC / 2>(p), hi = vldg<T, VEC / 2>(p + VEC / 2);
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) {
      r.v[k] = lo.v[k];
      r.v[k + VEC / 2] = hi.v[k];
    }
  } else if constexpr (sizeof(T) * VEC == 16) {
    if constexpr (sizeof(T) == 4) {
      const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
      r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
    } else {
      const double2 q = __ldg(reinterpret_cast<const double2 *>(p));
      r.v[0] = q.x; r.v[1] = q.y;
    }
  } else {
    const float2 q = __ldg(reinterpret_cast<const float2 *>(p));
    r.v[0] = q.x; r.v[1] = q.y;
  }
  return r;
}
template <class T, int VEC>
__device__ __forceinline__ void vstore(T *p, const Vec<T, VEC> &r) {
  if constexpr (VEC == 1) {
    *p = r.v[0];
  } else if constexpr (sizeof(T) * VEC == 32) {
    Vec<T, VEC / 2> lo, hi;
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) {
      lo.v[k] = r.v[k];
      hi.v[k] = r.v[k + VEC / 2];
    }
    vstore<T, VEC / 2>(p, lo);
    vstore<T, VEC / 2>(p + VEC / 2, hi);
  } else if constexpr (sizeof(T) * VEC == 16) {
    if constexpr (sizeof(T) == 4)
      *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    else
      *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
  } else {
    *reinterpret_cast<float2 *>(p) = make_float2(r.v[0], r.v[1]);
  }
}

// The epilogue of the vector row kernels for row i (e = i NV + c0): the
// product sum acc (from zero, or from the init value for FP64 unscaled
// values) becomes v, and v is written and combined as enum Epi says.
template <class TB, class TV, int NV, int VEC, int EPI>
__device__ __forceinline__ void vec_epilogue(const RowOpT<TB> &op, int64_t i, int64_t e, Vec<TB, VEC> acc,
                                             const Vec<TB, VEC> &in0, const Vec<TB, VEC> &dpv, TB wv,
                                             const Vec<TB, VEC> &xv, TB s, double (&dsum)[VEC],
                                             double (&dsum2)[VEC]) {
  using VL = ValueLoad<TV>;
  using V = Vec<TB, VEC>;
  constexpr bool xlast = EPI == EPI_XLAST || EPI == EPI_XLAST_DOT || EPI == EPI_XLAST_DOT2;
  // s: the row scale of scaled (bf16) values, loaded before the product loop
  if constexpr (!sum_from_init<TB, VL::scaled>()) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc.v[v] = ep_combine<TB, VL::scaled>(acc.v[v], s, op.init != nullptr, in0.v[v]);
  }
  // epilogue (see enum Epi)
  if constexpr (!xlast) {
    if (op.y) vstore<TB, VEC>(op.y + e, acc);
  }
  if constexpr (EPI == EPI_Y_D0 || EPI == EPI_Y_DN || EPI == EPI_MID) {
    V dn;
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      dn.v[v] = EPI == EPI_Y_D0 ? ep_mul(wv, acc.v[v]) : ep_dn(op.c1, dpv.v[v], wv, acc.v[v]);
    vstore<TB, VEC>(op.dnext + e, dn);
  }
  if constexpr (EPI == EPI_Y_XDP || EPI == EPI_MID) {
    V xn;
#pragma unroll
    for (int v = 0; v < VEC; ++v) xn.v[v] = ep_add(xv.v[v], dpv.v[v]);
    vstore<TB, VEC>(op.x + e, xn);
  }
  if constexpr (xlast) {
    V xn;
#pragma unroll
    for (int v = 0; v < VEC; ++v) xn.v[v] = ep_xlast(xv.v[v], op.c1, dpv.v[v], wv, acc.v[v]);
    vstore<TB, VEC>(op.x + e, xn);
    if constexpr (EPI == EPI_XLAST_DOT || EPI == EPI_XLAST_DOT2) {
#pragma unroll
      for (int v = 0; v < VEC; ++v) dsum[v] = fma(op.dot_u[e + v], (double)xn.v[v], dsum[v]);
    }
    if constexpr (EPI == EPI_XLAST_DOT2) {
#pragma unroll
      for (int v = 0; v < VEC; ++v) dsum2[v] = fma(op.dot_u2[e + v], (double)xn.v[v], dsum2[v]);
    }
  }
  if constexpr (EPI == EPI_Y_DOT) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) dsum[v] = fma(op.dot_u[e + v], (double)acc.v[v], dsum[v]);
  }
  if constexpr (EPI == EPI_Y_DOT2) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      if (op.dot_u) dsum[v] = fma(op.dot_u[e + v], (double)acc.v[v], dsum[v]);
      dsum2[v] = fma((double)acc.v[v], (double)acc.v[v], dsum2[v]);
    }
  }
}

// Row kernel, S = 1.  A group of G = NV/VEC lanes owns one row (32/G rows per
// warp); lane g of the group holds the VEC adjacent columns g*VEC .. g*VEC+VEC-1
// and moves them with one 8/16-byte access, so a warp keeps 32/G rows' gathers
// in flight at once.  The group reads the row's column indices and values G
// at a time with one coalesced load each and passes them around with
// shuffles; all operand-row gathers of a chunk of eight entries are issued
// before their FMAs, so the dependent chain per row is row pointer ->
// index/value -> operand rows.  Each column's products are added in the row's
// storage order (no reduction adds), and a chunk's tail takes exactly as many
// FMAs as it has entries.  With scaled (bf16) values the products are summed
// first and the row scale applied once: v = init +/- s_i * sum_k q_ik x_k.
template <class TB, class TV, int NV, int VEC, int SL, bool NEG, int EPI, int XW = 1, bool COH = false,
          int CHX = 0, bool PIPE = false>
__device__ __forceinline__ void rows_vec(const RowOpT<TB> &op) {
  using VL = ValueLoad<TV>;
  using V = Vec<TB, VEC>;
  constexpr int G = NV / VEC;
  constexpr int RPW = 32 / (G * SL);
  // entries gathered per chunk: 8 for FP64 with one column per lane
  // (exact-count tails keep the FP64 FMA count at the algorithmic one); 4
  // for FP32 and for FP64 with two columns per lane, whose 16-byte gathers
  // already fill the registers; never more than the G lanes of a row group
  // hold, since a chunk's shuffles broadcast the group's own entries (narrow
  // blocks, m = 2..8, would otherwise spend most shuffles on empty slots)
  constexpr int CH0 = CHX > 0 ? CHX : (sizeof(TB) == 4 || VEC == 2 ? 4 : 8);
  constexpr int CH = CH0 < G ? CH0 : G;
  constexpr int K = 32 / G < 4 ? 32 / G : 4;  // entries each lane fetches per round
  constexpr bool xlast = EPI == EPI_XLAST || EPI == EPI_XLAST_DOT || EPI == EPI_XLAST_DOT2;
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  const int c0 = gl * VEC;
  const int sl = (lane / G) % SL;   // slice of the row
  const int grp = lane / (G * SL);  // row of the warp
  const int gbase = (lane / G) * G;
  // XW > 1 (a row already fills a warp): XW warps of a block share one row,
  // warp slice wx taking the entry rounds wx, wx + XW, ...; their partial
  // sums are added in a fixed order through shared memory, so the row loop is
  // block-uniform: block step b covers rows b * kWarps / XW + warp / XW
  static_assert(XW == 1 || RPW == 1, "warps per row need one row per warp");
  constexpr int RPB = kWarps / XW;
  const int wx = (threadIdx.x >> 5) % XW;
  const int64_t warp0 =
      XW == 1 ? (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5) : (int64_t)blockIdx.x * RPB;
  const int64_t wstride = XW == 1 ? (int64_t)gridDim.x * kWarps : (int64_t)gridDim.x * RPB;
  const int32_t *__restrict__ col = op.col;
  const TB *__restrict__ src = op.src;
  double dsum[VEC], dsum2[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) dsum[v] = dsum2[v] = 0.0;
  // a round of a row's column indices / values: slot q of lane g holds entry
  // kb + q*G + g
  auto load_cols = [&](int (&cl)[K], int start, int len, int kb) {
#pragma unroll
    for (int q = 0; q < K; ++q) cl[q] = kb + q * G + gl < len ? __ldg(col + start + kb + q * G + gl) : 0;
  };
  auto load_vals = [&](TB (&av)[K], int start, int len, int kb) {
#pragma unroll
    for (int q = 0; q < K; ++q)
      av[q] = kb + q * G + gl < len ? (TB)VL::get(op.val, start + kb + q * G + gl) : (TB)0;
  };
  // PIPE: software pipeline of the row loop (one warp per row group, 32-bit
  // indices).  While a row's operand rows are gathered, the next row's first
  // round of column indices and the row pointers of the row after it are
  // already in flight, so the dependent chain row pointer -> index -> operand
  // row costs one memory latency per row instead of three.  The sums are
  // those of the unpipelined loop, bit for bit.
  constexpr bool PF = PIPE && XW == 1 && !VL::idx16 && !COH;
  const int64_t rstep = wstride * RPW;
  int pf_s1 = 0, pf_l1 = 0, pf_s2 = 0, pf_l2 = 0;
  int pf_cl[K];
  if constexpr (PF) {
    const int64_t i0 = warp0 * RPW + grp;
    if (i0 < op.n) {
      pf_s1 = __ldg(op.rowptr + i0);
      pf_l1 = __ldg(op.rowptr + i0 + 1) - pf_s1;
    }
    if (i0 + rstep < op.n) {
      pf_s2 = __ldg(op.rowptr + i0 + rstep);
      pf_l2 = __ldg(op.rowptr + i0 + rstep + 1) - pf_s2;
    }
    load_cols(pf_cl, pf_s1, pf_l1, sl * G * K);
  }
  for (int64_t base = warp0 * RPW; base < op.n; base += rstep) {
    const int64_t i = base + (XW == 1 ? grp : (threadIdx.x >> 5) / XW);
    const bool valid = i < op.n;
    const int64_t e = i * NV + c0;
    int start = 0, len = 0;
    uint32_t meta = 0;
    int4 tb = make_int4(0, 0, 0, 0);
    V acc, dpv, xv, in0;
    TB wv = 0, rs = 1;
    int cl0[K];
    TB av0[K];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc.v[v] = dpv.v[v] = xv.v[v] = in0.v[v] = 0;
    if constexpr (PF) {
      start = pf_s1;
      len = pf_l1;
#pragma unroll
      for (int q = 0; q < K; ++q) cl0[q] = pf_cl[q];
      load_vals(av0, start, len, sl * G * K);
      pf_s1 = pf_s2;
      pf_l1 = pf_l2;
      load_cols(pf_cl, pf_s1, pf_l1, sl * G * K);
      pf_s2 = pf_l2 = 0;
      if (i + 2 * rstep < op.n) {
        pf_s2 = __ldg(op.rowptr + i + 2 * rstep);
        pf_l2 = __ldg(op.rowptr + i + 2 * rstep + 1) - pf_s2;
      }
    }
    if (valid) {
      if constexpr (!PF) {
        start = __ldg(op.rowptr + i);
        len = __ldg(op.rowptr + i + 1) - start;
      }
      if constexpr (VL::scaled) rs = (TB)__ldg(op.rscale + i);
      if constexpr (VL::idx16) {
        meta = __ldg(op.rowmeta + i);
        tb = __ldg(reinterpret_cast<const int4 *>(op.tbase) + i / kSegTile);
      }
      if (wx == 0) {
        // the init value: the start of the product sum (FP64, unscaled
        // values), else added after it; loaded before the product loop either
        // way, so that its latency hides behind the gathers
        if (sum_from_init<TB, VL::scaled>() && op.init && sl == 0) acc = vload<TB, VEC>(op.init + e);
        if (!sum_from_init<TB, VL::scaled>() && op.init && sl == 0) in0 = vload<TB, VEC>(op.init + e);
        if constexpr (EPI == EPI_Y_DN || EPI == EPI_Y_XDP || EPI == EPI_MID || xlast)
          dpv = vload<TB, VEC>(op.dp + e);
        if constexpr (EPI == EPI_Y_D0 || EPI == EPI_Y_DN || EPI == EPI_MID || xlast) wv = op.w[i];
        if constexpr (EPI == EPI_Y_XDP || EPI == EPI_MID || xlast) xv = vload<TB, VEC>(op.x + e);
      }
    }
    const int maxlen = (RPW == 1 && SL == 1) ? len : __reduce_max_sync(0xffffffffu, len);
    // slice sl takes rounds sl, sl + SL, ...; every slice runs the same number
    // of rounds (entries past the row's end are zeros), so the shuffles stay
    // warp-uniform
    for (int kb0 = 0; kb0 < maxlen; kb0 += G * K * SL * XW) {
      const int kb = kb0 + (sl + wx * SL) * G * K;
      // the group fetches G*K entries per round: slot q of lane g holds entry
      // kb + q*G + g (coalesced across the group for every q)
      int cl[K];
      TB av[K];
      if (PF && kb0 == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
          cl[q] = cl0[q];
          av[q] = av0[q];
        }
      } else if constexpr (VL::idx16) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int kl = kb + q * G + gl;
          const bool own = kl < len;
          cl[q] = own ? seg16_col(tb, meta, kl, __ldg(op.colw + start + kl)) : 0;
          av[q] = own ? (TB)VL::get(op.val, start + kl) : (TB)0;
        }
      } else {
        load_cols(cl, start, len, kb);
        load_vals(av, start, len, kb);
      }
      const int cnt = min(G * K, maxlen - kb0);  // uniform over the warp
#pragma unroll
      for (int q = 0; q < K; ++q) {
        if (q * G >= cnt) break;
        const int cq = min(G, cnt - q * G);
        const int kq = kb + q * G;
        for (int t = 0; t < cq; t += CH) {
          V xs[CH];
          TB as[CH];
#pragma unroll
          for (int u = 0; u < CH; ++u) {
            const int from = (gbase + t + u) & 31;
            const int cc = __shfl_sync(0xffffffffu, cl[q], from);
            as[u] = __shfl_sync(0xffffffffu, av[q], from);
            if (t + u < cq && kq + t + u < len) {
              // COH: the operand block was written earlier in the same kernel
              // (the fused coarse tail), so it is read through the coherent
              // path, not the read-only one
              xs[u] = COH ? vload<TB, VEC>(src + (int64_t)cc * NV + c0)
                          : vldg<TB, VEC>(src + (int64_t)cc * NV + c0);
            } else {
#pragma unroll
              for (int v = 0; v < VEC; ++v) xs[u].v[v] = 0;
            }
          }
          // entries past this row's own end carry a = x = 0 (rows of one warp
          // may differ in length)
          const int rem = min(CH, cq - t);
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            TB xv8[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) xv8[u] = xs[u].v[v];
            if (rem == CH) {
#pragma unroll
              for (int u = 0; u < CH; ++u) acc.v[v] = fmadd<NEG>(as[u], xv8[u], acc.v[v]);
            } else if constexpr (CH == 8) {
              acc.v[v] = tail_fma<NEG>(rem, as, xv8, acc.v[v]);
            } else {
#pragma unroll
              for (int u = 0; u < CH - 1; ++u)
                if (u < rem) acc.v[v] = fmadd<NEG>(as[u], xv8[u], acc.v[v]);
            }
          }
        }
      }
    }
    if constexpr (SL > 1) {
      // add the slices (fixed xor order); the sum is valid in every slice
#pragma unroll
      for (int v = 0; v < VEC; ++v)
#pragma unroll
        for (int o = G; o < G * SL; o <<= 1) acc.v[v] += __shfl_xor_sync(0xffffffffu, acc.v[v], o);
    }
    if constexpr (XW > 1) {
      // slice 0 (which holds the init value) adds slices 1 .. XW-1 in order
      __shared__ TB xw_red[kWarps][32 * VEC];
      const int w = threadIdx.x >> 5;
#pragma unroll
      for (int v = 0; v < VEC; ++v) xw_red[w][lane * VEC + v] = acc.v[v];
      __syncthreads();
      if (wx == 0) {
#pragma unroll
        for (int v = 0; v < VEC; ++v)
#pragma unroll
          for (int j = 1; j < XW; ++j) acc.v[v] += xw_red[w + j][lane * VEC + v];
      }
      __syncthreads();
    }
    if (valid && sl == 0 && wx == 0) vec_epilogue<TB, TV, NV, VEC, EPI>(op, i, e, acc, in0, dpv, wv, xv, rs, dsum, dsum2);
  }
  if constexpr (epi_has_dot<EPI>()) {
    if (EPI != EPI_Y_DOT2 || op.dot_u) block_colsum_store_vec<NV, VEC>(dsum, op.partials);
    if constexpr (EPI == EPI_Y_DOT2 || EPI == EPI_XLAST_DOT2) {
      __syncthreads();
      block_colsum_store_vec<NV, VEC>(dsum2, op.partials2);
    }
  }
}

// Asynchronous 4- and 8-byte global -> shared copies (no registers held while
// they are in flight).
__device__ __forceinline__ void cp_async_4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- FP32 row kernel with operand rows staged through shared memory ----
// 16-byte asynchronous global -> shared copy (cached in L1, like the
// read-only gathers it replaces), and the group bookkeeping of cp.async.
__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Depth of the operand ring (entries in flight per lane) and the per-warp
// window of staged column indices and values: 32 entries per row of the
// warp's row group on average (the host takes this kernel only for levels
// whose every aligned group of rows fits).
constexpr int kAsyncDepth = 8;
template <int NV>
__host__ __device__ constexpr int async_rows_per_warp() { return 32 / (NV / 4); }
template <int NV>
__host__ __device__ constexpr int async_window() { return 32 * async_rows_per_warp<NV>(); }
template <class TV, int NV>
__host__ __device__ constexpr int async_warp_bytes() {
  return kAsyncDepth * 32 * 16 + async_window<NV>() * 4 +
         ((async_window<NV>() + 2) * (int)sizeof(typename ValueLoad<TV>::T) + 15) / 16 * 16;
}

// The narrow split of FP32 blocks (NV >= 8: a group of G = NV/4 lanes per
// row, each lane holding 4 adjacent columns) with deeper memory parallelism.
// A warp's RPW consecutive rows own one contiguous range of the CSR arrays:
// the warp first copies that range's column indices and values into its
// shared window (cp.async, 32 consecutive entries per instruction), then each
// lane streams its 16-byte slice of the rows' operand rows through a private
// ring of kAsyncDepth slots in shared memory -- entry k + depth is in flight
// while entry k is multiplied -- so a lane keeps depth gathers outstanding
// without holding their registers.  Each lane reads back only what it copied
// itself, so the ring needs no synchronization beyond the lane's own
// cp.async groups.  The products are added in storage order from zero
// exactly as rows_vec's narrow split adds them, so the results are bitwise
// the same; the epilogue is vec_epilogue.
template <class TB, class TV, int NV, bool NEG, int EPI>
__device__ __forceinline__ void rows_async(const RowOpT<TB> &op, unsigned char *smem) {
  static_assert(sizeof(TB) == 4 && NV >= 8, "FP32 blocks of 8 or more columns");
  using VL = ValueLoad<TV>;
  using TS = typename VL::T;
  static_assert(!VL::idx16, "the staged kernel reads 32-bit column indices");
  constexpr int VEC = 4, G = NV / VEC, RPW = 32 / G, W = async_window<NV>(), D = kAsyncDepth;
  constexpr bool pairs = sizeof(TS) == 2;
  constexpr bool xlast = EPI == EPI_XLAST || EPI == EPI_XLAST_DOT || EPI == EPI_XLAST_DOT2;
  using V = Vec<TB, VEC>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane % G, c0 = gl * VEC, grp = lane / G;
  unsigned char *wsm = smem + warp * async_warp_bytes<TV, NV>();
  float4 *ring = reinterpret_cast<float4 *>(wsm);                  // [D][32]
  int32_t *s_col = reinterpret_cast<int32_t *>(wsm + D * 32 * 16);  // [W]
  TS *s_val = reinterpret_cast<TS *>(s_col + W);                   // [W + 2]
  const TS *gval = static_cast<const TS *>(op.val);
  const int64_t warp0 = (int64_t)blockIdx.x * kWarps + warp;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  double dsum[VEC], dsum2[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) dsum[v] = dsum2[v] = 0.0;
  for (int64_t base = warp0 * RPW; base < op.n; base += wstride * RPW) {
    const int64_t i = base + grp;
    const bool valid = i < op.n;
    const int64_t e = i * NV + c0;
    int start = 0, len = 0;
    V acc, dpv, xv, in0;
    TB wv = 0, rs = 1;
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc.v[v] = dpv.v[v] = xv.v[v] = in0.v[v] = 0;
    if (valid) {
      start = __ldg(op.rowptr + i);
      len = __ldg(op.rowptr + i + 1) - start;
      if constexpr (VL::scaled) rs = (TB)__ldg(op.rscale + i);
      if (op.init) in0 = vload<TB, VEC>(op.init + e);
      if constexpr (EPI == EPI_Y_DN || EPI == EPI_Y_XDP || EPI == EPI_MID || xlast)
        dpv = vload<TB, VEC>(op.dp + e);
      if constexpr (EPI == EPI_Y_D0 || EPI == EPI_Y_DN || EPI == EPI_MID || xlast) wv = op.w[i];
      if constexpr (EPI == EPI_Y_XDP || EPI == EPI_MID || xlast) xv = vload<TB, VEC>(op.x + e);
    }
    // the warp's contiguous range of entries [wb, we) (at most W: host rule)
    const int wb = (int)__reduce_min_sync(0xffffffffu, valid ? (unsigned)start : 0x7fffffffu);
    const int we = (int)__reduce_max_sync(0xffffffffu, valid ? (unsigned)(start + len) : 0u);
    const int vb = pairs ? (wb & ~1) : wb;
    __syncwarp();  // every lane is done with the previous window
    for (int k = wb + lane; k < we; k += 32) cp_async_4(s_col + (k - wb), op.col + k);
    if constexpr (pairs) {
      for (int k = vb + 2 * lane; k < we; k += 64) cp_async_4(s_val + (k - vb), gval + k);
    } else {
      for (int k = wb + lane; k < we; k += 32) cp_async_4(s_val + (k - vb), gval + k);
    }
    cp_async_commit();
    cp_async_wait_group<0>();
    __syncwarp();
    const int maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
    const int off = start - wb, voff = start - vb;
    // prologue: the first D entries of the lane's row in flight
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (d < len) cp_async_16(&ring[d * 32 + lane], op.src + (int64_t)s_col[off + d] * NV + c0);
      cp_async_commit();
    }
    for (int k = 0; k < maxlen; ++k) {
      cp_async_wait_group<D - 1>();  // entry k of this lane has landed
      const int slot = (k % D) * 32 + lane;
      if (k < len) {
        const float4 q = ring[slot];
        const TB a = pairs ? (TB)__bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(s_val + voff + k))
                           : (TB)s_val[voff + k];
        acc.v[0] = fmadd<NEG>(a, (TB)q.x, acc.v[0]);
        acc.v[1] = fmadd<NEG>(a, (TB)q.y, acc.v[1]);
        acc.v[2] = fmadd<NEG>(a, (TB)q.z, acc.v[2]);
        acc.v[3] = fmadd<NEG>(a, (TB)q.w, acc.v[3]);
      }
      // refill the slot just read (its products above consumed it first)
      if (k + D < len) cp_async_16(&ring[slot], op.src + (int64_t)s_col[off + k + D] * NV + c0);
      cp_async_commit();
    }
    cp_async_wait_group<0>();
    if (valid) vec_epilogue<TB, TV, NV, VEC, EPI>(op, i, e, acc, in0, dpv, wv, xv, rs, dsum, dsum2);
  }
  if constexpr (epi_has_dot<EPI>()) {
    if (EPI != EPI_Y_DOT2 || op.dot_u) block_colsum_store_vec<NV, VEC>(dsum, op.partials);
    if constexpr (EPI == EPI_Y_DOT2 || EPI == EPI_XLAST_DOT2) {
      __syncthreads();
      block_colsum_store_vec<NV, VEC>(dsum2, op.partials2);
    }
  }
}

// Row kernel with S > 1 slices per column (narrow blocks, m = 1): a group of
// G = NV*S lanes owns one row, lane -> column c = lane % NV and slice
// s = (lane / NV) % S; slice s takes the row's entries s, s+S, ... and the
// slices are added with shuffles.
template <class TB, class TV, int NV, int S, bool NEG, int EPI>
__device__ __forceinline__ void rows_sliced(const RowOpT<TB> &op) {
  using VL = ValueLoad<TV>;
  constexpr int G = NV * S;
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int c = lane % NV;
  const int s = (lane / NV) % S;
  const int grp = lane / G;
  const int64_t warp0 = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  const int32_t *__restrict__ col = op.col;
  const TB *__restrict__ src = op.src;
  double dsum = 0.0, dsum2 = 0.0;
  for (int64_t base = warp0 * RPW; base < op.n; base += wstride * RPW) {
    const int64_t i = base + grp;
    const bool valid = i < op.n;
    TB acc = 0, dpv = 0, wv = 0, xv = 0, rs = 1, iv = 0;
    double du = 0.0, du2 = 0.0;
    if (valid) {
      if (sum_from_init<TB, VL::scaled>() && op.init && s == 0) acc = op.init[i * NV + c];
      // the row scale and (for sums from zero) the init value, before the loop
      if constexpr (VL::scaled) rs = (TB)__ldg(op.rscale + i);
      if (!sum_from_init<TB, VL::scaled>() && op.init) iv = op.init[i * NV + c];
      row_operands<TB, NV, EPI>(op, i, c, dpv, wv, xv, du, du2);
      int k = __ldg(op.rowptr + i) + s;
      const int end = __ldg(op.rowptr + i + 1);
      for (; k + 3 * S < end; k += 4 * S) {
        const int k0 = __ldg(col + k), k1 = __ldg(col + k + S), k2 = __ldg(col + k + 2 * S),
                  k3 = __ldg(col + k + 3 * S);
        const TB a0 = VL::get(op.val, k), a1 = VL::get(op.val, k + S),
                 a2 = VL::get(op.val, k + 2 * S), a3 = VL::get(op.val, k + 3 * S);
        const TB x0 = __ldg(src + (int64_t)k0 * NV + c), x1 = __ldg(src + (int64_t)k1 * NV + c),
                 x2 = __ldg(src + (int64_t)k2 * NV + c), x3 = __ldg(src + (int64_t)k3 * NV + c);
        acc = fmadd<NEG>(a0, x0, acc);
        acc = fmadd<NEG>(a1, x1, acc);
        acc = fmadd<NEG>(a2, x2, acc);
        acc = fmadd<NEG>(a3, x3, acc);
      }
      for (; k < end; k += S) {
        const TB a = VL::get(op.val, k);
        acc = fmadd<NEG>(a, __ldg(src + (int64_t)__ldg(col + k) * NV + c), acc);
      }
    }
#pragma unroll
    for (int o = NV; o < G; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if constexpr (!sum_from_init<TB, VL::scaled>()) {
      if (valid) acc = ep_combine<TB, VL::scaled>(acc, rs, op.init != nullptr, iv);
    }
    if (valid && s == 0) row_epilogue<TB, NV, EPI>(op, i, c, acc, dpv, wv, xv, du, du2, dsum, dsum2);
  }
  if constexpr (epi_has_dot<EPI>()) {
    if (EPI != EPI_Y_DOT2 || op.dot_u) block_colsum_store<NV>(dsum, op.partials);
    if constexpr (EPI == EPI_Y_DOT2 || EPI == EPI_XLAST_DOT2) {
      __syncthreads();
      block_colsum_store<NV>(dsum2, op.partials2);
    }
  }
}

// ---- m = 1 stream kernel ----

// Shared-memory bytes of one warp's window of R entries: R column indices,
// then R + 2 values (bf16 values are copied in aligned pairs, so a window may
// start one entry early and end one entry late).
template <class TV, int R>
__host__ __device__ constexpr int stream_warp_bytes() {
  return ((R * 4 + (R + 2) * (int)sizeof(typename ValueLoad<TV>::T)) + 15) / 16 * 16;
}

// Row kernel for m = 1 (CSR-stream).  A warp owns 32 / LPR consecutive rows
// (lanes g*LPR .. g*LPR + LPR - 1 share row r0 + g); the rows' entries are one
// contiguous range of the CSR arrays, which the warp copies into its
// shared-memory window (R entries at a time) with per-lane asynchronous copies
// -- 32 consecutive entries per instruction -- and then the LPR lanes of each
// row walk the row's entries in the window with stride LPR, gathering the
// operands eight at a time (consecutive rows of a stencil-like matrix gather
// consecutive operands) and adding the products in order; the LPR partial
// sums are added in a fixed xor tree.  With LPR = 1 every FMA instruction of
// the walk carries one entry per lane and the epilogue runs on every lane,
// which matters at m = 1: the FP64 issue rate (about two FMAs per SM per
// clock) is as tight a bound as the HBM stream.  Wider LPR serve longer rows
// (the dense Galerkin levels), whose range per row would not fit a window.  A
// range longer than the window is walked window by window.  The next chunk's
// row pointers are read ahead.
template <class TB, class TV, int LPR, int R, bool NEG, int EPI>
__device__ __forceinline__ void rows_stream(const RowOpT<TB> &op, unsigned char *smem) {
  using VL = ValueLoad<TV>;
  using TS = typename VL::T;
  static_assert(!VL::idx16, "the stream kernel reads 32-bit column indices");
  constexpr bool pairs = sizeof(TS) == 2;
  constexpr int RPC = 32 / LPR;  // rows per chunk
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / LPR, p = lane % LPR;
  int32_t *s_col = reinterpret_cast<int32_t *>(smem + warp * stream_warp_bytes<TV, R>());
  TS *s_val = reinterpret_cast<TS *>(s_col + R);
  const int64_t n = op.n;
  const int64_t step = (int64_t)gridDim.x * kWarps * RPC;
  const TS *gval = static_cast<const TS *>(op.val);
  double dsum = 0.0, dsum2 = 0.0;
  int64_t r0 = ((int64_t)blockIdx.x * kWarps + warp) * RPC;
  int rs = 0, re = 0;
  if (r0 < n) {
    rs = __ldg(op.rowptr + min(r0 + g, n));
    re = __ldg(op.rowptr + min(r0 + g + 1, n));
  }
  for (; r0 < n; r0 += step) {
    const int64_t i = r0 + g;
    const bool valid = i < n;
    const bool owner = valid && p == 0;  // the lane that runs the row's epilogue
    TB dpv = 0, wv = 0, xv = 0, iv = 0;
    double du = 0.0, du2 = 0.0;
    float rsc = 1.0f;
    if (owner) {
      row_operands<TB, 1, EPI>(op, i, 0, dpv, wv, xv, du, du2);
      if (op.init) iv = op.init[i];
      if constexpr (VL::scaled) rsc = __ldg(op.rscale + i);
    }
    int nrs = 0, nre = 0;
    if (r0 + step < n) {
      nrs = __ldg(op.rowptr + min(r0 + step + g, n));
      nre = __ldg(op.rowptr + min(r0 + step + g + 1, n));
    }
    const int e0 = __shfl_sync(0xffffffffu, rs, 0), e1 = __shfl_sync(0xffffffffu, re, 31);
    // the owner lane starts from the init value (FP64, unscaled values), so
    // that no FP64 add is spent on it
    TB acc = sum_from_init<TB, VL::scaled>() ? iv : (TB)0;
    for (int wb = e0; wb < e1; wb += R) {
      const int we = min(e1, wb + R);
      const int vb = pairs ? (wb & ~1) : wb;  // first value in the window's buffer
      __syncwarp();  // every lane is done with the previous window
      for (int k = wb + lane; k < we; k += 32) cp_async_4(s_col + (k - wb), op.col + k);
      if constexpr (pairs) {
        // aligned pairs (vb, vb+1), ..., covering [wb, we); the value array
        // holds an even number of entries
        for (int k = vb + 2 * lane; k < we; k += 64) cp_async_4(s_val + (k - vb), gval + k);
      } else if constexpr (sizeof(TS) == 8) {
        for (int k = wb + lane; k < we; k += 32) cp_async_8(s_val + (k - vb), gval + k);
      } else {
        for (int k = wb + lane; k < we; k += 32) cp_async_4(s_val + (k - vb), gval + k);
      }
      cp_async_wait_all();
      __syncwarp();
      // this lane's entries of the window: lo, lo + LPR, ... < hi
      const int lo = max(rs, wb) + p, hi = min(re, we);
      const int cnt = hi > lo ? (hi - lo + LPR - 1) / LPR : 0;
      const int wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt);
      // blocks of eight entries, then a warp-uniform tail of exactly
      // wmax % 8 FMAs (the FP64 issue rate is the bound; a masked lane adds
      // 0 * 0)
      for (int q = 0; q < wmax; q += 8) {
        TB a[8], xg[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          a[u] = (TB)0;
          xg[u] = (TB)0;
          const int k = lo + (q + u) * LPR;
          if (k < hi) {
            const int c = s_col[k - wb];
            if constexpr (pairs) a[u] = __bfloat162float(s_val[k - vb]);
            else a[u] = (TB)s_val[k - vb];
            xg[u] = __ldg(op.src + c);
          }
        }
        if (q + 8 <= wmax) {
#pragma unroll
          for (int u = 0; u < 8; ++u) acc = fmadd<NEG>(a[u], xg[u], acc);
        } else {
          acc = tail_fma<NEG>(wmax - q, a, xg, acc);
        }
      }
    }
#pragma unroll
    for (int o = 1; o < LPR; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if constexpr (!sum_from_init<TB, VL::scaled>()) acc = ep_combine<TB, VL::scaled>(acc, (TB)rsc, op.init != nullptr, iv);
    if (owner) row_epilogue<TB, 1, EPI>(op, i, 0, acc, dpv, wv, xv, du, du2, dsum, dsum2);
    rs = nrs;
    re = nre;
  }
  if constexpr (epi_has_dot<EPI>()) {
    if (EPI != EPI_Y_DOT2 || op.dot_u) block_colsum_store<1>(dsum, op.partials);
    if constexpr (EPI == EPI_Y_DOT2 || EPI == EPI_XLAST_DOT2) {
      __syncthreads();
      block_colsum_store<1>(dsum2, op.partials2);
    }
  }
}

// The stream kernel for narrow blocks of NV = 2 or 4 columns (8 to 32 bytes of
// block row: FP64 with 2 or 4 columns, FP32 with 2 or 4): one lane per row holds
// the row's NV columns, and the warp's entries are staged in shared memory
// exactly as at m = 1, so the lane walks its row from the window and gathers
// one NV-wide operand row per entry (one 8- or 16-byte access, two for 32
// bytes).  Each
// column's products are added in storage order, as in the narrow split; the
// epilogue is vec_epilogue on the lane's NV columns.
template <class TB, class TV, int NV, int R, bool NEG, int EPI>
__device__ __forceinline__ void rows_stream_v(const RowOpT<TB> &op, unsigned char *smem) {
  using VL = ValueLoad<TV>;
  using TS = typename VL::T;
  using V = Vec<TB, NV>;
  static_assert(!VL::idx16, "the stream kernel reads 32-bit column indices");
  static_assert(NV * sizeof(TB) == 8 || NV * sizeof(TB) == 16 || NV * sizeof(TB) == 32,
                "8-, 16- or 32-byte block rows");
  constexpr bool pairs = sizeof(TS) == 2;
  constexpr bool xlast = EPI == EPI_XLAST || EPI == EPI_XLAST_DOT || EPI == EPI_XLAST_DOT2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t *s_col = reinterpret_cast<int32_t *>(smem + warp * stream_warp_bytes<TV, R>());
  TS *s_val = reinterpret_cast<TS *>(s_col + R);
  const int64_t n = op.n;
  const int64_t step = (int64_t)gridDim.x * kWarps * 32;
  const TS *gval = static_cast<const TS *>(op.val);
  double dsum[NV], dsum2[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) dsum[v] = dsum2[v] = 0.0;
  int64_t r0 = ((int64_t)blockIdx.x * kWarps + warp) * 32;
  int rs = 0, re = 0;
  if (r0 < n) {
    rs = __ldg(op.rowptr + min(r0 + lane, n));
    re = __ldg(op.rowptr + min(r0 + lane + 1, n));
  }
  for (; r0 < n; r0 += step) {
    const int64_t i = r0 + lane;
    const bool valid = i < n;
    const int64_t e = i * NV;
    V acc, dpv, xv, in0;
    TB wv = 0, rsc = 1;
#pragma unroll
    for (int v = 0; v < NV; ++v) acc.v[v] = dpv.v[v] = xv.v[v] = in0.v[v] = 0;
    if (valid) {
      if (op.init) in0 = vload<TB, NV>(op.init + e);
      if constexpr (VL::scaled) rsc = (TB)__ldg(op.rscale + i);
      if constexpr (EPI == EPI_Y_DN || EPI == EPI_Y_XDP || EPI == EPI_MID || xlast) dpv = vload<TB, NV>(op.dp + e);
      if constexpr (EPI == EPI_Y_D0 || EPI == EPI_Y_DN || EPI == EPI_MID || xlast) wv = op.w[i];
      if constexpr (EPI == EPI_Y_XDP || EPI == EPI_MID || xlast) xv = vload<TB, NV>(op.x + e);
    }
    // FP64 unscaled values start the sums at the init value (no FP64 add)
    if constexpr (sum_from_init<TB, VL::scaled>()) acc = in0;
    int nrs = 0, nre = 0;
    if (r0 + step < n) {
      nrs = __ldg(op.rowptr + min(r0 + step + lane, n));
      nre = __ldg(op.rowptr + min(r0 + step + lane + 1, n));
    }
    const int e0 = __shfl_sync(0xffffffffu, rs, 0), e1 = __shfl_sync(0xffffffffu, re, 31);
    for (int wb = e0; wb < e1; wb += R) {
      const int we = min(e1, wb + R);
      const int vb = pairs ? (wb & ~1) : wb;
      __syncwarp();
      for (int k = wb + lane; k < we; k += 32) cp_async_4(s_col + (k - wb), op.col + k);
      if constexpr (pairs) {
        for (int k = vb + 2 * lane; k < we; k += 64) cp_async_4(s_val + (k - vb), gval + k);
      } else if constexpr (sizeof(TS) == 8) {
        for (int k = wb + lane; k < we; k += 32) cp_async_8(s_val + (k - vb), gval + k);
      } else {
        for (int k = wb + lane; k < we; k += 32) cp_async_4(s_val + (k - vb), gval + k);
      }
      cp_async_wait_all();
      __syncwarp();
      const int lo = max(rs, wb), hi = min(re, we);
      const int cnt = hi > lo ? hi - lo : 0;
      const int wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt);
      // blocks of four entries (their gathers in flight together), then a
      // warp-uniform tail of exactly wmax % 4 (a masked lane adds 0 * 0)
      for (int q = 0; q < wmax; q += 4) {
        TB a[4];
        V xg[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = (TB)0;
#pragma unroll
          for (int v = 0; v < NV; ++v) xg[u].v[v] = (TB)0;
          const int k = lo + q + u;
          if (k < hi) {
            const int c = s_col[k - wb];
            if constexpr (pairs) a[u] = __bfloat162float(s_val[k - vb]);
            else a[u] = (TB)s_val[k - vb];
            xg[u] = vldg<TB, NV>(op.src + (int64_t)c * NV);
          }
        }
        const int rem = min(4, wmax - q);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u < rem) {
#pragma unroll
            for (int v = 0; v < NV; ++v) acc.v[v] = fmadd<NEG>(a[u], xg[u].v[v], acc.v[v]);
          }
        }
      }
    }
    if (valid) vec_epilogue<TB, TV, NV, NV, EPI>(op, i, e, acc, in0, dpv, wv, xv, rsc, dsum, dsum2);
    rs = nrs;
    re = nre;
  }
  if constexpr (epi_has_dot<EPI>()) {
    if (EPI != EPI_Y_DOT2 || op.dot_u) block_colsum_store_vec<NV, NV>(dsum, op.partials);
    if constexpr (EPI == EPI_Y_DOT2 || EPI == EPI_XLAST_DOT2) {
      __syncthreads();
      block_colsum_store_vec<NV, NV>(dsum2, op.partials2);
    }
  }
}

// Stream-kernel variants of the m = 1 split (the S < 0 codes of the row
// launchers): lanes per row and window entries.
template <int S> struct StreamCfg;
template <> struct StreamCfg<-1> { static constexpr int LPR = 1, R = 256; };
template <> struct StreamCfg<-2> { static constexpr int LPR = 1, R = 1024; };
template <> struct StreamCfg<-3> { static constexpr int LPR = 4, R = 1024; };
template <> struct StreamCfg<-4> { static constexpr int LPR = 32, R = 1024; };
template <> struct StreamCfg<-5> { static constexpr int LPR = 1, R = 512; };
template <> struct StreamCfg<-6> { static constexpr int LPR = 2, R = 512; };

// Columns per lane: FP32 blocks move 4 columns (16 bytes) per lane, which
// keeps 4x more rows' gathers in flight than one column per lane; FP64 blocks
// keep one column per lane (their bound is the FP64 FMA rate, not latency).
template <class TB, int NV>
__host__ __device__ constexpr int row_vec() {
  if constexpr (sizeof(TB) == 4) return NV >= 4 ? 4 : NV;
  return 1;
}
// Columns per lane of the row kernel with `slices` code S: two for the
// kNarrow2 / kPipeNarrow2 forms, else row_vec.
template <class TB, int NV, int S>
__host__ __device__ constexpr int split_vec() {
  return (S == kNarrow2 || S == kPipeNarrow2) ? 2 : row_vec<TB, NV>();
}

// The fused row kernel.  Warps walk the rows in a grid-stride loop, so the
// row -> block map (and with it the order of the partial dot sums) depends
// only on n and the grid size.  At most 64 registers per thread (four
// 256-thread blocks per SM): measured faster than the uncapped build, whose
// wider epilogues took 80 registers and three blocks per SM.  The pipelined
// narrow split (kPipeNarrow) holds the next rows' indices and row pointers
// as well and takes the 80 registers.
template <class TB, class TV, int NV, int S, bool NEG, int EPI>
__global__ void __launch_bounds__(kBlock, (S == kPipeNarrow || S == kPipeNarrow2) ? 3 : 4) k_rows(RowOpT<TB> op) {
  if constexpr (S == kPipeNarrow || S == kPipeNarrow2) {
    // the pipelined narrow split: 80 registers, three blocks per SM
    rows_vec<TB, TV, NV, split_vec<TB, NV, S>(), 1, NEG, EPI, 1, false, 0, true>(op);
  } else if constexpr (S == kNarrow2) {
    rows_vec<TB, TV, NV, 2, 1, NEG, EPI>(op);
  } else if constexpr (S == 1) {
    rows_vec<TB, TV, NV, row_vec<TB, NV>(), 1, NEG, EPI>(op);
  } else if constexpr (NV > 1 && S < 0) {
    // one row per warp (in 32 / (NV / VEC) slices), -S warps per row
    rows_vec<TB, TV, NV, row_vec<TB, NV>(), 32 / (NV / row_vec<TB, NV>()), NEG, EPI, -S>(op);
  } else if constexpr (NV > 1) {
    rows_vec<TB, TV, NV, row_vec<TB, NV>(), S, NEG, EPI>(op);
  } else {
    rows_sliced<TB, TV, NV, S, NEG, EPI>(op);
  }
}

// The stream kernel for 2- and 4-column blocks (rows_stream_v), window of R
// entries per warp as at m = 1.
template <class TB, class TV, int NV, int R, bool NEG, int EPI>
__global__ void __launch_bounds__(kBlock, R <= 512 ? 4 : 2) k_rows_stream_v(RowOpT<TB> op) {
  extern __shared__ __align__(16) unsigned char xamg_stream_v_smem[];
  if constexpr ((NV * sizeof(TB) == 8 || NV * sizeof(TB) == 16 || (sizeof(TB) == 8 && NV == 4)) &&
                !ValueLoad<TV>::idx16)
    rows_stream_v<TB, TV, NV, R, NEG, EPI>(op, xamg_stream_v_smem);
}

// The staged FP32 kernel (rows_async): kWarps windows of
// async_warp_bytes<TV, NV>() bytes of dynamic shared memory per block.
template <class TB, class TV, int NV, bool NEG, int EPI>
__global__ void __launch_bounds__(kBlock, 3) k_rows_async(RowOpT<TB> op) {
  extern __shared__ __align__(16) unsigned char xamg_async_smem[];
  if constexpr (sizeof(TB) == 4 && NV >= 8 && !ValueLoad<TV>::idx16) rows_async<TB, TV, NV, NEG, EPI>(op, xamg_async_smem);
}

// The m = 1 stream kernel: window of R entries per warp in dynamic shared
// memory (kWarps * stream_warp_bytes<TV, R>() bytes).  The 1024-entry window
// takes 96 KB per block in FP64, so two blocks share an SM; the 512-entry
// window 48 KB, four blocks.
template <class TB, class TV, int LPR, int R, bool NEG, int EPI>
__global__ void __launch_bounds__(kBlock, R <= 512 ? 4 : 2) k_rows_stream(RowOpT<TB> op) {
  extern __shared__ __align__(16) unsigned char xamg_stream_smem[];
  rows_stream<TB, TV, LPR, R, NEG, EPI>(op, xamg_stream_smem);
}

}  // namespace xamg
