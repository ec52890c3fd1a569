// kernels.cu -- solve-phase kernels and their launchers (sm_103a).
//
// Every reduction in this file is deterministic: per-block partial sums are
// formed in a fixed thread order and reduced by one block in a fixed order,
// so repeated runs of the same solve give identical bits.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "elem.cuh"
#include "launch.h"

namespace xamg {

std::atomic<int64_t> g_launches{0};

// SM count of the current device, cached per device ordinal (atomics: the
// library may be called from several host threads).
int device_sm_count() {
  constexpr int kDevs = 64;
  static std::atomic<int> cache[kDevs];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const int slot = dev >= 0 && dev < kDevs ? dev : -1;
  if (slot >= 0) {
    const int c = cache[slot].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  if (slot >= 0) cache[slot].store(sms, std::memory_order_relaxed);
  return sms;
}

// Elementwise grid: at most 8 blocks per SM and never more than kMaxGrid, the
// block count the per-block partial-sum buffers are sized for.
int elem_grid(int64_t n, int nv) {
  const int64_t need = (n * nv + kBlock - 1) / kBlock;
  const int64_t cap = std::min<int64_t>((int64_t)device_sm_count() * 8, kMaxGrid);
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, cap));
}

// ------------------------------------------------------------------ rows
int launch_rows(const RowOp &op, int nv, int slices, bool neg, int epi, cudaStream_t st) {
  switch (nv) {
    case 1: return launch_rows_nv1(op, slices, neg, epi, st);
    case 2: return launch_rows_nv2(op, slices, neg, epi, st);
    case 4: return launch_rows_nv4(op, slices, neg, epi, st);
    case 8: return launch_rows_nv8(op, slices, neg, epi, st);
    case 16: return launch_rows_nv16(op, slices, neg, epi, st);
    case 32: return launch_rows_nv32(op, slices, neg, epi, st);
  }
  return -1;
}

int launch_rows_f(const RowOpF &op, int nv, int slices, bool neg, int epi, int vt, cudaStream_t st) {
  switch (nv) {
    case 1: return launch_rowsf_nv1(op, slices, neg, epi, vt, st);
    case 2: return launch_rowsf_nv2(op, slices, neg, epi, vt, st);
    case 4: return launch_rowsf_nv4(op, slices, neg, epi, vt, st);
    case 8: return launch_rowsf_nv8(op, slices, neg, epi, vt, st);
    case 16: return launch_rowsf_nv16(op, slices, neg, epi, vt, st);
    case 32: return launch_rowsf_nv32(op, slices, neg, epi, vt, st);
  }
  return -1;
}

// ------------------------------------------------------------------ elementwise

// R, Bn = B (padded to NV columns), X = 0, Z = w0 * R (first smoother
// iterate of the preconditioner), partial ||R||^2.
template <int NV>
__global__ void __launch_bounds__(kBlock) k_init_pcg(int64_t n, const double *B, int m, double *Bn,
                                                     double *R, double *X, double *Z,
                                                     const double *w0, double *part) {
  const int c = threadIdx.x % NV;
  double acc = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const int64_t i = e / NV;
    const double b = c < m ? B[i * m + c] : 0.0;
    Bn[e] = b;
    R[e] = b;
    X[e] = 0.0;
    Z[e] = w0 ? w0[i] * b : 0.0;
    acc = fma(b, b, acc);
  }
  block_colsum_store<NV>(acc, part);
}

template <int NV>
__global__ void __launch_bounds__(kBlock) k_init_bicg(int64_t n, const double *B, int m, double *Bn,
                                                      double *R, double *RH, double *X, double *P,
                                                      double *V, double *part) {
  const int c = threadIdx.x % NV;
  double acc = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const int64_t i = e / NV;
    const double b = c < m ? B[i * m + c] : 0.0;
    Bn[e] = b;
    R[e] = b;
    RH[e] = b;
    X[e] = 0.0;
    P[e] = 0.0;
    V[e] = 0.0;
    acc = fma(b, b, acc);
  }
  block_colsum_store<NV>(acc, part);
}

// x += alpha p ; r -= alpha q ; z = w0 r ; partial ||r||^2
template <int NV>
__global__ void __launch_bounds__(kBlock) k_pcg_xr(int64_t n, double *X, double *R, const double *P,
                                                   const double *Q, const ColState *cs,
                                                   const double *w0, double *Z, double *part) {
  const int c = threadIdx.x % NV;
  const double a = cs->alpha[c];
  double acc = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const double r = fma(-a, Q[e], R[e]);
    X[e] = fma(a, P[e], X[e]);
    R[e] = r;
    if (w0) Z[e] = w0[e / NV] * r;
    acc = fma(r, r, acc);
  }
  block_colsum_store<NV>(acc, part);
}

// p = z + beta p
template <int NV>
__global__ void __launch_bounds__(kBlock) k_pcg_p(int64_t n, double *P, const double *Z,
                                                  const ColState *cs) {
  const int c = threadIdx.x % NV;
  const double b = cs->beta[c];
  if (b == 0.0) {
    XAMG_ELEM_LOOP(NV, n) { P[e] = Z[e]; }
  } else {
    XAMG_ELEM_LOOP(NV, n) { P[e] = fma(b, P[e], Z[e]); }
  }
}

// p = r + beta (p - omega v) ; ph = w0 p
template <int NV>
__global__ void __launch_bounds__(kBlock) k_bicg_p(int64_t n, double *P, const double *R,
                                                   const double *V, const ColState *cs,
                                                   const double *w0, double *PH) {
  const int c = threadIdx.x % NV;
  const double b = cs->beta[c], om = cs->omega[c];
  XAMG_ELEM_LOOP(NV, n) {
    const double p = fma(b, fma(-om, V[e], P[e]), R[e]);
    P[e] = p;
    if (w0) PH[e] = w0[e / NV] * p;
  }
}

// s = r - alpha v ; sh = w0 s ; partial ||s||^2
template <int NV>
__global__ void __launch_bounds__(kBlock) k_bicg_s(int64_t n, double *S, const double *R,
                                                   const double *V, const ColState *cs,
                                                   const double *w0, double *SH, double *part) {
  const int c = threadIdx.x % NV;
  const double a = cs->alpha[c];
  double acc = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const double s = fma(-a, V[e], R[e]);
    S[e] = s;
    if (w0) SH[e] = w0[e / NV] * s;
    acc = fma(s, s, acc);
  }
  block_colsum_store<NV>(acc, part);
}

// x += alpha ph + omega sh ; r = s - omega t ; partials ||r||^2 and rhat.r
template <int NV>
__global__ void __launch_bounds__(kBlock) k_bicg_xr(int64_t n, double *X, double *R, const double *S,
                                                    const double *T, const double *PH,
                                                    const double *SH, const double *RH,
                                                    const ColState *cs, double *part_rr,
                                                    double *part_rhr) {
  const int c = threadIdx.x % NV;
  const double a = cs->alpha[c], om = cs->omega[c];
  double rr = 0.0, rhr = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    X[e] = fma(om, SH[e], fma(a, PH[e], X[e]));
    const double r = fma(-om, T[e], S[e]);
    R[e] = r;
    rr = fma(r, r, rr);
    rhr = fma(RH[e], r, rhr);
  }
  block_colsum_store<NV>(rr, part_rr);
  __syncthreads();
  block_colsum_store<NV>(rhr, part_rhr);
}

template <int NV>
__global__ void __launch_bounds__(kBlock) k_copy_cols(int64_t n, double *dst, const double *src,
                                                      const ColState *cs) {
  d_copy_cols<NV>(n, dst, src, cs);
}


template <int NV>
__global__ void __launch_bounds__(kBlock) k_copy_out(int64_t n, const double *Xin, double *Xu, int m) {
  d_copy_out<NV>(n, Xin, Xu, m);
}


template <int NV>
__global__ void __launch_bounds__(kBlock) k_pad_in(int64_t n, const double *Xu, int m, double *Xp) {
  const int c = threadIdx.x % NV;
  XAMG_ELEM_LOOP(NV, n) { Xp[e] = c < m ? Xu[(e / NV) * m + c] : 0.0; }
}

template <int NV>
__global__ void __launch_bounds__(kBlock) k_scale_rows(int64_t n, const double *w, const double *B,
                                                       double *X) {
  XAMG_ELEM_LOOP(NV, n) { X[e] = w[e / NV] * B[e]; }
}

// x += d ; optional partial u.x
template <int NV>
__global__ void __launch_bounds__(kBlock) k_axpy_dot(int64_t n, double *X, const double *D,
                                                     const double *U, double *part) {
  double acc = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const double x = X[e] + D[e];
    X[e] = x;
    if (U) acc = fma(U[e], x, acc);
  }
  if (part) block_colsum_store<NV>(acc, part);
}

template <int NV>
__global__ void __launch_bounds__(kBlock) k_coldot(int64_t n, const double *U, const double *V,
                                                   double *part) {
  double acc = 0.0;
  XAMG_ELEM_LOOP(NV, n) { acc = fma(U[e], V[e], acc); }
  block_colsum_store<NV>(acc, part);
}

template <int NV>
__global__ void __launch_bounds__(1024) k_scalar(int mode, ColState *cs, const double *p0,
                                                 const double *p1, int nblk, double tol, int k,
                                                 Flags *fl) {
  d_scalar<NV>(mode, cs, p0, p1, nblk, tol, k, fl);
}


// ------------------------------------------------------------------ coarsest
// X = A_c^-1 B as a dense product on the FP64 tensor cores (elem.cuh).
template <int NV>
__global__ void __launch_bounds__(kBlock) k_coarse(int nc, const double *Ainv, const double *B, double *X) {
  d_coarse_mma<NV, double, double>(nc, Ainv, B, X);
}

// ------------------------------------------------------------------ mixed precision
// Kernels of the outer FP64 loop around a reduced-precision (FP32 block)
// preconditioner: FP64 vectors are rounded once to FP32 for the V-cycle and
// its FP32 result is widened again where the FP64 loop reads it.

template <int NV>
__global__ void __launch_bounds__(kBlock) k_init_fpcg(int64_t n, const double *B, int m, double *Bn,
                                                      double *R, double *X, float *R32, float *Z32,
                                                      const float *w0, double *part) {
  d_init_fpcg<NV>(n, B, m, Bn, R, X, R32, Z32, w0, part);
}


template <int NV>
__global__ void __launch_bounds__(kBlock) k_fpcg_xr(int64_t n, double *X, double *R, const double *P,
                                                    const double *Q, const ColState *cs,
                                                    const float *w0, float *R32, float *Z32,
                                                    double *part) {
  d_fpcg_xr<NV>(n, X, R, P, Q, cs, w0, R32, Z32, part);
}


template <int NV>
__global__ void __launch_bounds__(kBlock) k_fpcg_p(int64_t n, double *P, const float *Z32,
                                                   const ColState *cs) {
  d_fpcg_p<NV>(n, P, Z32, cs);
}


template <int NV>
__global__ void __launch_bounds__(kBlock) k_to_f32(int64_t n, const double *X, float *Y32,
                                                   const float *w0, float *Z32) {
  d_to_f32<NV>(n, X, Y32, w0, Z32);
}


template <int NV>
__global__ void __launch_bounds__(kBlock) k_to_f64(int64_t n, const float *X32, double *Y) {
  d_to_f64<NV>(n, X32, Y);
}


// x += d (FP32) ; optional FP64 partials u . x and u2 . x
template <int NV>
__global__ void __launch_bounds__(kBlock) k_axpy_dot_f(int64_t n, float *X, const float *D,
                                                       const double *U, const double *U2,
                                                       double *part, double *part2) {
  double acc = 0.0, acc2 = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const float x = X[e] + D[e];
    X[e] = x;
    if (U) acc = fma(U[e], (double)x, acc);
    if (U2) acc2 = fma(U2[e], (double)x, acc2);
  }
  if (part) block_colsum_store<NV>(acc, part);
  if (part2) {
    __syncthreads();
    block_colsum_store<NV>(acc2, part2);
  }
}

template <int NV>
__global__ void __launch_bounds__(kBlock) k_coarse_f(int nc, const double *Ainv, const float *B, float *X) {
  d_coarse_mma<NV, float, float>(nc, Ainv, B, X);
}


// X[:, c] = 0 for the columns with a zero right-hand side (state 4)
template <int NV>
__global__ void __launch_bounds__(kBlock) k_zero_rhs_cols(int64_t n, double *X, const ColState *cs) {
  const int c = threadIdx.x % NV;
  if (cs->state[c] != 4) return;
  XAMG_ELEM_LOOP(NV, n) { X[e] = 0.0; }
}

// ------------------------------------------------------------------ runtime-m dots
// Thread t of a block owns column t % m for t < (kBlock / m) * m; rows are
// strided over the grid.  Partials: per block and column, summed over the
// block's threads of that column in thread order.
__global__ void __launch_bounds__(kBlock) k_coldot_rt(int64_t n, int m, const double *U,
                                                      const double *V, double *part) {
  __shared__ double sh[kBlock];
  const int per = kBlock / m;
  const int t = threadIdx.x;
  double acc = 0.0;
  if (t < per * m) {
    const int c = t % m, r0 = t / m;
    for (int64_t i = (int64_t)blockIdx.x * per + r0; i < n; i += (int64_t)gridDim.x * per)
      acc = fma(U[i * m + c], V[i * m + c], acc);
  }
  sh[t] = acc;
  __syncthreads();
  if (t < m) {
    double s = 0.0;
    for (int r = 0; r < per; ++r) s += sh[r * m + t];
    part[(size_t)blockIdx.x * m + t] = s;
  }
}

__global__ void __launch_bounds__(1024) k_reduce_rt(int m, const double *part, int nblk, double *out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= m) return;
  double a = 0.0;
  for (int g = lane; g < nblk; g += 32) a += part[(size_t)g * m + warp];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) out[warp] = a;
}

// ------------------------------------------------------------------ dispatch
#define XAMG_NV_SWITCH(nv, CALL) \
  g_launches++;                  \
  switch (nv) {                  \
    case 1: { constexpr int NV = 1; CALL; } break;   \
    case 2: { constexpr int NV = 2; CALL; } break;   \
    case 4: { constexpr int NV = 4; CALL; } break;   \
    case 8: { constexpr int NV = 8; CALL; } break;   \
    case 16: { constexpr int NV = 16; CALL; } break; \
    case 32: { constexpr int NV = 32; CALL; } break; \
    default: break;              \
  }

void launch_init_pcg(int nv, int64_t n, const double *B, int m, double *Bn, double *R, double *X,
                     double *Z, const double *w0, double *part, int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_init_pcg<NV><<<grid, kBlock, 0, st>>>(n, B, m, Bn, R, X, Z, w0, part)));
}
void launch_init_bicg(int nv, int64_t n, const double *B, int m, double *Bn, double *R, double *RH,
                      double *X, double *P, double *V, double *part, int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_init_bicg<NV><<<grid, kBlock, 0, st>>>(n, B, m, Bn, R, RH, X, P, V, part)));
}
void launch_pcg_xr(int nv, int64_t n, double *X, double *R, const double *P, const double *Q,
                   const ColState *cs, const double *w0, double *Z, double *part, int grid,
                   cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_pcg_xr<NV><<<grid, kBlock, 0, st>>>(n, X, R, P, Q, cs, w0, Z, part)));
}
void launch_pcg_p(int nv, int64_t n, double *P, const double *Z, const ColState *cs, int grid,
                  cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_pcg_p<NV><<<grid, kBlock, 0, st>>>(n, P, Z, cs)));
}
void launch_bicg_p(int nv, int64_t n, double *P, const double *R, const double *V,
                   const ColState *cs, const double *w0, double *PH, int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_bicg_p<NV><<<grid, kBlock, 0, st>>>(n, P, R, V, cs, w0, PH)));
}
void launch_bicg_s(int nv, int64_t n, double *S, const double *R, const double *V,
                   const ColState *cs, const double *w0, double *SH, double *part, int grid,
                   cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_bicg_s<NV><<<grid, kBlock, 0, st>>>(n, S, R, V, cs, w0, SH, part)));
}
void launch_bicg_xr(int nv, int64_t n, double *X, double *R, const double *S, const double *T,
                    const double *PH, const double *SH, const double *RH, const ColState *cs,
                    double *part_rr, double *part_rhr, int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_bicg_xr<NV><<<grid, kBlock, 0, st>>>(n, X, R, S, T, PH, SH, RH, cs, part_rr,
                                                              part_rhr)));
}
void launch_copy_cols(int nv, int64_t n, double *dst, const double *src, const ColState *cs,
                      int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_copy_cols<NV><<<grid, kBlock, 0, st>>>(n, dst, src, cs)));
}
void launch_copy_out(int nv, int64_t n, const double *Xin, double *Xuser, int m, int grid,
                     cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_copy_out<NV><<<grid, kBlock, 0, st>>>(n, Xin, Xuser, m)));
}
void launch_pad_in(int nv, int64_t n, const double *Xuser, int m, double *Xp, int grid,
                   cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_pad_in<NV><<<grid, kBlock, 0, st>>>(n, Xuser, m, Xp)));
}
void launch_scale_rows(int nv, int64_t n, const double *w, const double *B, double *X, int grid,
                       cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_scale_rows<NV><<<grid, kBlock, 0, st>>>(n, w, B, X)));
}
void launch_axpy_dot(int nv, int64_t n, double *X, const double *D, const double *U, double *part,
                     int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_axpy_dot<NV><<<grid, kBlock, 0, st>>>(n, X, D, U, part)));
}
void launch_coldot(int nv, int64_t n, const double *U, const double *V, double *part, int grid,
                   cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_coldot<NV><<<grid, kBlock, 0, st>>>(n, U, V, part)));
}
void launch_scalar(int nv, int mode, ColState *cs, const double *p0, const double *p1, int nblk,
                   double tol, int k, Flags *flags, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_scalar<NV><<<1, 1024, 0, st>>>(mode, cs, p0, p1, nblk, tol, k, flags)));
}
void launch_coarse(int nv, int nc, const double *Ainv, const double *B, double *X, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_coarse<NV><<<1, kBlock, 0, st>>>(nc, Ainv, B, X)));
}

void launch_init_fpcg(int nv, int64_t n, const double *B, int m, double *Bn, double *R, double *X,
                      float *R32, float *Z32, const float *w0, double *part, int grid,
                      cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_init_fpcg<NV><<<grid, kBlock, 0, st>>>(n, B, m, Bn, R, X, R32, Z32, w0, part)));
}
void launch_fpcg_xr(int nv, int64_t n, double *X, double *R, const double *P, const double *Q,
                    const ColState *cs, const float *w0, float *R32, float *Z32, double *part,
                    int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_fpcg_xr<NV><<<grid, kBlock, 0, st>>>(n, X, R, P, Q, cs, w0, R32, Z32, part)));
}
void launch_fpcg_p(int nv, int64_t n, double *P, const float *Z32, const ColState *cs, int grid,
                   cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_fpcg_p<NV><<<grid, kBlock, 0, st>>>(n, P, Z32, cs)));
}
void launch_to_f32(int nv, int64_t n, const double *X, float *Y32, const float *w0, float *Z32,
                   int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_to_f32<NV><<<grid, kBlock, 0, st>>>(n, X, Y32, w0, Z32)));
}
void launch_to_f64(int nv, int64_t n, const float *X32, double *Y, int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_to_f64<NV><<<grid, kBlock, 0, st>>>(n, X32, Y)));
}
void launch_axpy_dot_f(int nv, int64_t n, float *X, const float *D, const double *U,
                       const double *U2, double *part, double *part2, int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_axpy_dot_f<NV><<<grid, kBlock, 0, st>>>(n, X, D, U, U2, part, part2)));
}
void launch_coarse_f(int nv, int nc, const double *Ainv, const float *B, float *X, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_coarse_f<NV><<<1, kBlock, 0, st>>>(nc, Ainv, B, X)));
}

void launch_zero_rhs_cols(int nv, int64_t n, double *X, const ColState *cs, int grid, cudaStream_t st) {
  XAMG_NV_SWITCH(nv, (k_zero_rhs_cols<NV><<<grid, kBlock, 0, st>>>(n, X, cs)));
}

int coldot_rt_grid(int64_t n, int m) {
  const int per = kBlock / m;
  const int64_t need = (n + per - 1) / per;
  const int64_t cap = std::min<int64_t>((int64_t)device_sm_count() * 8, kMaxGrid);
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, cap));
}
void launch_coldot_rt(int64_t n, int m, const double *U, const double *V, double *part, int grid,
                      cudaStream_t st) {
  k_coldot_rt<<<grid, kBlock, 0, st>>>(n, m, U, V, part);
  g_launches++;
}
void launch_reduce_rt(int m, const double *part, int nblk, double *out, cudaStream_t st) {
  k_reduce_rt<<<1, 1024, 0, st>>>(m, part, nblk, out);
  g_launches++;
}

}  // namespace xamg
