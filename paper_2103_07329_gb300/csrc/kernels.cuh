// kernels.cuh -- device kernels of the solve phase (sm_103a).
//
// Blocks of NV columns are n x NV row-major (element (i, c) at i*NV + c); NV
// is a compile-time power of two in {1, 2, 4, 8, 16, 32}, the counterpart of
// the paper's compile-time RHS count (Sec. 2.3: "The number of RHSs is also
// given as a template parameter").
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace xamg {

constexpr int kBlock = 256;  // threads per block of the row and element kernels
constexpr int kWarps = kBlock / 32;

// One fused row operation (paper Sec. 2.2-2.3: the "blas2" SpMV-like group,
// here with m columns at once).  For every row i of the sparse matrix M and
// column c:
//   v      = init[i,c] (or 0)  +/-  sum_k M_ik * src[k,c]      (sign: template NEG)
//   y[i,c] = v                                                 (if y)
//   dn     = c1 * dp[i,c] + w[i] * v                           (if w; dp may be null)
//   dnext[i,c] = dn                                            (if dnext)
//   x[i,c] += dp[i,c] (if x_dp) + dn (if x_dn)                 (if x)
//   partial dot: sum over the block's rows of dot_u[i,c] * t with t = v, the
//   new x or dn (dot_of = 0, 1, 2), written to partials[block*NV + c].
// All pointers except rowptr/col/val/src may alias each other only at the
// same element (own-row reads before own-row writes); src never aliases an
// output.
struct RowOp {
  int n;
  const int32_t *rowptr;
  const int32_t *col;
  const double *val;
  const double *src;
  const double *init;
  double *y;
  const double *dp;
  const double *w;
  double c1;
  double *dnext;
  double *x;
  int x_dp, x_dn;
  const double *dot_u;
  int dot_of;
  double *partials;
  double *partials2;  // if set: partial sums of v * v (second reduction)
};

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

// Row kernel.  A group of G = NV*S lanes owns one row: lane -> column
// c = lane % NV and slice s = (lane / NV) % S; slice s takes the row's
// entries s, s+S, s+2S, ...  With S = 1 every lane does exactly the row's
// FMAs for its column (no reduction adds); S > 1 splits long rows or narrow
// blocks over more lanes and adds the slices with shuffles.  Warps walk the
// rows in a grid-stride loop, so the row -> block map (and with it the order
// of the partial dot sums) depends only on n and the grid size.
template <int NV, int S, bool NEG>
__global__ void __launch_bounds__(kBlock) k_rows(RowOp op) {
  constexpr int G = NV * S;
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int c = lane % NV;
  const int s = (lane / NV) % S;
  const int grp = lane / G;
  const int64_t warp0 = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  const double *__restrict__ val = op.val;
  const int32_t *__restrict__ col = op.col;
  const double *__restrict__ src = op.src;
  double dsum = 0.0, dsum2 = 0.0;
  for (int64_t base = warp0 * RPW; base < op.n; base += wstride * RPW) {
    const int64_t i = base + grp;
    const bool valid = i < op.n;
    double acc = 0.0;
    if (valid) {
      if (op.init && s == 0) acc = op.init[i * NV + c];
      int k = __ldg(op.rowptr + i) + s;
      const int end = __ldg(op.rowptr + i + 1);
      for (; k + 3 * S < end; k += 4 * S) {
        const int k0 = __ldg(col + k), k1 = __ldg(col + k + S), k2 = __ldg(col + k + 2 * S),
                  k3 = __ldg(col + k + 3 * S);
        const double a0 = __ldg(val + k), a1 = __ldg(val + k + S), a2 = __ldg(val + k + 2 * S),
                     a3 = __ldg(val + k + 3 * S);
        const double x0 = __ldg(src + (int64_t)k0 * NV + c), x1 = __ldg(src + (int64_t)k1 * NV + c),
                     x2 = __ldg(src + (int64_t)k2 * NV + c), x3 = __ldg(src + (int64_t)k3 * NV + c);
        if (NEG) {
          acc = fma(-a0, x0, acc); acc = fma(-a1, x1, acc);
          acc = fma(-a2, x2, acc); acc = fma(-a3, x3, acc);
        } else {
          acc = fma(a0, x0, acc); acc = fma(a1, x1, acc);
          acc = fma(a2, x2, acc); acc = fma(a3, x3, acc);
        }
      }
      for (; k < end; k += S) {
        const double a = __ldg(val + k);
        const double xv = __ldg(src + (int64_t)__ldg(col + k) * NV + c);
        acc = NEG ? fma(-a, xv, acc) : fma(a, xv, acc);
      }
    }
    if (S > 1) {
#pragma unroll
      for (int o = NV; o < G; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    }
    if (valid && s == 0) {
      const int64_t e = i * NV + c;
      if (op.y) op.y[e] = acc;
      double dn = 0.0, dpv = 0.0, xn = 0.0;
      if (op.dp) dpv = op.dp[e];
      if (op.w) {
        const double wr = op.w[i] * acc;
        dn = op.dp ? fma(op.c1, dpv, wr) : wr;
        if (op.dnext) op.dnext[e] = dn;
      }
      if (op.x) {
        xn = op.x[e];
        if (op.x_dp) xn += dpv;
        if (op.x_dn) xn += dn;
        op.x[e] = xn;
      }
      if (op.partials) {
        const double t = op.dot_of == 0 ? acc : (op.dot_of == 1 ? xn : dn);
        dsum = fma(op.dot_u[e], t, dsum);
      }
      if (op.partials2) dsum2 = fma(acc, acc, dsum2);
    }
  }
  if (op.partials) block_colsum_store<NV>(dsum, op.partials);
  if (op.partials2) {
    __syncthreads();
    block_colsum_store<NV>(dsum2, op.partials2);
  }
}

}  // namespace xamg
