// elem.cuh -- device bodies of the elementwise, scalar and coarsest-level
// steps of the Krylov loops (paper Sec. 2.1-2.3: the "blas" vector updates,
// column dots and the direct solve at the bottom of the cycle).  The
// single-system kernels of kernels.cu and the batched kernels of batch.cu
// both call them, so both paths execute the same arithmetic.
#pragma once
#include "launch.h"

namespace xamg {

#define XAMG_ELEM_LOOP(NV, n)                                                            \
  for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x, total__ = (n) * (NV); e < total__; \
       e += (int64_t)gridDim.x * kBlock)

// Bn = R = B (padded), X = 0, R32 = fl32(B), Z32 = w0 * R32, partial ||B||^2.
template <int NV>
__device__ __forceinline__ void d_init_fpcg(int64_t n, const double *B, int m, double *Bn,
                                                      double *R, double *X, float *R32, float *Z32,
                                                      const float *w0, double *part) {
  const int c = threadIdx.x % NV;
  double acc = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const int64_t i = e / NV;
    const double b = c < m ? B[i * m + c] : 0.0;
    Bn[e] = b;
    R[e] = b;
    X[e] = 0.0;
    const float b32 = (float)b;
    R32[e] = b32;
    Z32[e] = w0 ? w0[i] * b32 : 0.0f;
    acc = fma(b, b, acc);
  }
  block_colsum_store<NV>(acc, part);
}
// x += alpha p ; r -= alpha q ; R32 = fl32(r) ; Z32 = w0 * R32 ; partial ||r||^2
template <int NV>
__device__ __forceinline__ void d_fpcg_xr(int64_t n, double *X, double *R, const double *P,
                                                    const double *Q, const ColState *cs,
                                                    const float *w0, float *R32, float *Z32,
                                                    double *part) {
  const int c = threadIdx.x % NV;
  const double a = cs->alpha[c];
  double acc = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const double r = fma(-a, Q[e], R[e]);
    X[e] = fma(a, P[e], X[e]);
    R[e] = r;
    const float r32 = (float)r;
    R32[e] = r32;
    if (w0) Z32[e] = w0[e / NV] * r32;
    acc = fma(r, r, acc);
  }
  block_colsum_store<NV>(acc, part);
}
// p = z + beta p with z the preconditioner's FP32 output
template <int NV>
__device__ __forceinline__ void d_fpcg_p(int64_t n, double *P, const float *Z32,
                                                   const ColState *cs) {
  const int c = threadIdx.x % NV;
  const double b = cs->beta[c];
  if (b == 0.0) {
    XAMG_ELEM_LOOP(NV, n) { P[e] = (double)Z32[e]; }
  } else {
    XAMG_ELEM_LOOP(NV, n) { P[e] = fma(b, P[e], (double)Z32[e]); }
  }
}
// Y32 = fl32(X) and, if w0, Z32 = w0 * Y32
template <int NV>
__device__ __forceinline__ void d_to_f32(int64_t n, const double *X, float *Y32,
                                                   const float *w0, float *Z32) {
  XAMG_ELEM_LOOP(NV, n) {
    const float y = (float)X[e];
    Y32[e] = y;
    if (w0) Z32[e] = w0[e / NV] * y;
  }
}
// dst[:, c] = src[:, c] for the columns restarted by the last confirmation
template <int NV>
__device__ __forceinline__ void d_copy_cols(int64_t n, double *dst, const double *src,
                                                      const ColState *cs) {
  const int c = threadIdx.x % NV;
  if (!cs->reac[c]) return;
  XAMG_ELEM_LOOP(NV, n) { dst[e] = src[e]; }
}
template <int NV>
__device__ __forceinline__ void d_copy_out(int64_t n, const double *Xin, double *Xu, int m) {
  const int c = threadIdx.x % NV;
  XAMG_ELEM_LOOP(NV, n) {
    if (c < m) Xu[(e / NV) * m + c] = Xin[e];
  }
}
// ------------------------------------------------------------------ scalars
// One block of 1024 threads.  Warp c reduces column c of the partial sums
// (lane t takes blocks t, t+32, ... in order, then a fixed xor tree); thread c
// then applies the per-column step of the Krylov method.
template <int NV>
__device__ __forceinline__ void d_scalar(int mode, ColState *cs, const double *p0,
                                                 const double *p1, int nblk, double tol, int k,
                                                 Flags *fl) {
  __shared__ double s0[32], s1[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < NV) {
    double a = 0.0, b = 0.0;
    if (p0)
      for (int g = lane; g < nblk; g += 32) a += p0[(size_t)g * NV + warp];
    if (p1)
      for (int g = lane; g < nblk; g += 32) b += p1[(size_t)g * NV + warp];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      s0[warp] = a;
      s1[warp] = b;
    }
  }
  __syncthreads();
  // k < 0: the iteration number is the device counter's next value (a
  // captured iteration replays with the same arguments)
  const int kk = k >= 0 ? k : cs->kdev + 1;
  if (threadIdx.x < NV) {
    const int c = threadIdx.x;
    const double d0 = s0[c], d1 = s1[c];
    const int st = cs->state[c];
    switch (mode) {
      case SM_INIT: {
        const double nb = sqrt(d0);
        cs->nb[c] = nb;
        cs->state[c] = nb > 0.0 ? 0 : 4;
        cs->restart[c] = 1;
        cs->iters[c] = 0;
        cs->reac[c] = 0;
        cs->alpha[c] = cs->beta[c] = cs->omega[c] = cs->rho[c] = cs->tn[c] = 0.0;
        break;
      }
      case SM_PCG_ALPHA:
        if (st == 0) {
          if (!(d0 > 0.0)) {
            cs->state[c] = 3;
            cs->alpha[c] = 0.0;
          } else {
            cs->alpha[c] = cs->rho[c] / d0;
            cs->iters[c] = kk;
          }
        } else {
          cs->alpha[c] = 0.0;
        }
        break;
      case SM_PCG_CONV:
      case SM_BI_CONV:
        if (st == 0 && sqrt(d0) <= tol * cs->nb[c]) cs->state[c] = 1;
        break;
      case SM_PCG_BETA:
        if (st == 0) {
          if (!(d0 > 0.0)) {
            cs->state[c] = 3;
            cs->beta[c] = 0.0;
          } else {
            cs->beta[c] = cs->restart[c] ? 0.0 : d0 / cs->rho[c];
            cs->restart[c] = 0;
            cs->rho[c] = d0;
          }
        } else {
          cs->beta[c] = 0.0;
        }
        break;
      case SM_CONFIRM: {
        const double tn = sqrt(d0);
        cs->tn[c] = tn;
        cs->reac[c] = 0;
        if (st == 1) {
          if (tn <= tol * cs->nb[c]) {
            cs->state[c] = 2;
          } else {
            cs->state[c] = 0;
            cs->restart[c] = 1;
            cs->reac[c] = 1;
          }
        }
        break;
      }
      case SM_FINAL:
        cs->tn[c] = sqrt(d0);
        break;
      case SM_FPCG_BETA:
        // flexible CG (FP32 preconditioner): beta = z_new . (r_new - r_old) / (z_old . r_old)
        // with r_new - r_old = -alpha q, i.e. beta = -alpha (z_new . q) / rho_old
        if (st == 0) {
          if (!(d0 > 0.0)) {
            cs->state[c] = 3;
            cs->beta[c] = 0.0;
          } else {
            cs->beta[c] = cs->restart[c] ? 0.0 : -cs->alpha[c] * d1 / cs->rho[c];
            cs->restart[c] = 0;
            cs->rho[c] = d0;
          }
        } else {
          cs->beta[c] = 0.0;
        }
        break;
      case SM_BI_RHO:
        if (st == 0) {
          if (d0 == 0.0 || !isfinite(d0)) {
            cs->state[c] = 3;
            cs->beta[c] = 0.0;
          } else {
            cs->beta[c] = cs->restart[c] ? 0.0 : (d0 / cs->rho[c]) * (cs->alpha[c] / cs->omega[c]);
            cs->restart[c] = 0;
            cs->rho[c] = d0;
          }
        } else {
          cs->beta[c] = 0.0;
        }
        break;
      case SM_BI_ALPHA:
        if (st == 0) {
          if (d0 == 0.0 || !isfinite(d0)) {
            cs->state[c] = 3;
            cs->alpha[c] = 0.0;
            cs->omega[c] = 0.0;
          } else {
            cs->alpha[c] = cs->rho[c] / d0;
          }
        } else {
          cs->alpha[c] = 0.0;
          cs->omega[c] = 0.0;
        }
        break;
      case SM_BI_HALF:
        if (st == 0) {
          cs->iters[c] = kk;
          if (sqrt(d0) <= tol * cs->nb[c]) {
            cs->state[c] = 1;
            cs->omega[c] = 0.0;
          }
        }
        break;
      case SM_BI_OMEGA:
        if (st == 0) {
          const double om = d0 / d1;
          if (d1 == 0.0 || d0 == 0.0 || !isfinite(om)) {
            cs->state[c] = 3;
            cs->alpha[c] = 0.0;
            cs->omega[c] = 0.0;
          } else {
            cs->omega[c] = om;
          }
        }
        break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (mode == SM_INIT) cs->kdev = 0;
    if (mode == SM_PCG_ALPHA || mode == SM_BI_HALF) cs->kdev = kk;
  }
  if (threadIdx.x == 0 && fl) {
    int act = 0, fr = 0, re = 0, br = 0;
    for (int c = 0; c < NV; ++c) {
      act += cs->state[c] == 0;
      fr += cs->state[c] == 1;
      re += cs->reac[c];
      br += cs->state[c] == 3;
    }
    volatile Flags *vf = fl;
    vf->active = act;
    vf->frozen = fr;
    vf->reactivated = re;
    vf->breakdown = br;
    if (mode == SM_INIT) {
      int nonfinite = 0;
      for (int c = 0; c < NV; ++c) nonfinite |= !isfinite(s0[c]);
      vf->breakdown = nonfinite ? -1 : 0;
    }
  }
}
// FP64 tensor-core product D += A B of one 8x8x4 step (mma.sync m8n8k4):
// lane (g = lane / 4, q = lane % 4) holds a = A[g][q], b = B[q][g] and
// d = D[g][2q], D[g][2q + 1].
__device__ __forceinline__ void dmma884(double (&d)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

// Coarsest-level direct solve (paper Tab. 1, "Direct") as the dense product
// X = Ainv B on the FP64 tensor cores: Ainv (nc x nc, row-major) is the
// inverse of the coarsest operator, formed at upload from its LU factors;
// B, X are nc x NV blocks (TI / TO: double, or float widened and rounded).
// One block; warp w takes the 8 x 8 output tiles w, w + warps, ...; rows and
// columns past nc and NV read as zero.  FP64 products and sums throughout.
template <int NV, class TI, class TO>
__device__ __forceinline__ void d_coarse_mma(int nc, const double *Ainv, const TI *B, TO *X) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int mt_n = (nc + 7) / 8;
  constexpr int nt_n = (NV + 7) / 8;
  for (int tile = warp; tile < mt_n * nt_n; tile += (int)(blockDim.x >> 5)) {
    const int mt = tile / nt_n, nt = tile % nt_n;
    const int row = mt * 8 + g;   // row of the A fragment and of the output
    const int colb = nt * 8 + g;  // column of the B fragment
    double acc[2] = {0.0, 0.0};
    for (int k = 0; k < nc; k += 4) {
      const int kk = k + q;
      const double a = (row < nc && kk < nc) ? Ainv[(size_t)row * nc + kk] : 0.0;
      const double b = (kk < nc && colb < NV) ? (double)B[(size_t)kk * NV + colb] : 0.0;
      dmma884(acc, a, b);
    }
    const int c0 = nt * 8 + 2 * q;
    if (row < nc) {
      if (c0 < NV) X[(size_t)row * NV + c0] = (TO)acc[0];
      if (c0 + 1 < NV) X[(size_t)row * NV + c0 + 1] = (TO)acc[1];
    }
  }
}
template <int NV>
__device__ __forceinline__ void d_to_f64(int64_t n, const float *X32, double *Y) {
  XAMG_ELEM_LOOP(NV, n) { Y[e] = (double)X32[e]; }
}
}  // namespace xamg
