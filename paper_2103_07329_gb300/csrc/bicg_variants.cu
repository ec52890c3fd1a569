// bicg_variants.cu -- elementwise and scalar kernels of the two BiCGStab
// variants the paper lists beside the classical method (Sec. 2.1): the
// reordered form (Krasnopolsky 2010), whose dot products fall in two groups
// per iteration with recurrences for rho and ||r||, and the pipelined form
// (Cools and Vanroose 2017), whose auxiliary products w = B r, s = B p,
// z = B s, t = B w, v = B z (B = A M) let each group of dot products run
// beside one application of B.  Vector updates carry their dot products
// (the merged formulation), partial sums per block, reduced in a fixed order.
#include "elem.cuh"
#include "launch.h"

namespace xamg {

// ---- reordered ----
// s = r - alpha v ; sh = w0 s ; partials s.s and rhat.s
template <int NV>
__global__ void __launch_bounds__(kBlock) k_rb_s(int64_t n, double *S, const double *R, const double *V,
                                                 const double *RH, const ColState *cs, const double *w0,
                                                 double *SH, double *part_ss, double *part_rs) {
  const int c = threadIdx.x % NV;
  const double a = cs->alpha[c];
  double ss = 0.0, rs = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const double s = fma(-a, V[e], R[e]);
    S[e] = s;
    if (w0) SH[e] = w0[e / NV] * s;
    ss = fma(s, s, ss);
    rs = fma(RH[e], s, rs);
  }
  block_colsum_store<NV>(ss, part_ss);
  __syncthreads();
  block_colsum_store<NV>(rs, part_rs);
}

// x += alpha ph + omega sh ; r = s - omega t ; partials rhat.t
template <int NV>
__global__ void __launch_bounds__(kBlock) k_rb_xr(int64_t n, double *X, double *R, const double *S,
                                                  const double *T, const double *PH, const double *SH,
                                                  const double *RH, const ColState *cs, double *part_rt) {
  const int c = threadIdx.x % NV;
  const double a = cs->alpha[c], om = cs->omega[c];
  double rt = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    X[e] = fma(om, SH[e], fma(a, PH[e], X[e]));
    R[e] = fma(-om, T[e], S[e]);
    rt = fma(RH[e], T[e], rt);
  }
  block_colsum_store<NV>(rt, part_rt);
}

// ---- pipelined ----
// p = r + beta (p - omega s) ; s = w + beta (s - omega z) ; z = t + beta (z - omega v)
// (p = r, s = w, z = t for a column that starts afresh)
template <int NV>
__global__ void __launch_bounds__(kBlock) k_pb_psz(int64_t n, double *P, double *S, double *Z, const double *R,
                                                   const double *W, const double *T, const double *V,
                                                   const ColState *cs) {
  const int c = threadIdx.x % NV;
  const bool fresh = cs->restart[c] != 0;
  const double b = cs->beta[c], om = cs->omega[c];
  XAMG_ELEM_LOOP(NV, n) {
    if (fresh) {
      P[e] = R[e];
      S[e] = W[e];
      Z[e] = T[e];
    } else {
      const double s = S[e], z = Z[e];
      P[e] = fma(b, fma(-om, s, P[e]), R[e]);
      S[e] = fma(b, fma(-om, z, s), W[e]);
      Z[e] = fma(b, fma(-om, V[e], z), T[e]);
    }
  }
}

// q = r - alpha s ; y = w - alpha z ; partials q.y and y.y
template <int NV>
__global__ void __launch_bounds__(kBlock) k_pb_qy(int64_t n, double *Q, double *Y, const double *R,
                                                  const double *S, const double *W, const double *Z,
                                                  const ColState *cs, double *part_qy, double *part_yy) {
  const int c = threadIdx.x % NV;
  const double a = cs->alpha[c];
  double qy = 0.0, yy = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    const double q = fma(-a, S[e], R[e]);
    const double y = fma(-a, Z[e], W[e]);
    Q[e] = q;
    Y[e] = y;
    qy = fma(q, y, qy);
    yy = fma(y, y, yy);
  }
  block_colsum_store<NV>(qy, part_qy);
  __syncthreads();
  block_colsum_store<NV>(yy, part_yy);
}

// u += alpha p + omega q ; r = q - omega y ; w = y - omega (t - alpha v) ;
// partials rhat.r, rhat.w, rhat.s, rhat.z, r.r
template <int NV>
__global__ void __launch_bounds__(kBlock) k_pb_urw(int64_t n, double *U, double *R, double *W, const double *P,
                                                   const double *Q, const double *Y, const double *T,
                                                   const double *V, const double *S, const double *Z,
                                                   const double *RH, const ColState *cs, double *p0, double *p1,
                                                   double *p2, double *p3, double *p4) {
  const int c = threadIdx.x % NV;
  const double a = cs->alpha[c], om = cs->omega[c];
  double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0, d4 = 0.0;
  XAMG_ELEM_LOOP(NV, n) {
    U[e] = fma(om, Q[e], fma(a, P[e], U[e]));
    const double r = fma(-om, Y[e], Q[e]);
    const double w = fma(-om, fma(-a, V[e], T[e]), Y[e]);
    R[e] = r;
    W[e] = w;
    const double rh = RH[e];
    d0 = fma(rh, r, d0);
    d1 = fma(rh, w, d1);
    d2 = fma(rh, S[e], d2);
    d3 = fma(rh, Z[e], d3);
    d4 = fma(r, r, d4);
  }
  block_colsum_store<NV>(d0, p0);
  __syncthreads();
  block_colsum_store<NV>(d1, p1);
  __syncthreads();
  block_colsum_store<NV>(d2, p2);
  __syncthreads();
  block_colsum_store<NV>(d3, p3);
  __syncthreads();
  block_colsum_store<NV>(d4, p4);
}

// X = X0 + D (the solution from the accumulated preconditioned correction)
template <int NV>
__global__ void __launch_bounds__(kBlock) k_pb_form_x(int64_t n, double *X, const double *X0, const double *D) {
  XAMG_ELEM_LOOP(NV, n) { X[e] = X0[e] + D[e]; }
}

// columns restarted by the last confirmation: X0 = X, U = 0, RH = R
template <int NV>
__global__ void __launch_bounds__(kBlock) k_pb_restart(int64_t n, const double *X, double *X0, double *U,
                                                       double *RH, const double *R, const ColState *cs) {
  const int c = threadIdx.x % NV;
  if (!cs->reac[c]) return;
  XAMG_ELEM_LOOP(NV, n) {
    X0[e] = X[e];
    U[e] = 0.0;
    RH[e] = R[e];
  }
}

// ---- scalar steps of both variants ----
// Five partial-sum arrays, each with its own block count; warp c reduces
// column c of every array (lanes take blocks in order, then a fixed xor
// tree); thread c applies the step.
template <int NV>
__global__ void __launch_bounds__(1024) k_vscalar(int mode, ColState *cs, VParts P, double tol, int k, Flags *fl) {
  __shared__ double sd[5][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < NV) {
    for (int q = 0; q < 5; ++q) {
      double a = 0.0;
      if (P.p[q])
        for (int g = lane; g < P.nblk[q]; g += 32) a += P.p[q][(size_t)g * NV + warp];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) sd[q][warp] = a;
    }
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int c = threadIdx.x;
    const double d0 = sd[0][c], d1 = sd[1][c], d2 = sd[2][c], d3 = sd[3][c], d4 = sd[4][c];
    const int st = cs->state[c];
    const double tb = tol * cs->nb[c];
    switch (mode) {
      case VS_RHO0:  // rho = rhat.r (d0) for every column that starts afresh
        if (cs->restart[c]) cs->rho[c] = d0;
        break;
      case VS_RB_BETA:  // beta of the direction update (first step or restart: 0)
        if (st == 0) {
          const double rho = cs->rho[c];
          if (rho == 0.0 || !isfinite(rho)) {
            cs->state[c] = 3;
            cs->beta[c] = 0.0;
          } else {
            cs->beta[c] = cs->restart[c] ? 0.0 : (rho / cs->rho_old[c]) * (cs->alpha[c] / cs->omega[c]);
            cs->restart[c] = 0;
          }
        } else {
          cs->beta[c] = 0.0;
        }
        break;
      case VS_RB_OMEGA:  // d0 = t.s, d1 = t.t, d2 = s.s
        if (st == 0) {
          cs->iters[c] = k;
          if (sqrt(d2) <= tb) {  // s already meets the tolerance: x += alpha ph, r = s
            cs->omega[c] = 0.0;
            cs->state[c] = 1;
          } else {
            const double om = d0 / d1;
            if (d1 == 0.0 || d0 == 0.0 || !isfinite(om)) {
              cs->state[c] = 3;
              cs->alpha[c] = 0.0;
              cs->omega[c] = 0.0;
            } else {
              cs->omega[c] = om;
              const double rr = d2 - 2.0 * om * d0 + om * om * d1;
              if (rr <= tb * tb) cs->state[c] = 1;
            }
          }
        } else {
          cs->alpha[c] = 0.0;
          cs->omega[c] = 0.0;
        }
        break;
      case VS_RB_RHO:  // d0 = rhat.s, d1 = rhat.t: rho' = rhat.s - omega rhat.t
        if (cs->omega[c] != 0.0 && cs->state[c] != 3) {
          cs->rho_old[c] = cs->rho[c];
          cs->rho[c] = d0 - cs->omega[c] * d1;
        }
        break;
      case VS_PB_INIT:  // d0 = rhat.r, d1 = rhat.w for columns that start afresh
        if (st == 0 && cs->restart[c]) {
          if (d0 == 0.0 || d1 == 0.0 || !isfinite(d0 / d1)) {
            cs->state[c] = 3;
            cs->alpha[c] = cs->beta[c] = cs->omega[c] = 0.0;
          } else {
            cs->rho[c] = d0;
            cs->alpha[c] = d0 / d1;
          }
        }
        break;
      case VS_PB_OMEGA:  // d0 = q.y, d1 = y.y
        if (st == 0) {
          cs->iters[c] = k;
          cs->restart[c] = 0;
          const double om = d0 / d1;
          if (d1 == 0.0 || d0 == 0.0 || !isfinite(om)) {
            cs->state[c] = 3;
            cs->alpha[c] = cs->beta[c] = cs->omega[c] = 0.0;
          } else {
            cs->omega[c] = om;
          }
        } else {
          cs->alpha[c] = cs->beta[c] = cs->omega[c] = 0.0;
        }
        break;
      case VS_PB_ALPHA:  // d0 = rhat.r, d1 = rhat.w, d2 = rhat.s, d3 = rhat.z, d4 = r.r
        if (st == 0) {
          if (sqrt(d4) <= tb) {
            cs->state[c] = 1;
            cs->alpha[c] = cs->beta[c] = cs->omega[c] = 0.0;
          } else {
            const double om = cs->omega[c];
            const double beta = (cs->alpha[c] / om) * (d0 / cs->rho[c]);
            const double den = d1 + beta * d2 - beta * om * d3;
            if (d0 == 0.0 || den == 0.0 || !isfinite(d0 / den) || !isfinite(beta)) {
              cs->state[c] = 3;
              cs->alpha[c] = cs->beta[c] = cs->omega[c] = 0.0;
            } else {
              cs->beta[c] = beta;
              cs->rho[c] = d0;
              cs->alpha[c] = d0 / den;
            }
          }
        }
        break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && fl) {
    int act = 0, fr = 0, br = 0;
    for (int c = 0; c < NV; ++c) {
      act += cs->state[c] == 0;
      fr += cs->state[c] == 1;
      br += cs->state[c] == 3;
    }
    volatile Flags *vf = fl;
    vf->active = act;
    vf->frozen = fr;
    vf->breakdown = br;
  }
}

#define XAMG_VNV(nv, CALL)                           \
  switch (nv) {                                      \
    case 1: { constexpr int NV = 1; CALL; } break;   \
    case 2: { constexpr int NV = 2; CALL; } break;   \
    case 4: { constexpr int NV = 4; CALL; } break;   \
    case 8: { constexpr int NV = 8; CALL; } break;   \
    case 16: { constexpr int NV = 16; CALL; } break; \
    case 32: { constexpr int NV = 32; CALL; } break; \
    default: break;                                  \
  }

void launch_rb_s(int nv, int64_t n, double *S, const double *R, const double *V, const double *RH,
                 const ColState *cs, const double *w0, double *SH, double *part_ss, double *part_rs, int grid,
                 cudaStream_t st) {
  XAMG_VNV(nv, (k_rb_s<NV><<<grid, kBlock, 0, st>>>(n, S, R, V, RH, cs, w0, SH, part_ss, part_rs)));
  g_launches++;
}
void launch_rb_xr(int nv, int64_t n, double *X, double *R, const double *S, const double *T, const double *PH,
                  const double *SH, const double *RH, const ColState *cs, double *part_rt, int grid,
                  cudaStream_t st) {
  XAMG_VNV(nv, (k_rb_xr<NV><<<grid, kBlock, 0, st>>>(n, X, R, S, T, PH, SH, RH, cs, part_rt)));
  g_launches++;
}
void launch_pb_psz(int nv, int64_t n, double *P, double *S, double *Z, const double *R, const double *W,
                   const double *T, const double *V, const ColState *cs, int grid, cudaStream_t st) {
  XAMG_VNV(nv, (k_pb_psz<NV><<<grid, kBlock, 0, st>>>(n, P, S, Z, R, W, T, V, cs)));
  g_launches++;
}
void launch_pb_qy(int nv, int64_t n, double *Q, double *Y, const double *R, const double *S, const double *W,
                  const double *Z, const ColState *cs, double *part_qy, double *part_yy, int grid,
                  cudaStream_t st) {
  XAMG_VNV(nv, (k_pb_qy<NV><<<grid, kBlock, 0, st>>>(n, Q, Y, R, S, W, Z, cs, part_qy, part_yy)));
  g_launches++;
}
void launch_pb_urw(int nv, int64_t n, double *U, double *R, double *W, const double *P, const double *Q,
                   const double *Y, const double *T, const double *V, const double *S, const double *Z,
                   const double *RH, const ColState *cs, double *const part[5], int grid, cudaStream_t st) {
  XAMG_VNV(nv, (k_pb_urw<NV><<<grid, kBlock, 0, st>>>(n, U, R, W, P, Q, Y, T, V, S, Z, RH, cs, part[0], part[1],
                                                     part[2], part[3], part[4])));
  g_launches++;
}
void launch_pb_form_x(int nv, int64_t n, double *X, const double *X0, const double *D, int grid, cudaStream_t st) {
  XAMG_VNV(nv, (k_pb_form_x<NV><<<grid, kBlock, 0, st>>>(n, X, X0, D)));
  g_launches++;
}
void launch_pb_restart(int nv, int64_t n, const double *X, double *X0, double *U, double *RH, const double *R,
                       const ColState *cs, int grid, cudaStream_t st) {
  XAMG_VNV(nv, (k_pb_restart<NV><<<grid, kBlock, 0, st>>>(n, X, X0, U, RH, R, cs)));
  g_launches++;
}
void launch_vscalar(int nv, int mode, ColState *cs, const VParts &P, double tol, int k, Flags *flags,
                    cudaStream_t st) {
  XAMG_VNV(nv, (k_vscalar<NV><<<1, 1024, 0, st>>>(mode, cs, P, tol, k, flags)));
  g_launches++;
}

}  // namespace xamg
