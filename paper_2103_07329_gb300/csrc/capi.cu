// capi.cu -- the library's C entry points: device upload of the hierarchy, the
// V(1,1) Chebyshev cycle, the PCG and BiCGStab drivers and the single-step
// entry points.  Declarations and contracts: include/xamg_gpu.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "batch.h"
#include "hier_host.h"
#include "launch.h"
#include "vtail.cuh"

using namespace xamg;

namespace {

struct DevCsr {
  int n = 0, ncols = 0;
  int64_t nnz = 0;
  // entries of the longest aligned group of 4, 8 and 16 consecutive rows (the
  // rows one warp of the staged FP32 kernel takes at 32, 16 and 8 columns)
  int span[3] = {0, 0, 0};
  int32_t *rowptr = nullptr;
  int32_t *col = nullptr;
  double *val = nullptr;
};

struct DevLevel {
  DevCsr A, P, R;
  double *w[4] = {nullptr, nullptr, nullptr, nullptr};  // Chebyshev row weights per step
  double c1[4] = {0, 0, 0, 0};                          // Chebyshev step coefficients
  // reduced-precision copies for the FP32-block preconditioner (same index arrays)
  float *a32 = nullptr, *p32 = nullptr, *r32 = nullptr;
  __nv_bfloat16 *a16 = nullptr;  // bf16(fl32(a_ij) / s_i)
  float *a16s = nullptr;         // s_i = fl32(max_j |a_ij|)
  // 16-bit column indices of A, P, R (index 0, 1, 2) in the segmented form
  // of kernels.cuh (offsets, row boundaries, tile bases), where the operator
  // fits it (else null)
  uint16_t *w16[3] = {nullptr, nullptr, nullptr};
  uint32_t *m16[3] = {nullptr, nullptr, nullptr};
  int32_t *t16[3] = {nullptr, nullptr, nullptr};
  float *w32[4] = {nullptr, nullptr, nullptr, nullptr};
  float c1f[4] = {0, 0, 0, 0};
  // row split of the sparse products chosen by xamg_autotune, per values
  // (0: FP32 blocks, 1: FP32 blocks with bf16 A, 2: FP64), operator (A, P, R)
  // and block width (log2 nv): -1 untuned (the default rule), else the
  // tuning candidate that won (split_slices)
  signed char split[3][3][6];
  DevLevel() { std::memset(split, -1, sizeof(split)); }
};

struct TimerRec {
  cudaEvent_t a, b;
  int level, which;
  double flops, bytes;
};

struct TimeAcc {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};

// Device blocks of one solve (n x nv row-major unless noted).
struct Work {
  int nv = 0;
  double *Bn = nullptr, *X = nullptr, *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr;
  double *RH = nullptr, *V = nullptr, *S = nullptr, *T = nullptr, *PH = nullptr, *SH = nullptr;
  std::vector<double *> vb, vx, vr, vd, vd2;  // V-cycle blocks per level
  // FP32-block preconditioner: level-0 input/output and per-level blocks
  float *R32 = nullptr, *Z32 = nullptr;
  std::vector<float *> fb, fx, fr, fd, fd2;
  double *cw = nullptr;  // FP64 working copy of the coarsest block
  double *E[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // pipelined BiCGStab: Z, Q, Y, U, X0
  double *part[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  ColState *cs = nullptr;
};

// The block scalar's view of the hierarchy and the work blocks.
template <class TB> struct Blocks;
template <> struct Blocks<double> {
  static double *b(Work &W, int l) { return W.vb[l]; }
  static double *x(Work &W, int l) { return W.vx[l]; }
  static double *r(Work &W, int l) { return W.vr[l]; }
  static double *d(Work &W, int l) { return W.vd[l]; }
  static double *d2(Work &W, int l) { return W.vd2[l]; }
  static const double *w(const DevLevel &D, int k) { return D.w[k]; }
  static double c1(const DevLevel &D, int k) { return D.c1[k]; }
};
template <> struct Blocks<float> {
  static float *b(Work &W, int l) { return W.fb[l]; }
  static float *x(Work &W, int l) { return W.fx[l]; }
  static float *r(Work &W, int l) { return W.fr[l]; }
  static float *d(Work &W, int l) { return W.fd[l]; }
  static float *d2(Work &W, int l) { return W.fd2[l]; }
  static const float *w(const DevLevel &D, int k) { return D.w32[k]; }
  static float c1(const DevLevel &D, int k) { return D.c1f[k]; }
};

}  // namespace

// One captured steady iteration: the kernels of V-cycle, beta, direction
// update, A p, alpha, x/r update and convergence test, with the arguments of
// this key (block width, preconditioner precision, workspace, tolerance).
struct GraphRec {
  int nv = 0, prec = 0;
  const void *ws = nullptr;
  double tol = 0.0;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;  // kernels per replay
};

struct xamg_hier {
  HostHier host;
  xamg_amg_params prm{};
  bool on_device = false;
  int device = 0;
  std::vector<DevLevel> lv;
  double *ainv = nullptr;     // inverse of the coarsest operator (nc x nc, row-major)
  std::vector<void *> owned;  // device allocations of the hierarchy
  void *ws = nullptr;         // cached solve workspace
  size_t ws_bytes = 0;
  double *hb = nullptr;       // staging blocks of xamg_solve_host
  size_t hb_bytes = 0;
  Flags *flags_h = nullptr;   // mapped pinned counters
  Flags *flags_d = nullptr;
  bool lowp_ready = false;    // reduced-precision copies uploaded
  // 16-bit column indices in the reduced-precision products (off by default:
  // measured slower at every block width, xamg_set_index16)
  bool use_idx16 = false;
  bool timing = false;
  std::vector<TimerRec> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<TimeAcc> tacc;  // [level * 3 + which]
  // CUDA graphs of the steady PCG iteration (capture stream, cache); cleared
  // whenever what they captured may change (workspace, row splits)
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  std::vector<GraphRec> graphs;
  // fused coarse tail of the V-cycle (vtail.cuh): levels whose blocks hold at
  // most tail_elems elements (rows x block width) run as one cooperative
  // launch; 0 (the default: measured slower than graph-replayed launches)
  // turns it off.  tail_limit_s bounds each grid-barrier wait; tail_extra is
  // added to the barrier's expected arrivals (fault injection)
  int64_t tail_elems = 0;
  double tail_limit_s = 2.0;
  int tail_extra = 0;
  TailSync *tail_sync = nullptr;  // device barrier words
  // while a tail program is being recorded: the program (TailProg<TB> of the
  // recording vcycle's block scalar) and whether every stage fit it
  void *rec = nullptr;
  bool rec_ok = true;
  std::unique_ptr<TailProg<double>> tp64;
  std::unique_ptr<TailProg<float>> tp32;
};

namespace {

#define XCK(call)                              \
  do {                                         \
    cudaError_t e__ = (call);                  \
    if (e__ != cudaSuccess) {                  \
      return e__ == cudaErrorMemoryAllocation ? XAMG_ERR_OOM : XAMG_ERR_CUDA; \
    }                                          \
  } while (0)

int pad_nv(int m) {
  int v = 1;
  while (v < m) v <<= 1;
  return v;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <class T>
int dev_upload(xamg_hier *h, T **dst, const T *src, size_t count) {
  *dst = nullptr;
  if (count == 0) return XAMG_OK;
  void *p = nullptr;
  XCK(cudaMalloc(&p, count * sizeof(T)));
  h->owned.push_back(p);
  XCK(cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice));
  *dst = (T *)p;
  return XAMG_OK;
}

int upload_csr(xamg_hier *h, const HostCsr &a, DevCsr &d) {
  d.n = a.n;
  d.ncols = a.ncols;
  d.nnz = a.nnz();
  for (int t = 0; t < 3; ++t) {
    const int rpw = 4 << t;
    int mx = 0;
    for (int r0 = 0; r0 < a.n; r0 += rpw)
      mx = std::max(mx, a.rowptr[std::min(a.n, r0 + rpw)] - a.rowptr[r0]);
    d.span[t] = mx;
  }
  int rc;
  if ((rc = dev_upload(h, &d.rowptr, a.rowptr.data(), a.rowptr.size())) != XAMG_OK) return rc;
  if ((rc = dev_upload(h, &d.col, a.col.data(), a.col.size())) != XAMG_OK) return rc;
  return dev_upload(h, &d.val, a.val.data(), a.val.size());
}

// Chebyshev coefficients of level l (interval [lo, hi] of D^-1 A):
//   theta = (hi+lo)/2, delta = (hi-lo)/2, sigma = theta/delta, rho_0 = 1/sigma
//   step 0: d_0 = (D^-1 / theta) r_0
//   step k: rho_k = 1/(2 sigma - rho_{k-1}), d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k/delta) D^-1 r_k
// Inverse of the coarsest operator from its LU factors (partial pivoting,
// unit lower L): column j solves A x = e_j by the row interchanges, then
// forward and back substitution.  Row-major nc x nc.
std::vector<double> lu_inverse(int nc, const std::vector<double> &lu, const std::vector<int32_t> &piv) {
  std::vector<double> inv((size_t)nc * nc), x(nc);
  for (int j = 0; j < nc; ++j) {
    std::fill(x.begin(), x.end(), 0.0);
    x[j] = 1.0;
    for (int k = 0; k < nc; ++k)
      if (piv[k] != k) std::swap(x[k], x[piv[k]]);
    for (int i = 1; i < nc; ++i)
      for (int k = 0; k < i; ++k) x[i] -= lu[(size_t)i * nc + k] * x[k];
    for (int i = nc - 1; i >= 0; --i) {
      for (int k = i + 1; k < nc; ++k) x[i] -= lu[(size_t)i * nc + k] * x[k];
      x[i] /= lu[(size_t)i * nc + i];
    }
    for (int i = 0; i < nc; ++i) inv[(size_t)i * nc + j] = x[i];
  }
  return inv;
}

int upload_level(xamg_hier *h, int l) {
  const HostLevel &H = h->host.lv[l];
  DevLevel &D = h->lv[l];
  int rc;
  if ((rc = upload_csr(h, H.A, D.A)) != XAMG_OK) return rc;
  const bool coarsest = l + 1 == (int)h->host.lv.size();
  if (coarsest) return XAMG_OK;
  if ((rc = upload_csr(h, H.P, D.P)) != XAMG_OK) return rc;
  if ((rc = upload_csr(h, H.R, D.R)) != XAMG_OK) return rc;
  const double theta = 0.5 * (H.hi + H.lo), delta = 0.5 * (H.hi - H.lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  std::vector<double> w(H.dinv.size());
  for (int k = 0; k < h->host.cheb_steps; ++k) {
    double coef;
    if (k == 0) {
      coef = 1.0 / theta;
      D.c1[0] = 0.0;
    } else {
      const double rn = 1.0 / (2.0 * sigma - rho);
      D.c1[k] = rn * rho;
      coef = 2.0 * rn / delta;
      rho = rn;
    }
    for (size_t i = 0; i < w.size(); ++i) w[i] = coef * H.dinv[i];
    if ((rc = dev_upload(h, &D.w[k], w.data(), w.size())) != XAMG_OK) return rc;
  }
  return XAMG_OK;
}

// 16-bit column indices of one operator in the segmented form of
// kernels.cuh (seg16_col; paper Sec. 2.3: CSR index types reduced to
// uint16_t).  Each tile of kSegTile rows takes its segment bases greedily
// over the sorted columns of its rows: a base is the first column not covered
// by the previous segment [b, b + 65535].  The operator keeps its 32-bit
// indices (*w, *m, *tb stay null) when a tile needs more than kSegs
// segments or a row's boundary lies at an entry position beyond 1022.
int upload_idx16(xamg_hier *h, const HostCsr &M, uint16_t **w, uint32_t **m, int32_t **tb) {
  *w = nullptr;
  *m = nullptr;
  *tb = nullptr;
  if (M.n == 0 || M.col.empty()) return XAMG_OK;
  const int tiles = (M.n + kSegTile - 1) / kSegTile;
  std::vector<uint16_t> off(M.col.size());
  std::vector<uint32_t> meta((size_t)M.n);
  std::vector<int32_t> base((size_t)tiles * kSegs, 0);
  std::vector<int32_t> cols;
  for (int t = 0; t < tiles; ++t) {
    const int r0 = t * kSegTile, r1 = std::min(M.n, r0 + kSegTile);
    cols.assign(M.col.begin() + M.rowptr[r0], M.col.begin() + M.rowptr[r1]);
    std::sort(cols.begin(), cols.end());
    int nseg = 0;
    int32_t *b = &base[(size_t)t * kSegs];
    for (int32_t c : cols) {
      if (nseg == 0 || (int64_t)c - b[nseg - 1] > 65535) {
        if (nseg == kSegs) return XAMG_OK;
        b[nseg++] = c;
      }
    }
    for (int s = std::max(nseg, 1); s < kSegs; ++s) b[s] = b[s - 1];
    for (int i = r0; i < r1; ++i) {
      uint32_t e[3] = {(uint32_t)kSegNone, (uint32_t)kSegNone, (uint32_t)kSegNone};
      int seg = 0;
      // a row past position 1022 decodes as segment 0 only when the tile has
      // one segment
      if (nseg > 1 && M.rowptr[i + 1] - M.rowptr[i] > kSegNone) return XAMG_OK;
      for (int p = M.rowptr[i]; p < M.rowptr[i + 1]; ++p) {
        const int k = p - M.rowptr[i];
        while (seg + 1 < nseg && M.col[p] >= b[seg + 1]) {
          ++seg;
          if (k >= kSegNone) return XAMG_OK;
          e[seg - 1] = (uint32_t)k;  // entries before k lie below segment seg
        }
        off[p] = (uint16_t)(M.col[p] - b[seg]);
      }
      // a boundary that no entry of the row crosses stays kSegNone, above
      // every position of the row
      meta[i] = e[0] | e[1] << 10 | e[2] << 20;
    }
  }
  int rc;
  if ((rc = dev_upload(h, w, off.data(), off.size())) != XAMG_OK) return rc;
  if ((rc = dev_upload(h, m, meta.data(), meta.size())) != XAMG_OK) return rc;
  return dev_upload(h, tb, base.data(), base.size());
}

// Reduced-precision copies of the hierarchy for the FP32-block preconditioner:
// fl32 of every value of A, P, R; bf16 values of A relative to the row scale
// s_i = fl32(max_j |a_ij|), q_ij = bf16_rne(fl32(a_ij) / s_i); the Chebyshev
// row weights and step coefficients rounded to FP32.
int upload_lowp(xamg_hier *h) {
  if (h->lowp_ready) return XAMG_OK;
  const int L = (int)h->host.lv.size();
  int rc;
  for (int l = 0; l < L; ++l) {
    const HostLevel &H = h->host.lv[l];
    DevLevel &D = h->lv[l];
    std::vector<float> f(H.A.val.size());
    for (size_t k = 0; k < f.size(); ++k) f[k] = (float)H.A.val[k];
    if ((rc = dev_upload(h, &D.a32, f.data(), f.size())) != XAMG_OK) return rc;
    std::vector<float> s((size_t)H.A.n);
    std::vector<__nv_bfloat16> q(H.A.val.size());
    for (int i = 0; i < H.A.n; ++i) {
      double mx = 0.0;
      for (int p = H.A.rowptr[i]; p < H.A.rowptr[i + 1]; ++p) mx = std::max(mx, std::fabs(H.A.val[p]));
      s[i] = mx > 0.0 ? (float)mx : 1.0f;
      for (int p = H.A.rowptr[i]; p < H.A.rowptr[i + 1]; ++p) q[p] = __float2bfloat16_rn(f[p] / s[i]);
    }
    // an even number of values: the m = 1 stream kernel copies aligned pairs
    if (q.size() & 1) q.push_back(__float2bfloat16_rn(0.0f));
    if ((rc = dev_upload(h, &D.a16, q.data(), q.size())) != XAMG_OK) return rc;
    if ((rc = dev_upload(h, &D.a16s, s.data(), s.size())) != XAMG_OK) return rc;
    if ((rc = upload_idx16(h, H.A, &D.w16[0], &D.m16[0], &D.t16[0])) != XAMG_OK) return rc;
    if (l + 1 == L) continue;
    std::vector<float> pf(H.P.val.size()), rf(H.R.val.size());
    for (size_t k = 0; k < pf.size(); ++k) pf[k] = (float)H.P.val[k];
    for (size_t k = 0; k < rf.size(); ++k) rf[k] = (float)H.R.val[k];
    if ((rc = dev_upload(h, &D.p32, pf.data(), pf.size())) != XAMG_OK) return rc;
    if ((rc = dev_upload(h, &D.r32, rf.data(), rf.size())) != XAMG_OK) return rc;
    if ((rc = upload_idx16(h, H.P, &D.w16[1], &D.m16[1], &D.t16[1])) != XAMG_OK) return rc;
    if ((rc = upload_idx16(h, H.R, &D.w16[2], &D.m16[2], &D.t16[2])) != XAMG_OK) return rc;
    const double theta = 0.5 * (H.hi + H.lo), delta = 0.5 * (H.hi - H.lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    std::vector<float> w(H.dinv.size());
    for (int k = 0; k < h->host.cheb_steps; ++k) {
      double coef;
      if (k == 0) {
        coef = 1.0 / theta;
        D.c1f[0] = 0.0f;
      } else {
        const double rn = 1.0 / (2.0 * sigma - rho);
        D.c1f[k] = (float)(rn * rho);
        coef = 2.0 * rn / delta;
        rho = rn;
      }
      for (size_t i = 0; i < w.size(); ++i) w[i] = (float)(coef * H.dinv[i]);
      if ((rc = dev_upload(h, &D.w32[k], w.data(), w.size())) != XAMG_OK) return rc;
    }
  }
  h->lowp_ready = true;
  return XAMG_OK;
}

void clear_graphs(xamg_hier *h) {
  for (auto &g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

void free_device(xamg_hier *h) {
  clear_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  h->cap_stream = nullptr;
  for (void *p : h->owned) cudaFree(p);
  h->owned.clear();
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  if (h->hb) cudaFree(h->hb);
  h->hb = nullptr;
  h->hb_bytes = 0;
  if (h->flags_h) cudaFreeHost(h->flags_h);
  h->flags_h = nullptr;
  h->flags_d = nullptr;
  for (auto &p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  h->pending.clear();
  for (auto e : h->event_pool) cudaEventDestroy(e);
  h->event_pool.clear();
}

// ---- workspace ----
size_t plan(const xamg_hier *h, int nv, int method, int prec, Work *w, char *base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char * {
    char *p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const size_t n0 = (size_t)h->host.lv[0].A.n;
  const size_t blk = n0 * nv * sizeof(double);
  Work tmp;
  Work &W = w ? *w : tmp;
  W.nv = nv;
  W.Bn = (double *)take(blk);
  W.X = (double *)take(blk);
  W.R = (double *)take(blk);
  W.P = (double *)take(blk);
  if (method == XAMG_PCG) {
    W.Z = (double *)take(blk);
    W.Q = (double *)take(blk);
  } else {
    W.RH = (double *)take(blk);
    W.V = (double *)take(blk);
    W.S = (double *)take(blk);
    W.T = (double *)take(blk);
    W.PH = (double *)take(blk);
    W.SH = (double *)take(blk);
    if (method == XAMG_BICGSTAB_PIPELINED)
      for (int i = 0; i < 5; ++i) W.E[i] = (double *)take(blk);
  }
  const int L = (int)h->host.lv.size();
  const bool dd = h->host.cheb_steps >= 3;
  W.vb.assign(L, nullptr);
  W.vx.assign(L, nullptr);
  W.vr.assign(L, nullptr);
  W.vd.assign(L, nullptr);
  W.vd2.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    const size_t b = (size_t)h->host.lv[l].A.n * nv * sizeof(double);
    if (l > 0) {
      W.vb[l] = (double *)take(b);
      W.vx[l] = (double *)take(b);
    }
    if (l + 1 < L) {
      W.vr[l] = (double *)take(b);
      W.vd[l] = (double *)take(b);
      if (dd) W.vd2[l] = (double *)take(b);
    }
  }
  W.fb.assign(L, nullptr);
  W.fx.assign(L, nullptr);
  W.fr.assign(L, nullptr);
  W.fd.assign(L, nullptr);
  W.fd2.assign(L, nullptr);
  W.R32 = W.Z32 = nullptr;
  W.cw = nullptr;
  if (prec != XAMG_PREC_FP64) {
    const size_t fblk = n0 * nv * sizeof(float);
    W.R32 = (float *)take(fblk);
    W.Z32 = (float *)take(fblk);
    W.fb[0] = W.R32;
    W.fx[0] = W.Z32;
    for (int l = 0; l < L; ++l) {
      const size_t b = (size_t)h->host.lv[l].A.n * nv * sizeof(float);
      if (l > 0) {
        W.fb[l] = (float *)take(b);
        W.fx[l] = (float *)take(b);
      }
      if (l + 1 < L) {
        W.fr[l] = (float *)take(b);
        W.fd[l] = (float *)take(b);
        if (dd) W.fd2[l] = (float *)take(b);
      }
    }
    W.cw = (double *)take((size_t)h->host.nc * nv * sizeof(double));
  }
  for (int i = 0; i < 5; ++i) W.part[i] = (double *)take((size_t)kMaxGrid * 32 * sizeof(double));
  W.cs = (ColState *)take(sizeof(ColState));
  return off;
}

int ensure_workspace(xamg_hier *h, int nv, int method, int prec, const xamg_solve_opts *o,
                     Work &w) {
  if (prec != XAMG_PREC_FP64) {
    const int rc = upload_lowp(h);
    if (rc != XAMG_OK) return rc;
  }
  const size_t need = plan(h, nv, method, prec, nullptr, nullptr);
  char *base;
  if (o && o->workspace) {
    if (o->workspace_bytes < need || ((uintptr_t)o->workspace & 255)) return XAMG_ERR_INVALID_ARG;
    base = (char *)o->workspace;
  } else {
    if (h->ws_bytes < need) {
      clear_graphs(h);  // they captured addresses in the old workspace
      if (h->ws) cudaFree(h->ws);
      h->ws = nullptr;
      h->ws_bytes = 0;
      XCK(cudaMalloc(&h->ws, need));
      h->ws_bytes = need;
    }
    base = (char *)h->ws;
  }
  plan(h, nv, method, prec, &w, base);
  return XAMG_OK;
}

// ---- timing ----
cudaEvent_t pool_event(xamg_hier *h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void flush_timing(xamg_hier *h) {
  for (auto &p : h->pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      TimeAcc &t = h->tacc[(size_t)p.level * 6 + p.which];
      t.launches++;
      t.ms += ms;
      t.flops += p.flops;
      t.bytes += p.bytes;
    }
    h->event_pool.push_back(p.a);
    h->event_pool.push_back(p.b);
  }
  h->pending.clear();
}

// ---- row kernel wrapper ----
// Blocks of 2 or 4 columns (8- to 32-byte rows) can take the stream kernel
// with one lane per row (rows_stream_v).
bool stream_v_ok(int nv, bool /*fp32*/) { return nv == 2 || nv == 4; }
// FP64 blocks of 8 or more columns can take the pipelined narrow split.
bool pipe_ok(int nv, bool fp32) { return !fp32 && nv >= 8; }

// Whether the staged FP32 narrow kernel (rows_async) can take operator M on
// blocks of nv columns: every aligned group of a warp's rows fits its window.
bool async_fits(const DevCsr &M, int nv, bool fp32) {
  if (!fp32 || nv < 8) return false;
  const int t = nv == 32 ? 0 : nv == 16 ? 1 : 2;
  const int window[3] = {async_window<32>(), async_window<16>(), async_window<8>()};
  return M.span[t] <= window[t];
}

// m = 1: 4 or 16 lanes per row.  FP32 blocks of >= 16 columns with long rows
// (the dense coarse Galerkin levels): one row per warp, split into slices.
int slices_for(const DevCsr &M, int nv, bool fp32) {
  if (M.n == 0) return 1;
  const double avg = (double)M.nnz / M.n;
  // m = 1: the stream kernel with as many lanes per row as keep a chunk's
  // rows inside one window (32 x 7.5 = 240 of 256 entries, 32 x 30 = 960 of
  // 1024; 4 lanes per row up to 64 entries), 16 lanes per row beyond, which
  // measured fastest on the dense Galerkin levels
  if (nv == 1)
    return avg <= 7.5 ? kStreamShort : avg <= 30.0 ? kStreamLong : avg <= 64.0 ? kStreamQuad : kSliced16;
  if (fp32 && nv >= 16 && avg >= 64.0) return 32 / (nv / 4);
  // a dense Galerkin level with fewer row groups than resident warps under the
  // default split (rows per warp = 32 / lanes per row): one row per warp, the
  // row's entries split over the warp
  const int vec = fp32 ? (nv >= 4 ? 4 : nv) : 1;
  const double warps = (double)M.n / (32 / (nv / vec));
  // FP64 blocks of 16 and 32 columns, whose wide split spreads a row over
  // four warps, take it below two waves of narrow warps: measured faster from
  // 11 696 rows (1 025 entries) down at 16 columns and 5 739 (1 537) at 32
  const double waves = (!fp32 && nv >= 16) ? 2.0 : 1.0;
  if (avg >= 32.0 && warps < waves * 32.0 * device_sm_count()) return 2;
  // 2- and 4-column blocks on sparse levels: one lane per row over the warp's
  // staged entries (measured per level at m = 2 and 4 on the 7- and 27-point
  // hierarchies: FP64 faster up to 27 entries per row and slower at 35; FP32
  // faster from 19 to 35 and slower at 7).  FP64 levels below 131 072 rows
  // keep the narrow split: its blocks hold a quarter (m = 4) or half (m = 2)
  // of the stream kernel's 256 rows, so small levels still fill the GPU
  // (CUDA-graph solves of the 7-point 32^3 and 48^3 cases, m = 4, measured
  // 5 % faster that way; 64^3 and above at most 1 % apart).  FP32 levels of
  // short rows below 131 072 rows take the stream kernel, latency-bound
  // there (2 % faster solves at 32^3 and 48^3, 2 % slower at 96^3)
  const bool small = M.n < 131072;
  if (stream_v_ok(nv, fp32) &&
      (fp32 ? ((avg > 10.0 || small) && avg <= 40.0) : (avg <= 30.0 && !small)))
    return kStreamV1024;
  // FP64 blocks of 8, 16 and 32 columns: the pipelined narrow split on levels
  // of more than 10 entries per row (measured 3 to 7 % faster per launch on
  // levels 1 to 6 of the 7-point 192^3 hierarchy at m = 32, 3 % slower on
  // level 0 with its 7 entries per row, where the fourth block per SM pays
  // more than the pipeline).  Two columns per lane (a warp on two rows) on
  // the sparser levels: level 0 6-9 % faster at m = 8, 16 and 32, level 1
  // (18.8 entries per row) 4 % at m = 32, 17 % at m = 8 and 21 % at m = 16,
  // level 2 (34.7) 8-10 % at m = 8 and 16 but 3 % slower at m = 32, the
  // denser levels 4-13 % slower at m = 16 and 32
  if (pipe_ok(nv, fp32)) {
    if (avg <= 10.0) return kNarrow2;
    if (avg <= 20.0 || (nv <= 16 && avg <= 40.0)) return kPipeNarrow2;
    return kPipeNarrow;
  }
  // (the staged narrow split, kAsyncNarrow, is a tuning candidate only: it
  // measured slower than this one on every level it fits)
  return 1;
}

// Row split of tuning candidate t: m = 1 has seven (the stream-kernel
// variants and 16 lanes per row, launch.h), wider blocks two (narrow, one row
// per warp) and a third where one exists: blocks of 8 or more FP32 columns
// the staged narrow split, blocks of 2 or 4 columns the stream kernel, FP64
// blocks of 8 or more columns the pipelined narrow split, and for those two
// more, the narrow split and its pipelined form with two columns per lane.
int split_candidates(int nv, bool fp32) {
  if (nv == 1) return 7;
  if (pipe_ok(nv, fp32)) return 5;
  return ((fp32 && nv >= 8) || stream_v_ok(nv, fp32)) ? 3 : 2;
}
int split_slices(int nv, int t, bool fp32) {
  if (nv == 1) {
    static const int c[7] = {kStreamShort, kSliced16, kStreamLong, kStreamQuad, kStreamWarp, kStreamMid,
                             kStreamPair};
    return c[t];
  }
  if (t == 2) return fp32 && nv >= 8 ? kAsyncNarrow : stream_v_ok(nv, fp32) ? kStreamV1024 : kPipeNarrow;
  if (t == 3) return kNarrow2;
  if (t == 4) return kPipeNarrow2;
  return t ? 2 : 1;
}

// Algorithmic bytes of one fused row launch: the matrix once, the operand
// block once, and every block the epilogue reads or writes once.
template <class TB>
double row_bytes(const DevCsr &M, const RowOpT<TB> &op, int nv, double val_bytes) {
  const double blk = (double)M.n * nv * sizeof(TB);
  const double idx_bytes = op.colw ? 2.0 : 4.0;
  double b = (idx_bytes + val_bytes) * (double)M.nnz + 4.0 * (M.n + 1) + (double)M.ncols * nv * sizeof(TB);
  if (op.rscale) b += 4.0 * M.n;
  if (op.rowmeta) b += 4.0 * M.n + 16.0 * ((M.n + kSegTile - 1) / kSegTile);
  if (op.init) b += blk;
  if (op.y) b += blk;
  if (op.dp) b += blk;
  if (op.w) b += (double)M.n * sizeof(TB);
  if (op.dnext) b += blk;
  if (op.x) b += 2 * blk;
  if (op.dot_u) b += (double)M.n * nv * 8.0;
  if (op.dot_u2) b += (double)M.n * nv * 8.0;
  return b;
}

// Operator `which` (0 = A, 1 = P, 2 = R) of level `level` with the values of
// block scalar TB and preconditioner precision `prec`.
template <class TB>
int rows(xamg_hier *h, int level, int which, int prec, RowOpT<TB> op, int nv, bool neg, int epi,
         cudaStream_t st) {
  const DevLevel &D = h->lv[level];
  const DevCsr &M = which == 0 ? D.A : which == 1 ? D.P : D.R;
  op.n = M.n;
  op.rowptr = M.rowptr;
  op.col = M.col;
  int vt = 0;
  double vbytes = 8.0;
  if constexpr (sizeof(TB) == 8) {
    op.val = M.val;
    op.rscale = nullptr;
  } else {
    vbytes = 4.0;
    // 16-bit column indices (wider blocks; m = 1 reads the 32-bit ones)
    const bool i16 = h->use_idx16 && D.w16[which] && nv > 1;
    if (i16) {
      op.colw = D.w16[which];
      op.rowmeta = D.m16[which];
      op.tbase = D.t16[which];
    }
    if (which == 0 && prec == XAMG_PREC_BF16) {
      op.val = D.a16;
      op.rscale = D.a16s;
      vt = i16 ? 2 : 1;
      vbytes = 2.0;
    } else {
      op.val = which == 0 ? D.a32 : which == 1 ? D.p32 : D.r32;
      op.rscale = nullptr;
      vt = i16 ? 3 : 0;
    }
  }
  if (h->rec) {
    // recording a tail program: the stage runs later inside the cooperative
    // kernel, with the split this launch would take and 32-bit indices
    int sl = slices_for(M, nv, sizeof(TB) == 4);
    int lg = 0;
    while ((1 << lg) < nv) ++lg;
    const int t = D.split[sizeof(TB) == 8 ? 2 : ((vt == 1 || vt == 2) ? 1 : 0)][which][lg];
    if (t >= 0) sl = split_slices(nv, t, sizeof(TB) == 4);
    op.colw = nullptr;
    op.rowmeta = nullptr;
    op.tbase = nullptr;
    int kind = -1;
    if (which == 0 && neg && epi == EPI_Y_DN) kind = TK_A_YDN;
    else if (which == 0 && neg && epi == EPI_Y_XDP) kind = TK_A_YXDP;
    else if (which == 0 && neg && epi == EPI_Y_D0) kind = TK_A_YD0;
    else if (which == 0 && neg && epi == EPI_XLAST) kind = TK_A_XLAST;
    else if (which != 0 && !neg && epi == EPI_Y) kind = TK_PR_Y;
    else if (which == 2 && !neg && epi == EPI_Y_D0) kind = TK_PR_YD0;
    TailProg<TB> *prog = static_cast<TailProg<TB> *>(h->rec);
    if (kind < 0 || nv < 2 || prog->nstages >= kTailMaxStages) {
      h->rec_ok = false;
      return 1;
    }
    TailStage<TB> &s = prog->st[prog->nstages++];
    s.op = op;
    s.kind = kind;
    s.wide = sl > 1 && sl < kAsyncNarrow ? 1 : 0;  // the staged / stream / pipelined codes sum as the narrow split
    return 1;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->timing) {
    a = pool_event(h);
    b = pool_event(h);
    cudaEventRecord(a, st);
  }
  int g;
  if constexpr (sizeof(TB) == 8) {
    int sl = slices_for(M, nv, false);
    int lg = 0;
    while ((1 << lg) < nv) ++lg;
    const int t = D.split[2][which][lg];
    if (t >= 0) sl = split_slices(nv, t, false);
    g = launch_rows(op, nv, sl, neg, epi, st);
  } else {
    int sl = slices_for(M, nv, true);
    int lg = 0;
    while ((1 << lg) < nv) ++lg;
    const int t = D.split[(vt == 1 || vt == 2) ? 1 : 0][which][lg];
    if (t >= 0) sl = split_slices(nv, t, true);
    if (sl == kAsyncNarrow && !async_fits(M, nv, true)) sl = 1;
    g = launch_rows_f(op, nv, sl, neg, epi, vt, st);
  }
  if (h->timing) {
    cudaEventRecord(b, st);
    const int slot = which + (sizeof(TB) == 8 ? 0 : 3);
    h->pending.push_back({a, b, level, slot, 2.0 * (double)M.nnz * nv, row_bytes(M, op, nv, vbytes)});
  }
  return g;
}

template <class TB>
RowOpT<TB> blank() {
  RowOpT<TB> o;
  std::memset(&o, 0, sizeof(o));
  return o;
}

// ---- Chebyshev smoothing (cheb_steps steps) on level l ----
// Pre-smoothing from x = 0: on entry x holds d_0 = w_0 .* b (= x_1); on exit
// x holds the smoothed iterate and r = b - A x.
template <class TB>
int presmooth(xamg_hier *h, Work &W, int prec, int l, const TB *b, TB *x, TB *r, cudaStream_t st) {
  using BL = Blocks<TB>;
  const int nv = W.nv;
  const int s = h->host.cheb_steps;
  const DevLevel &D = h->lv[l];
  TB *dA = BL::d(W, l), *dB = BL::d2(W, l);
  if (s == 1) {
    RowOpT<TB> o = blank<TB>();
    o.init = b; o.src = x; o.y = r;
    return rows<TB>(h, l, 0, prec, o, nv, true, EPI_Y, st) < 0 ? XAMG_ERR_CUDA : XAMG_OK;
  }
  RowOpT<TB> o = blank<TB>();
  o.init = b; o.src = x; o.y = r; o.dp = x; o.w = BL::w(D, 1); o.c1 = BL::c1(D, 1); o.dnext = dA;
  if (rows<TB>(h, l, 0, prec, o, nv, true, EPI_Y_DN, st) < 0) return XAMG_ERR_CUDA;
  TB *dprev = dA, *dnext = dB;
  for (int k = 2; k < s; ++k) {
    RowOpT<TB> m = blank<TB>();
    m.init = r; m.src = dprev; m.y = r; m.dp = dprev; m.w = BL::w(D, k); m.c1 = BL::c1(D, k);
    m.dnext = dnext; m.x = x;
    if (rows<TB>(h, l, 0, prec, m, nv, true, EPI_MID, st) < 0) return XAMG_ERR_CUDA;
    std::swap(dprev, dnext);
  }
  RowOpT<TB> f = blank<TB>();
  f.init = r; f.src = dprev; f.y = r; f.dp = dprev; f.x = x;
  return rows<TB>(h, l, 0, prec, f, nv, true, EPI_Y_XDP, st) < 0 ? XAMG_ERR_CUDA : XAMG_OK;
}

// FP64 partial dots of the final iterate: dot_u . x into dot_part and, when
// dot_u2 is set, dot_u2 . x into dot_part2; *dot_grid gets their block count.
struct Dots {
  const double *u = nullptr, *u2 = nullptr;
  double *part = nullptr, *part2 = nullptr;
  int *grid = nullptr;
};

// Post-smoothing of x (r is scratch), in two parts: the first step (r = b -
// A x, d_0 = w_0 r), then the rest (the fused coarse tail ends between them).
template <class TB>
int postsmooth_first(xamg_hier *h, Work &W, int prec, int l, const TB *b, TB *x, TB *r, cudaStream_t st) {
  using BL = Blocks<TB>;
  const DevLevel &D = h->lv[l];
  RowOpT<TB> o = blank<TB>();
  o.init = b; o.src = x; o.y = r; o.w = BL::w(D, 0); o.dnext = BL::d(W, l);
  return rows<TB>(h, l, 0, prec, o, W.nv, true, EPI_Y_D0, st) < 0 ? XAMG_ERR_CUDA : XAMG_OK;
}

template <class TB>
int postsmooth_rest(xamg_hier *h, Work &W, int prec, int l, TB *x, TB *r, cudaStream_t st,
                    const Dots &dots) {
  using BL = Blocks<TB>;
  const int nv = W.nv;
  const int s = h->host.cheb_steps;
  const DevLevel &D = h->lv[l];
  TB *dA = BL::d(W, l), *dB = BL::d2(W, l);
  if (s == 1) {
    const int g = elem_grid(D.A.n, nv);
    if constexpr (sizeof(TB) == 8) {
      launch_axpy_dot(nv, D.A.n, x, dA, dots.part ? dots.u : nullptr, dots.part, g, st);
      if (dots.part2) launch_coldot(nv, D.A.n, dots.u2, x, dots.part2, g, st);
    } else {
      launch_axpy_dot_f(nv, D.A.n, x, dA, dots.part ? dots.u : nullptr,
                        dots.part2 ? dots.u2 : nullptr, dots.part, dots.part2, g, st);
    }
    if (dots.part) *dots.grid = g;
    return XAMG_OK;
  }
  TB *dprev = dA, *dnext = dB;
  for (int k = 1; k < s; ++k) {
    const bool last = k == s - 1;
    RowOpT<TB> o = blank<TB>();
    o.init = r; o.src = dprev; o.dp = dprev; o.w = BL::w(D, k); o.c1 = BL::c1(D, k); o.x = x;
    int epi = EPI_MID;
    if (last) {
      epi = EPI_XLAST;
      if (dots.part) {
        o.dot_u = dots.u;
        o.partials = dots.part;
        epi = EPI_XLAST_DOT;
        if (dots.part2) {
          o.dot_u2 = dots.u2;
          o.partials2 = dots.part2;
          epi = EPI_XLAST_DOT2;
        }
      }
    } else {
      o.y = r;
      o.dnext = dnext;
    }
    const int g = rows<TB>(h, l, 0, prec, o, nv, true, epi, st);
    if (g < 0) return XAMG_ERR_CUDA;
    if (last && dots.part) *dots.grid = g;
    std::swap(dprev, dnext);
  }
  return XAMG_OK;
}

// ---- fused coarse tail (vtail.cuh) ----
// First level of the tail for blocks of nv columns: the smallest l such that
// every level from l down holds at most tail_elems block elements, with at
// least one level above the coarsest and its stages within kTailMaxStages;
// -1: no tail (off, m = 1, or a smoother other than two Chebyshev steps).
int tail_start(const xamg_hier *h, int nv) {
  const int L = (int)h->lv.size();
  // (timing measures the unfused row launches, so it takes the plain cycle)
  if (h->tail_elems <= 0 || h->timing || nv < 2 || h->host.cheb_steps != 2 || L < 2) return -1;
  int l = L - 1;
  while (l > 0 && (int64_t)h->lv[l - 1].A.n * nv <= h->tail_elems && 6 * (L - l) <= kTailMaxStages) --l;
  return l <= L - 2 ? l : -1;
}

template <class TB> TailProg<TB> &tail_prog(xamg_hier *h);
template <> TailProg<double> &tail_prog<double>(xamg_hier *h) {
  if (!h->tp64) h->tp64.reset(new TailProg<double>());
  return *h->tp64;
}
template <> TailProg<float> &tail_prog<float>(xamg_hier *h) {
  if (!h->tp32) h->tp32.reset(new TailProg<float>());
  return *h->tp32;
}

template <class TB>
int vcycle(xamg_hier *h, Work &W, int prec, int l, const TB *b, TB *x, cudaStream_t st,
           const Dots &dots);

// The cycle from level l with its coarse part fused: the stages from the
// pre-smoothing of l down to the coarsest and back up to the first
// post-smoothing step of l are recorded (rows() in record mode) and run as one
// cooperative launch; the last post-smoothing step of l, which may carry the
// caller's dots, is launched as usual.  XAMG_ERR_SETUP: a stage did not fit
// the tail program (nothing was launched).
template <class TB>
int vcycle_tail(xamg_hier *h, Work &W, int prec, int l, const TB *b, TB *x, cudaStream_t st,
                const Dots &dots) {
  using BL = Blocks<TB>;
  const int nv = W.nv;
  if (!h->tail_sync) {
    void *p = nullptr;
    XCK(cudaMalloc(&p, sizeof(TailSync)));
    h->owned.push_back(p);
    h->tail_sync = static_cast<TailSync *>(p);
  }
  TailProg<TB> &prog = tail_prog<TB>(h);
  prog.nstages = 0;
  prog.extra = h->tail_extra;
  prog.limit_ns = (unsigned long long)(h->tail_limit_s * 1e9);
  prog.sync = h->tail_sync;
  prog.err_host = &h->flags_d->tail_err;
  h->rec = &prog;
  h->rec_ok = true;
  TB *r = BL::r(W, l);
  int rc = presmooth<TB>(h, W, prec, l, b, x, r, st);
  if (rc == XAMG_OK) {
    const bool next_coarsest = l + 2 == (int)h->lv.size();
    RowOpT<TB> o = blank<TB>();
    o.src = r; o.y = BL::b(W, l + 1);
    if (!next_coarsest) {
      o.w = BL::w(h->lv[l + 1], 0);
      o.dnext = BL::x(W, l + 1);
    }
    rows<TB>(h, l, 2, prec, o, nv, false, next_coarsest ? EPI_Y : EPI_Y_D0, st);
    rc = vcycle<TB>(h, W, prec, l + 1, BL::b(W, l + 1), BL::x(W, l + 1), st, Dots());
  }
  if (rc == XAMG_OK) {
    RowOpT<TB> o = blank<TB>();
    o.init = x; o.src = BL::x(W, l + 1); o.y = x;
    rows<TB>(h, l, 1, prec, o, nv, false, EPI_Y, st);
    rc = postsmooth_first<TB>(h, W, prec, l, b, x, r, st);
  }
  h->rec = nullptr;
  if (rc != XAMG_OK) return rc;
  if (!h->rec_ok) return XAMG_ERR_SETUP;
  XCK(cudaMemsetAsync(h->tail_sync, 0, sizeof(TailSync), st));
  int g;
  if constexpr (sizeof(TB) == 8) {
    g = launch_vtail_f64(prog, nv, st);
  } else {
    g = launch_vtail_f32(prog, nv, prec == XAMG_PREC_BF16 ? 1 : 0, st);
  }
  if (g < 0) return XAMG_ERR_CUDA;
  if ((rc = postsmooth_rest<TB>(h, W, prec, l, x, r, st, dots)) != XAMG_OK) return rc;
  return cudaPeekAtLastError() == cudaSuccess ? XAMG_OK : XAMG_ERR_CUDA;
}

// ---- V(1,1) Chebyshev cycle ----
// On entry x holds w0 .* b (the first smoother iterate) unless `level` is the
// coarsest.  TB = double: the FP64 preconditioner; TB = float: the
// reduced-precision one (FP32 blocks, FP32 or bf16 values of A, FP64 coarsest
// solve).  Optional FP64 dots of the final iterate (see Dots).
template <class TB>
int vcycle(xamg_hier *h, Work &W, int prec, int l, const TB *b, TB *x, cudaStream_t st,
           const Dots &dots) {
  using BL = Blocks<TB>;
  const int nv = W.nv;
  const int L = (int)h->lv.size();
  if (l == L - 1) {
    const int nc = h->host.nc;
    if (h->rec) {
      TailProg<TB> *prog = static_cast<TailProg<TB> *>(h->rec);
      if (dots.part || prog->nstages >= kTailMaxStages) {
        h->rec_ok = false;
        return XAMG_OK;
      }
      TailStage<TB> &t = prog->st[prog->nstages++];
      std::memset(&t.op, 0, sizeof(t.op));
      t.op.n = nc;
      t.op.val = h->ainv;
      t.op.src = b;
      t.op.y = x;
      t.kind = TK_COARSE;
      t.wide = 0;
      return XAMG_OK;
    }
    const double *xd;
    if constexpr (sizeof(TB) == 8) {
      launch_coarse(nv, nc, h->ainv, b, x, st);
      xd = x;
    } else {
      launch_coarse_f(nv, nc, h->ainv, b, x, st);
      launch_to_f64(nv, nc, x, W.cw, elem_grid(nc, nv), st);  // the dots read the FP32 result
      xd = W.cw;
    }
    if (dots.part) {
      const int g = elem_grid(nc, nv);
      launch_coldot(nv, nc, dots.u, xd, dots.part, g, st);
      if (dots.part2) launch_coldot(nv, nc, dots.u2, xd, dots.part2, g, st);
      *dots.grid = g;
    }
    return cudaPeekAtLastError() == cudaSuccess ? XAMG_OK : XAMG_ERR_CUDA;
  }
  if (!h->rec && tail_start(h, nv) == l) {
    const int rc = vcycle_tail<TB>(h, W, prec, l, b, x, st, dots);
    if (rc != XAMG_ERR_SETUP) return rc;  // else: the tail does not fit; the plain cycle below
  }
  TB *r = BL::r(W, l);
  int rc = presmooth<TB>(h, W, prec, l, b, x, r, st);
  if (rc != XAMG_OK) return rc;
  // restriction b_c = R r (and the coarse level's first smoother iterate)
  {
    const bool next_coarsest = l + 2 == L;
    RowOpT<TB> o = blank<TB>();
    o.src = r; o.y = BL::b(W, l + 1);
    if (!next_coarsest) {
      o.w = BL::w(h->lv[l + 1], 0);
      o.dnext = BL::x(W, l + 1);
    }
    if (rows<TB>(h, l, 2, prec, o, nv, false, next_coarsest ? EPI_Y : EPI_Y_D0, st) < 0)
      return XAMG_ERR_CUDA;
  }
  rc = vcycle<TB>(h, W, prec, l + 1, BL::b(W, l + 1), BL::x(W, l + 1), st, Dots());
  if (rc != XAMG_OK) return rc;
  // prolongation and correction x += P x_c
  {
    RowOpT<TB> o = blank<TB>();
    o.init = x; o.src = BL::x(W, l + 1); o.y = x;
    if (rows<TB>(h, l, 1, prec, o, nv, false, EPI_Y, st) < 0) return XAMG_ERR_CUDA;
  }
  if ((rc = postsmooth_first<TB>(h, W, prec, l, b, x, r, st)) != XAMG_OK) return rc;
  if ((rc = postsmooth_rest<TB>(h, W, prec, l, x, r, st, dots)) != XAMG_OK) return rc;
  return cudaPeekAtLastError() == cudaSuccess ? XAMG_OK : XAMG_ERR_CUDA;
}

Dots dot1(const double *u, double *part, int *grid) {
  Dots d;
  d.u = u;
  d.part = part;
  d.grid = grid;
  return d;
}

int sync_read(cudaStream_t st) {
  XCK(cudaStreamSynchronize(st));
  return XAMG_OK;
}

// true residual t = b - A x with partial ||t||^2 in part; returns the grid
int true_residual(xamg_hier *h, Work &W, double *T, double *part, cudaStream_t st) {
  RowOp o = blank<double>();
  o.init = W.Bn; o.src = W.X; o.y = T; o.partials2 = part;
  return rows<double>(h, 0, 0, XAMG_PREC_FP64, o, W.nv, true, EPI_Y_DOT2, st);
}

struct SolveCtx {
  xamg_hier *h;
  Work W;
  int m, nv;
  double tol;
  int maxit;
  int prec = XAMG_PREC_FP64;
  cudaStream_t st;
  int iterations = 0, vcycles = 0;
  // set when the loop ended on a confirmation that restarted no column: the
  // true residual norms in the column state are those of the final X
  bool confirmed = false;
  const double *x0 = nullptr;  // user initial guess (n x m), or null for X0 = 0
};

int sync_read(cudaStream_t st);

// The steady part of one PCG iteration: `body(stream)` issues the previous
// iteration's preconditioner, beta and direction update, then this
// iteration's A p, alpha, x/r update and convergence test, with the scalar
// steps reading the iteration number from the device counter.  With graphs
// on (and timing off) the body is captured once per key on a private stream
// and replayed on the solve's stream, one launch for the whole sequence.
template <class F>
int steady(SolveCtx &c, F &&body) {
  xamg_hier *h = c.h;
  if (!h->use_graphs || h->timing) return body(c.st);
  GraphRec *g = nullptr;
  for (auto &r : h->graphs)
    if (r.nv == c.nv && r.prec == c.prec && r.ws == (const void *)c.W.cs && r.tol == c.tol) g = &r;
  if (!g) {
    if (!h->cap_stream) XCK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const int64_t before = g_launches.load();
    XCK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = body(h->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
    const int64_t launched = g_launches.load() - before;
    g_launches -= launched;  // counted per replay below
    if (rc != XAMG_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc != XAMG_OK ? rc : XAMG_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return XAMG_ERR_CUDA;
    if (h->graphs.size() >= 16) {  // bounded cache: drop the oldest
      cudaGraphExecDestroy(h->graphs.front().exec);
      h->graphs.erase(h->graphs.begin());
    }
    GraphRec r;
    r.nv = c.nv;
    r.prec = c.prec;
    r.ws = c.W.cs;
    r.tol = c.tol;
    r.exec = exec;
    r.launches = launched;
    h->graphs.push_back(r);
    g = &h->graphs.back();
  }
  XCK(cudaGraphLaunch(g->exec, c.st));
  g_launches += g->launches;
  return XAMG_OK;
}

// Warm start: columns whose initial residual already meets the tolerance start
// frozen (state 1); the host reads how many stay active.
int initial_check(SolveCtx &c) {
  Work &W = c.W;
  const int64_t n = c.h->lv[0].A.n;
  const int ge = elem_grid(n, c.nv);
  launch_coldot(c.nv, n, W.R, W.R, W.part[3], ge, c.st);
  launch_scalar(c.nv, SM_PCG_CONV, W.cs, W.part[3], nullptr, ge, c.tol, 0, c.h->flags_d, c.st);
  return sync_read(c.st);
}

// Warm start: X = X0 (zero right-hand-side columns stay 0) and R = B - A X.
int load_x0(SolveCtx &c) {
  Work &W = c.W;
  const int64_t n = c.h->lv[0].A.n;
  const int ge = elem_grid(n, c.nv);
  launch_pad_in(c.nv, n, c.x0, c.m, W.X, ge, c.st);
  launch_zero_rhs_cols(c.nv, n, W.X, W.cs, ge, c.st);
  RowOp o = blank<double>();
  o.init = W.Bn; o.src = W.X; o.y = W.R;
  return rows<double>(c.h, 0, 0, XAMG_PREC_FP64, o, c.nv, true, EPI_Y, c.st) < 0 ? XAMG_ERR_CUDA : XAMG_OK;
}

// z = M r for the FP64 Krylov loops.  FP64 preconditioner: on entry z holds
// w0 .* r (written by the kernel that produced r).  Reduced precision: r is
// rounded to the FP32 block, the FP32 V-cycle runs, z is widened back.
int apply_precond(SolveCtx &c, const double *r, double *z) {
  xamg_hier *h = c.h;
  Work &W = c.W;
  c.vcycles++;
  if (c.prec == XAMG_PREC_FP64) return vcycle<double>(h, W, c.prec, 0, r, z, c.st, Dots());
  const int64_t n = h->lv[0].A.n;
  const int ge = elem_grid(n, c.nv);
  const float *w0f = h->lv.size() > 1 ? h->lv[0].w32[0] : nullptr;
  launch_to_f32(c.nv, n, r, W.R32, w0f, W.Z32, ge, c.st);
  const int rc = vcycle<float>(h, W, c.prec, 0, W.R32, W.Z32, c.st, Dots());
  if (rc != XAMG_OK) return rc;
  launch_to_f64(c.nv, n, W.Z32, z, ge, c.st);
  return cudaPeekAtLastError() == cudaSuccess ? XAMG_OK : XAMG_ERR_CUDA;
}

int finish(SolveCtx &c, double *Xuser, xamg_stats *stats) {
  xamg_hier *h = c.h;
  Work &W = c.W;
  const int64_t n = h->lv[0].A.n;
  double *T = W.Q ? W.Q : W.T;
  if (!c.confirmed) {
    const int g = true_residual(h, W, T, W.part[4], c.st);
    if (g < 0) return XAMG_ERR_CUDA;
    launch_scalar(c.nv, SM_FINAL, W.cs, W.part[4], nullptr, g, c.tol, 0, nullptr, c.st);
  }
  launch_copy_out(c.nv, n, W.X, Xuser, c.m, elem_grid(n, c.nv), c.st);
  ColState cs;
  XCK(cudaMemcpyAsync(&cs, W.cs, sizeof(cs), cudaMemcpyDeviceToHost, c.st));
  XCK(cudaStreamSynchronize(c.st));
  XCK(cudaGetLastError());
  if (h->timing) flush_timing(h);
  int rc = XAMG_OK;
  int maxits = 0;
  for (int j = 0; j < c.m; ++j) {
    int status;
    double rel = 0.0;
    if (cs.state[j] == 4) {
      status = XAMG_COL_CONVERGED;
    } else {
      rel = cs.tn[j] / cs.nb[j];
      if (cs.state[j] == 3) status = XAMG_COL_BREAKDOWN;
      else status = rel <= c.tol ? XAMG_COL_CONVERGED : XAMG_COL_NOT_CONVERGED;
    }
    if (status == XAMG_COL_BREAKDOWN) rc = XAMG_BREAKDOWN;
    else if (status == XAMG_COL_NOT_CONVERGED && rc == XAMG_OK) rc = XAMG_NOT_CONVERGED;
    maxits = std::max(maxits, (int)cs.iters[j]);
    if (stats) {
      if (stats->iters) stats->iters[j] = cs.iters[j];
      if (stats->relres) stats->relres[j] = rel;
      if (stats->status) stats->status[j] = status;
    }
  }
  if (stats) {
    stats->iterations = maxits;
    stats->vcycles = c.vcycles;
  }
  return rc;
}

int check_init(SolveCtx &c) {
  int rc = sync_read(c.st);
  if (rc != XAMG_OK) return rc;
  XCK(cudaGetLastError());
  if (c.h->flags_h->breakdown < 0) return XAMG_ERR_NONFINITE;
  return XAMG_OK;
}

int solve_pcg(SolveCtx &c, const double *B, double *Xuser, xamg_stats *stats) {
  xamg_hier *h = c.h;
  Work &W = c.W;
  const int nv = c.nv;
  const int64_t n = h->lv[0].A.n;
  const int ge = elem_grid(n, nv);
  const bool single = h->lv.size() == 1;
  const double *w0 = single ? nullptr : h->lv[0].w[0];
  Flags *fl = h->flags_d;
  cudaStream_t st = c.st;
  int g;
  launch_init_pcg(nv, n, B, c.m, W.Bn, W.R, W.X, W.Z, w0, W.part[0], ge, st);
  launch_scalar(nv, SM_INIT, W.cs, W.part[0], nullptr, ge, c.tol, 0, fl, st);
  int rc = check_init(c);
  if (rc != XAMG_OK) return rc;
  if (c.x0) {
    if ((rc = load_x0(c)) != XAMG_OK) return rc;
    if (w0) launch_scale_rows(nv, n, w0, W.R, W.Z, ge, st);
    if ((rc = initial_check(c)) != XAMG_OK) return rc;
  }
  if (h->flags_h->active > 0) {
    if ((rc = vcycle<double>(h, W, XAMG_PREC_FP64, 0, W.R, W.Z, st, dot1(W.R, W.part[1], &g))) != XAMG_OK)
      return rc;
    c.vcycles++;
    launch_scalar(nv, SM_PCG_BETA, W.cs, W.part[1], nullptr, g, c.tol, 0, fl, st);
    launch_pcg_p(nv, n, W.P, W.Z, W.cs, ge, st);
  }
  // A p (with p.q), alpha, x/r update (with |r|^2), convergence test; kk < 0:
  // the iteration number comes from the device counter
  auto head = [&](cudaStream_t s, int kk) -> int {
    RowOp o = blank<double>();
    o.src = W.P; o.y = W.Q; o.dot_u = W.P; o.partials = W.part[0];
    int gg;
    if ((gg = rows<double>(h, 0, 0, XAMG_PREC_FP64, o, nv, false, EPI_Y_DOT, s)) < 0) return XAMG_ERR_CUDA;
    launch_scalar(nv, SM_PCG_ALPHA, W.cs, W.part[0], nullptr, gg, c.tol, kk, fl, s);
    launch_pcg_xr(nv, n, W.X, W.R, W.P, W.Q, W.cs, w0, W.Z, W.part[1], ge, s);
    launch_scalar(nv, SM_PCG_CONV, W.cs, W.part[1], nullptr, ge, c.tol, kk, fl, s);
    return cudaPeekAtLastError() == cudaSuccess ? XAMG_OK : XAMG_ERR_CUDA;
  };
  // preconditioner with r.z, beta, direction update
  auto tail = [&](cudaStream_t s) -> int {
    int gg;
    const int r = vcycle<double>(h, W, XAMG_PREC_FP64, 0, W.R, W.Z, s, dot1(W.R, W.part[1], &gg));
    if (r != XAMG_OK) return r;
    launch_scalar(nv, SM_PCG_BETA, W.cs, W.part[1], nullptr, gg, c.tol, -1, fl, s);
    launch_pcg_p(nv, n, W.P, W.Z, W.cs, ge, s);
    return cudaPeekAtLastError() == cudaSuccess ? XAMG_OK : XAMG_ERR_CUDA;
  };
  for (int k = 1; k <= c.maxit && h->flags_h->active > 0; ++k) {
    c.iterations = k;
    if (k == 1) {
      rc = head(st, k);
    } else {
      c.vcycles++;
      rc = steady(c, [&](cudaStream_t s) {
        const int r = tail(s);
        return r != XAMG_OK ? r : head(s, -1);
      });
    }
    if (rc != XAMG_OK) return rc;
    if ((rc = sync_read(st)) != XAMG_OK) return rc;
    if (h->flags_h->active == 0) {
      if ((g = true_residual(h, W, W.Q, W.part[2], st)) < 0) return XAMG_ERR_CUDA;
      launch_scalar(nv, SM_CONFIRM, W.cs, W.part[2], nullptr, g, c.tol, k, fl, st);
      if ((rc = sync_read(st)) != XAMG_OK) return rc;
      if (h->flags_h->reactivated == 0) {
        c.confirmed = true;
        break;
      }
      launch_copy_cols(nv, n, W.R, W.Q, W.cs, ge, st);
      if (w0) launch_scale_rows(nv, n, w0, W.R, W.Z, ge, st);
    }
  }
  return finish(c, Xuser, stats);
}

// Flexible PCG in FP64 around the reduced-precision preconditioner: the
// rounding of the FP32 V-cycle makes M slightly non-symmetric, so the
// direction update uses beta = z_new . (r_new - r_old) / (z_old . r_old)
// (r_new - r_old = -alpha q, so only q . z is needed).  FP64 is kept for the
// residual update, the dots and the coarsest solve.
int solve_fpcg(SolveCtx &c, const double *B, double *Xuser, xamg_stats *stats) {
  xamg_hier *h = c.h;
  Work &W = c.W;
  const int nv = c.nv;
  const int64_t n = h->lv[0].A.n;
  const int ge = elem_grid(n, nv);
  const float *w0f = h->lv.size() > 1 ? h->lv[0].w32[0] : nullptr;
  Flags *fl = h->flags_d;
  cudaStream_t st = c.st;
  const int prec = c.prec;
  int g;
  launch_init_fpcg(nv, n, B, c.m, W.Bn, W.R, W.X, W.R32, W.Z32, w0f, W.part[0], ge, st);
  launch_scalar(nv, SM_INIT, W.cs, W.part[0], nullptr, ge, c.tol, 0, fl, st);
  int rc = check_init(c);
  if (rc != XAMG_OK) return rc;
  if (c.x0) {
    if ((rc = load_x0(c)) != XAMG_OK) return rc;
    launch_to_f32(nv, n, W.R, W.R32, w0f, W.Z32, ge, st);
    if ((rc = initial_check(c)) != XAMG_OK) return rc;
  }
  if (h->flags_h->active > 0) {
    if ((rc = vcycle<float>(h, W, prec, 0, W.R32, W.Z32, st, dot1(W.R, W.part[1], &g))) != XAMG_OK)
      return rc;
    c.vcycles++;
    launch_scalar(nv, SM_PCG_BETA, W.cs, W.part[1], nullptr, g, c.tol, 0, fl, st);
    launch_fpcg_p(nv, n, W.P, W.Z32, W.cs, ge, st);
  }
  // A p (with p.q), alpha, x/r update (with |r|^2 and the FP32 copy of r),
  // convergence test; kk < 0: the iteration number comes from the device
  // counter
  auto head = [&](cudaStream_t s, int kk) -> int {
    RowOp o = blank<double>();
    o.src = W.P; o.y = W.Q; o.dot_u = W.P; o.partials = W.part[0];
    int gg;
    if ((gg = rows<double>(h, 0, 0, XAMG_PREC_FP64, o, nv, false, EPI_Y_DOT, s)) < 0) return XAMG_ERR_CUDA;
    launch_scalar(nv, SM_PCG_ALPHA, W.cs, W.part[0], nullptr, gg, c.tol, kk, fl, s);
    launch_fpcg_xr(nv, n, W.X, W.R, W.P, W.Q, W.cs, w0f, W.R32, W.Z32, W.part[1], ge, s);
    launch_scalar(nv, SM_PCG_CONV, W.cs, W.part[1], nullptr, ge, c.tol, kk, fl, s);
    return cudaPeekAtLastError() == cudaSuccess ? XAMG_OK : XAMG_ERR_CUDA;
  };
  // reduced-precision preconditioner with z.r and z.q, flexible beta,
  // direction update
  auto tail = [&](cudaStream_t s) -> int {
    int gg;
    Dots d = dot1(W.R, W.part[1], &gg);
    d.u2 = W.Q;
    d.part2 = W.part[2];
    const int r = vcycle<float>(h, W, prec, 0, W.R32, W.Z32, s, d);
    if (r != XAMG_OK) return r;
    launch_scalar(nv, SM_FPCG_BETA, W.cs, W.part[1], W.part[2], gg, c.tol, -1, fl, s);
    launch_fpcg_p(nv, n, W.P, W.Z32, W.cs, ge, s);
    return cudaPeekAtLastError() == cudaSuccess ? XAMG_OK : XAMG_ERR_CUDA;
  };
  for (int k = 1; k <= c.maxit && h->flags_h->active > 0; ++k) {
    c.iterations = k;
    if (k == 1) {
      rc = head(st, k);
    } else {
      c.vcycles++;
      rc = steady(c, [&](cudaStream_t s) {
        const int r = tail(s);
        return r != XAMG_OK ? r : head(s, -1);
      });
    }
    if (rc != XAMG_OK) return rc;
    if ((rc = sync_read(st)) != XAMG_OK) return rc;
    if (h->flags_h->active == 0) {
      if ((g = true_residual(h, W, W.Q, W.part[2], st)) < 0) return XAMG_ERR_CUDA;
      launch_scalar(nv, SM_CONFIRM, W.cs, W.part[2], nullptr, g, c.tol, k, fl, st);
      if ((rc = sync_read(st)) != XAMG_OK) return rc;
      if (h->flags_h->reactivated == 0) {
        c.confirmed = true;
        break;
      }
      launch_copy_cols(nv, n, W.R, W.Q, W.cs, ge, st);
      launch_to_f32(nv, n, W.R, W.R32, w0f, W.Z32, ge, st);
    }
  }
  return finish(c, Xuser, stats);
}

int solve_bicgstab(SolveCtx &c, const double *B, double *Xuser, xamg_stats *stats) {
  xamg_hier *h = c.h;
  Work &W = c.W;
  const int nv = c.nv;
  const int64_t n = h->lv[0].A.n;
  const int ge = elem_grid(n, nv);
  const bool single = h->lv.size() == 1;
  // the FP64 preconditioner takes its first smoother iterate from the kernels
  // that produce p and s; the reduced-precision one forms it while rounding
  const double *w0 = (single || c.prec != XAMG_PREC_FP64) ? nullptr : h->lv[0].w[0];
  Flags *fl = h->flags_d;
  cudaStream_t st = c.st;
  int g;
  const size_t blk = (size_t)n * nv * sizeof(double);
  XCK(cudaMemsetAsync(W.T, 0, blk, st));
  XCK(cudaMemsetAsync(W.SH, 0, blk, st));
  launch_init_bicg(nv, n, B, c.m, W.Bn, W.R, W.RH, W.X, W.P, W.V, W.part[0], ge, st);
  launch_scalar(nv, SM_INIT, W.cs, W.part[0], nullptr, ge, c.tol, 0, fl, st);
  int rc = check_init(c);
  if (rc != XAMG_OK) return rc;
  if (c.x0) {
    // rhat = r_0 = b - A x_0
    if ((rc = load_x0(c)) != XAMG_OK) return rc;
    XCK(cudaMemcpyAsync(W.RH, W.R, blk, cudaMemcpyDeviceToDevice, st));
    if ((rc = initial_check(c)) != XAMG_OK) return rc;
    launch_coldot(nv, n, W.RH, W.R, W.part[0], ge, st);
  }
  double *prh = W.part[0];  // partial sums of rhat . r
  int grh = ge;
  for (int k = 1; k <= c.maxit && h->flags_h->active > 0; ++k) {
    c.iterations = k;
    launch_scalar(nv, SM_BI_RHO, W.cs, prh, nullptr, grh, c.tol, k, fl, st);
    launch_bicg_p(nv, n, W.P, W.R, W.V, W.cs, w0, W.PH, ge, st);
    if ((rc = apply_precond(c, W.P, W.PH)) != XAMG_OK) return rc;
    RowOp o = blank<double>();
    o.src = W.PH; o.y = W.V; o.dot_u = W.RH; o.partials = W.part[1];
    if ((g = rows<double>(h, 0, 0, XAMG_PREC_FP64, o, nv, false, EPI_Y_DOT, st)) < 0) return XAMG_ERR_CUDA;
    launch_scalar(nv, SM_BI_ALPHA, W.cs, W.part[1], nullptr, g, c.tol, k, fl, st);
    launch_bicg_s(nv, n, W.S, W.R, W.V, W.cs, w0, W.SH, W.part[2], ge, st);
    launch_scalar(nv, SM_BI_HALF, W.cs, W.part[2], nullptr, ge, c.tol, k, fl, st);
    if ((rc = sync_read(st)) != XAMG_OK) return rc;
    if (h->flags_h->active > 0) {
      if ((rc = apply_precond(c, W.S, W.SH)) != XAMG_OK) return rc;
      RowOp t = blank<double>();
      t.src = W.SH; t.y = W.T; t.dot_u = W.S; t.partials = W.part[1];
      t.partials2 = W.part[2];
      if ((g = rows<double>(h, 0, 0, XAMG_PREC_FP64, t, nv, false, EPI_Y_DOT2, st)) < 0) return XAMG_ERR_CUDA;
      launch_scalar(nv, SM_BI_OMEGA, W.cs, W.part[1], W.part[2], g, c.tol, k, fl, st);
    }
    launch_bicg_xr(nv, n, W.X, W.R, W.S, W.T, W.PH, W.SH, W.RH, W.cs, W.part[3], W.part[0], ge, st);
    prh = W.part[0];
    grh = ge;
    launch_scalar(nv, SM_BI_CONV, W.cs, W.part[3], nullptr, ge, c.tol, k, fl, st);
    if ((rc = sync_read(st)) != XAMG_OK) return rc;
    if (h->flags_h->active == 0) {
      if ((g = true_residual(h, W, W.T, W.part[2], st)) < 0) return XAMG_ERR_CUDA;
      launch_scalar(nv, SM_CONFIRM, W.cs, W.part[2], nullptr, g, c.tol, k, fl, st);
      if ((rc = sync_read(st)) != XAMG_OK) return rc;
      if (h->flags_h->reactivated == 0) {
        c.confirmed = true;
        break;
      }
      launch_copy_cols(nv, n, W.R, W.T, W.cs, ge, st);
      launch_copy_cols(nv, n, W.RH, W.T, W.cs, ge, st);
      launch_coldot(nv, n, W.RH, W.R, W.part[0], ge, st);
    }
  }
  return finish(c, Xuser, stats);
}

}  // namespace

namespace xamg {

int hier_view(xamg_hier *h, HierView *v) {
  if (!h || !h->on_device || !v) return XAMG_ERR_INVALID_ARG;
  const int L = (int)h->lv.size();
  if (L > kBatchMaxLevels) return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  const int rc = upload_lowp(h);
  if (rc != XAMG_OK) return rc;
  *v = HierView();
  v->L = L;
  v->nc = h->host.nc;
  v->cheb_steps = h->host.cheb_steps;
  v->device = h->device;
  v->ainv = h->ainv;
  for (int l = 0; l < L; ++l) {
    const DevLevel &D = h->lv[l];
    HierLevelView &o = v->lv[l];
    o.n = D.A.n;
    o.nnzA = D.A.nnz;
    o.Arp = D.A.rowptr;
    o.Aci = D.A.col;
    o.Av = D.a32;
    o.A64 = D.A.val;
    if (l + 1 < L) {
      o.nc = D.R.n;
      o.nnzP = D.P.nnz;
      o.nnzR = D.R.nnz;
      o.Prp = D.P.rowptr;
      o.Pci = D.P.col;
      o.Pv = D.p32;
      o.Rrp = D.R.rowptr;
      o.Rci = D.R.col;
      o.Rv = D.r32;
      for (int k = 0; k < 4; ++k) {
        o.w32[k] = D.w32[k];
        o.c1f[k] = D.c1f[k];
      }
    }
  }
  return XAMG_OK;
}

}  // namespace xamg

namespace {

VParts vparts(const double *p0, int n0, const double *p1 = nullptr, int n1 = 0, const double *p2 = nullptr,
              int n2 = 0, const double *p3 = nullptr, int n3 = 0, const double *p4 = nullptr, int n4 = 0) {
  VParts v;
  v.p[0] = p0; v.nblk[0] = n0;
  v.p[1] = p1; v.nblk[1] = n1;
  v.p[2] = p2; v.nblk[2] = n2;
  v.p[3] = p3; v.nblk[3] = n3;
  v.p[4] = p4; v.nblk[4] = n4;
  return v;
}

// Reordered BiCGStab (Krasnopolsky 2010), right-preconditioned: dot
// products in two groups per iteration, rho and ||r|| of the next iteration
// from recurrences, one host read per iteration (the test between the two
// halves is folded into the omega step: a column whose s meets the tolerance
// takes omega = 0, i.e. x += alpha M p, r = s).
int solve_rbicgstab(SolveCtx &c, const double *B, double *Xuser, xamg_stats *stats) {
  xamg_hier *h = c.h;
  Work &W = c.W;
  const int nv = c.nv;
  const int64_t n = h->lv[0].A.n;
  const int ge = elem_grid(n, nv);
  const bool single = h->lv.size() == 1;
  const double *w0 = (single || c.prec != XAMG_PREC_FP64) ? nullptr : h->lv[0].w[0];
  Flags *fl = h->flags_d;
  cudaStream_t st = c.st;
  const size_t blk = (size_t)n * nv * sizeof(double);
  XCK(cudaMemsetAsync(W.T, 0, blk, st));
  XCK(cudaMemsetAsync(W.SH, 0, blk, st));
  launch_init_bicg(nv, n, B, c.m, W.Bn, W.R, W.RH, W.X, W.P, W.V, W.part[0], ge, st);
  launch_scalar(nv, SM_INIT, W.cs, W.part[0], nullptr, ge, c.tol, 0, fl, st);
  int rc = check_init(c);
  if (rc != XAMG_OK) return rc;
  if (c.x0) {
    if ((rc = load_x0(c)) != XAMG_OK) return rc;
    XCK(cudaMemcpyAsync(W.RH, W.R, blk, cudaMemcpyDeviceToDevice, st));
    if ((rc = initial_check(c)) != XAMG_OK) return rc;
  }
  // rho = rhat . r, the only direct one
  launch_coldot(nv, n, W.RH, W.R, W.part[0], ge, st);
  launch_vscalar(nv, VS_RHO0, W.cs, vparts(W.part[0], ge), c.tol, 0, nullptr, st);
  int g;
  for (int k = 1; k <= c.maxit && h->flags_h->active > 0; ++k) {
    c.iterations = k;
    launch_vscalar(nv, VS_RB_BETA, W.cs, vparts(nullptr, 0), c.tol, k, nullptr, st);
    launch_bicg_p(nv, n, W.P, W.R, W.V, W.cs, w0, W.PH, ge, st);
    if ((rc = apply_precond(c, W.P, W.PH)) != XAMG_OK) return rc;
    RowOp o = blank<double>();
    o.src = W.PH; o.y = W.V; o.dot_u = W.RH; o.partials = W.part[0];
    if ((g = rows<double>(h, 0, 0, XAMG_PREC_FP64, o, nv, false, EPI_Y_DOT, st)) < 0) return XAMG_ERR_CUDA;
    launch_scalar(nv, SM_BI_ALPHA, W.cs, W.part[0], nullptr, g, c.tol, k, nullptr, st);
    launch_rb_s(nv, n, W.S, W.R, W.V, W.RH, W.cs, w0, W.SH, W.part[1], W.part[2], ge, st);
    if ((rc = apply_precond(c, W.S, W.SH)) != XAMG_OK) return rc;
    RowOp t = blank<double>();
    t.src = W.SH; t.y = W.T; t.dot_u = W.S; t.partials = W.part[3]; t.partials2 = W.part[4];
    if ((g = rows<double>(h, 0, 0, XAMG_PREC_FP64, t, nv, false, EPI_Y_DOT2, st)) < 0) return XAMG_ERR_CUDA;
    launch_vscalar(nv, VS_RB_OMEGA, W.cs, vparts(W.part[3], g, W.part[4], g, W.part[1], ge), c.tol, k, fl, st);
    launch_rb_xr(nv, n, W.X, W.R, W.S, W.T, W.PH, W.SH, W.RH, W.cs, W.part[0], ge, st);
    launch_vscalar(nv, VS_RB_RHO, W.cs, vparts(W.part[2], ge, W.part[0], ge), c.tol, k, nullptr, st);
    if ((rc = sync_read(st)) != XAMG_OK) return rc;
    if (h->flags_h->active == 0) {
      if ((g = true_residual(h, W, W.T, W.part[2], st)) < 0) return XAMG_ERR_CUDA;
      launch_scalar(nv, SM_CONFIRM, W.cs, W.part[2], nullptr, g, c.tol, k, fl, st);
      if ((rc = sync_read(st)) != XAMG_OK) return rc;
      if (h->flags_h->reactivated == 0) {
        c.confirmed = true;
        break;
      }
      // restarted columns: r = rhat = the true residual, rho = |r|^2
      launch_copy_cols(nv, n, W.R, W.T, W.cs, ge, st);
      launch_copy_cols(nv, n, W.RH, W.T, W.cs, ge, st);
      launch_coldot(nv, n, W.RH, W.R, W.part[0], ge, st);
      launch_vscalar(nv, VS_RHO0, W.cs, vparts(W.part[0], ge), c.tol, k, nullptr, st);
    }
  }
  return finish(c, Xuser, stats);
}

// out = A (M u) for the FP64 preconditioner; tmp receives M u.
int apply_B(SolveCtx &c, const double *u, double *tmp, double *out) {
  xamg_hier *h = c.h;
  const int64_t n = h->lv[0].A.n;
  if (h->lv.size() > 1) launch_scale_rows(c.nv, n, h->lv[0].w[0], u, tmp, elem_grid(n, c.nv), c.st);
  int rc = apply_precond(c, u, tmp);
  if (rc != XAMG_OK) return rc;
  RowOp o = blank<double>();
  o.src = tmp; o.y = out;
  return rows<double>(h, 0, 0, XAMG_PREC_FP64, o, c.nv, false, EPI_Y, c.st) < 0 ? XAMG_ERR_CUDA : XAMG_OK;
}

// Pipelined BiCGStab (Cools and Vanroose 2017) for B = A M.  Blocks: R, RH,
// W (in PH), T, P, S, Z, Q, Y, V, U (the correction in the preconditioned
// variable), X0; SH is the scratch that receives M applications.
int solve_pbicgstab(SolveCtx &c, const double *B, double *Xuser, xamg_stats *stats) {
  xamg_hier *h = c.h;
  Work &W = c.W;
  const int nv = c.nv;
  const int64_t n = h->lv[0].A.n;
  const int ge = elem_grid(n, nv);
  Flags *fl = h->flags_d;
  cudaStream_t st = c.st;
  const size_t blk = (size_t)n * nv * sizeof(double);
  double *Wv = W.PH, *TMP = W.SH, *Z = W.E[0], *Q = W.E[1], *Y = W.E[2], *U = W.E[3], *X0 = W.E[4];
  launch_init_bicg(nv, n, B, c.m, W.Bn, W.R, W.RH, W.X, W.P, W.V, W.part[0], ge, st);
  launch_scalar(nv, SM_INIT, W.cs, W.part[0], nullptr, ge, c.tol, 0, fl, st);
  int rc = check_init(c);
  if (rc != XAMG_OK) return rc;
  if (c.x0) {
    if ((rc = load_x0(c)) != XAMG_OK) return rc;
    XCK(cudaMemcpyAsync(W.RH, W.R, blk, cudaMemcpyDeviceToDevice, st));
    if ((rc = initial_check(c)) != XAMG_OK) return rc;
  }
  XCK(cudaMemcpyAsync(X0, W.X, blk, cudaMemcpyDeviceToDevice, st));
  XCK(cudaMemsetAsync(U, 0, blk, st));
  XCK(cudaMemsetAsync(Z, 0, blk, st));
  // (re)start of the fresh columns: w = B r, t = B w, rho = rhat.r, alpha = rho / rhat.w
  auto start = [&](int k) -> int {
    int r;
    if ((r = apply_B(c, W.R, TMP, Wv)) != XAMG_OK) return r;
    if ((r = apply_B(c, Wv, TMP, W.T)) != XAMG_OK) return r;
    launch_coldot(nv, n, W.RH, W.R, W.part[0], ge, st);
    launch_coldot(nv, n, W.RH, Wv, W.part[1], ge, st);
    launch_vscalar(nv, VS_PB_INIT, W.cs, vparts(W.part[0], ge, W.part[1], ge), c.tol, k, nullptr, st);
    return XAMG_OK;
  };
  // x = x0 + M u
  auto form_x = [&]() -> int {
    if (h->lv.size() > 1) launch_scale_rows(nv, n, h->lv[0].w[0], U, TMP, ge, st);
    const int r = apply_precond(c, U, TMP);
    if (r != XAMG_OK) return r;
    launch_pb_form_x(nv, n, W.X, X0, TMP, ge, st);
    return XAMG_OK;
  };
  if (h->flags_h->active > 0 && (rc = start(0)) != XAMG_OK) return rc;
  double *const parts[5] = {W.part[0], W.part[1], W.part[2], W.part[3], W.part[4]};
  bool formed = true;  // X holds x0 + M u
  for (int k = 1; k <= c.maxit && h->flags_h->active > 0; ++k) {
    c.iterations = k;
    formed = false;
    launch_pb_psz(nv, n, W.P, W.S, Z, W.R, Wv, W.T, W.V, W.cs, ge, st);
    launch_pb_qy(nv, n, Q, Y, W.R, W.S, Wv, Z, W.cs, W.part[0], W.part[1], ge, st);
    if ((rc = apply_B(c, Z, TMP, W.V)) != XAMG_OK) return rc;
    launch_vscalar(nv, VS_PB_OMEGA, W.cs, vparts(W.part[0], ge, W.part[1], ge), c.tol, k, nullptr, st);
    launch_pb_urw(nv, n, U, W.R, Wv, W.P, Q, Y, W.T, W.V, W.S, Z, W.RH, W.cs, parts, ge, st);
    if ((rc = apply_B(c, Wv, TMP, W.T)) != XAMG_OK) return rc;
    launch_vscalar(nv, VS_PB_ALPHA, W.cs,
                   vparts(W.part[0], ge, W.part[1], ge, W.part[2], ge, W.part[3], ge, W.part[4], ge), c.tol, k,
                   fl, st);
    if ((rc = sync_read(st)) != XAMG_OK) return rc;
    if (h->flags_h->active == 0) {
      if ((rc = form_x()) != XAMG_OK) return rc;
      formed = true;
      int g;
      if ((g = true_residual(h, W, TMP, W.part[2], st)) < 0) return XAMG_ERR_CUDA;
      launch_scalar(nv, SM_CONFIRM, W.cs, W.part[2], nullptr, g, c.tol, k, fl, st);
      if ((rc = sync_read(st)) != XAMG_OK) return rc;
      if (h->flags_h->reactivated == 0) {
        c.confirmed = true;
        break;
      }
      launch_copy_cols(nv, n, W.R, TMP, W.cs, ge, st);
      launch_pb_restart(nv, n, W.X, X0, U, W.RH, W.R, W.cs, ge, st);
      if ((rc = start(k)) != XAMG_OK) return rc;
    }
  }
  if (!formed && (rc = form_x()) != XAMG_OK) return rc;
  return finish(c, Xuser, stats);
}

int solve_impl(xamg_hier *h, const double *B, double *X, int m, double tol, int maxit,
               const xamg_solve_opts *opts, xamg_stats *stats) {
  if (!h || !h->on_device || !B || !X || m < 1 || m > XAMG_MAX_RHS || !(tol > 0.0) || maxit < 0)
    return XAMG_ERR_INVALID_ARG;
  xamg_solve_opts o;
  xamg_solve_opts_default(&o);
  if (opts) o = *opts;
  if (o.method != XAMG_PCG && o.method != XAMG_BICGSTAB && o.method != XAMG_BICGSTAB_REORDERED &&
      o.method != XAMG_BICGSTAB_PIPELINED)
    return XAMG_ERR_INVALID_ARG;
  if (o.method == XAMG_BICGSTAB_PIPELINED && o.precond != XAMG_PREC_FP64) return XAMG_ERR_INVALID_ARG;
  if (o.precond != XAMG_PREC_FP64 && o.precond != XAMG_PREC_FP32 && o.precond != XAMG_PREC_BF16)
    return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  SolveCtx c;
  c.h = h;
  c.m = m;
  c.nv = pad_nv(m);
  c.tol = tol;
  c.maxit = maxit;
  c.prec = o.precond;
  c.st = (cudaStream_t)o.stream;
  if (o.x0_given) c.x0 = X;
  int rc = ensure_workspace(h, c.nv, o.method, c.prec, &o, c.W);
  if (rc != XAMG_OK) return rc;
  h->flags_h->active = 0;
  h->flags_h->tail_err = 0;
  if (o.method == XAMG_PCG)
    rc = c.prec == XAMG_PREC_FP64 ? solve_pcg(c, B, X, stats) : solve_fpcg(c, B, X, stats);
  else if (o.method == XAMG_BICGSTAB_REORDERED)
    rc = solve_rbicgstab(c, B, X, stats);
  else if (o.method == XAMG_BICGSTAB_PIPELINED)
    rc = solve_pbicgstab(c, B, X, stats);
  else
    rc = solve_bicgstab(c, B, X, stats);
  if (h->timing && rc < 0) {
    cudaStreamSynchronize(c.st);
    flush_timing(h);
  }
  if (h->flags_h->tail_err) {  // a grid-barrier wait of the fused tail ran out
    cudaStreamSynchronize(c.st);
    h->flags_h->tail_err = 0;
    return XAMG_ERR_TIMEOUT;
  }
  return rc;
}

}  // namespace

// ===================================================================== C ABI
namespace {

// Times y = M x for operator `which` of level l under both row splits and
// keeps the faster in `slot`.
template <class TB>
int tune_product(xamg_hier *h, int l, int which, int precond, RowOpT<TB> o, int nv, signed char &slot,
                 cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int *wide) {
  float best = 1e30f;
  int best_opt = 0;
  for (int opt = 0; opt < split_candidates(nv, sizeof(TB) == 4); ++opt) {
    slot = (signed char)opt;
    if (rows<TB>(h, l, which, precond, o, nv, false, EPI_Y, st) < 0) return XAMG_ERR_CUDA;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) rows<TB>(h, l, which, precond, o, nv, false, EPI_Y, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return XAMG_ERR_CUDA;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_opt = opt;
    }
  }
  slot = (signed char)best_opt;
  *wide += best_opt != 0;
  return XAMG_OK;
}

}  // namespace

extern "C" {

const char *xamg_strerror(int code) {
  switch (code) {
    case XAMG_OK: return "success";
    case XAMG_ERR_INVALID_ARG: return "invalid argument";
    case XAMG_ERR_CUDA: return "CUDA runtime error";
    case XAMG_ERR_OOM: return "out of memory";
    case XAMG_ERR_NONFINITE: return "non-finite value in the input";
    case XAMG_ERR_TIMEOUT: return "bounded device wait timed out";
    case XAMG_ERR_SETUP: return "hierarchy setup failed";
    case XAMG_NOT_CONVERGED: return "some columns did not converge";
    case XAMG_BREAKDOWN: return "some columns broke down";
    default: return "unknown status";
  }
}

void xamg_amg_params_default(xamg_amg_params *p) {
  if (!p) return;
  p->theta = 0.25;
  p->max_coarse = 64;
  p->max_levels = 25;
  p->cheb_steps = 2;
  p->power_iters = 20;
  p->cheb_lo_frac = 0.3;
  p->cheb_hi_safety = 1.1;
  p->max_dense = 1024;
  p->nthreads = 0;
  p->device_upload = 1;
}

void xamg_solve_opts_default(xamg_solve_opts *o) {
  if (!o) return;
  o->method = XAMG_PCG;
  o->precond = XAMG_PREC_FP64;
  o->x0_given = 0;
  o->stream = nullptr;
  o->workspace = nullptr;
  o->workspace_bytes = 0;
}

static int attach_device(xamg_hier *h, xamg_hier **out);

int xamg_setup_hierarchy(const xamg_csr *A, const xamg_amg_params *p, xamg_hier **out) {
  if (!A || !out) return XAMG_ERR_INVALID_ARG;
  *out = nullptr;
  xamg_amg_params prm;
  xamg_amg_params_default(&prm);
  if (p) prm = *p;
  xamg_hier *h = new (std::nothrow) xamg_hier();
  if (!h) return XAMG_ERR_OOM;
  h->prm = prm;
  int rc = build_hierarchy(*A, prm, h->host);
  if (rc != XAMG_OK) {
    delete h;
    return rc;
  }
  return attach_device(h, out);
}

int xamg_hier_save(const xamg_hier *h, void *blob, size_t capacity, size_t *bytes) {
  if (!h || !bytes) return XAMG_ERR_INVALID_ARG;
  const std::vector<char> b = save_hier(h->prm, h->host);
  *bytes = b.size();
  if (!blob) return XAMG_OK;
  if (capacity < b.size()) return XAMG_ERR_INVALID_ARG;
  std::memcpy(blob, b.data(), b.size());
  return XAMG_OK;
}

int xamg_hier_load(const void *blob, size_t bytes, xamg_hier **out) {
  if (!blob || !out) return XAMG_ERR_INVALID_ARG;
  *out = nullptr;
  xamg_hier *h = new (std::nothrow) xamg_hier();
  if (!h) return XAMG_ERR_OOM;
  const int rc = load_hier(blob, bytes, h->prm, h->host);
  if (rc != XAMG_OK) {
    delete h;
    return rc;
  }
  return attach_device(h, out);
}

// Uploads a built (or loaded) host hierarchy when its parameters ask for it
// and hands it out; on failure frees it.
static int attach_device(xamg_hier *h, xamg_hier **out) {
  int rc = XAMG_OK;
  const xamg_amg_params &prm = h->prm;
  if (prm.device_upload) {
    if (cudaGetDevice(&h->device) != cudaSuccess) {
      delete h;
      return XAMG_ERR_CUDA;
    }
    const int L = (int)h->host.lv.size();
    h->lv.resize(L);
    for (int l = 0; l < L && rc == XAMG_OK; ++l) rc = upload_level(h, l);
    if (rc == XAMG_OK) {
      // the coarsest solve runs as a dense product with the explicit inverse
      // (its columns: the LU solves of the unit vectors)
      const std::vector<double> inv = lu_inverse(h->host.nc, h->host.lu, h->host.piv);
      rc = dev_upload(h, &h->ainv, inv.data(), inv.size());
    }
    if (rc == XAMG_OK) {
      if (cudaHostAlloc((void **)&h->flags_h, sizeof(Flags), cudaHostAllocMapped) != cudaSuccess ||
          cudaHostGetDevicePointer((void **)&h->flags_d, h->flags_h, 0) != cudaSuccess)
        rc = XAMG_ERR_CUDA;
      else
        std::memset(h->flags_h, 0, sizeof(Flags));
    }
    if (rc != XAMG_OK) {
      free_device(h);
      delete h;
      return rc;
    }
    h->tacc.assign((size_t)L * 6, TimeAcc());
    h->on_device = true;
  }
  *out = h;
  return XAMG_OK;
}

int xamg_destroy(xamg_hier *h) {
  if (!h) return XAMG_OK;
  if (h->on_device) {
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_device(h);
  }
  delete h;
  return XAMG_OK;
}

int xamg_hier_info(const xamg_hier *h, int32_t *levels, double *op_complexity) {
  if (!h) return XAMG_ERR_INVALID_ARG;
  if (levels) *levels = (int32_t)h->host.lv.size();
  if (op_complexity) {
    double s = 0;
    for (auto &L : h->host.lv) s += (double)L.A.nnz();
    *op_complexity = s / (double)h->host.lv[0].A.nnz();
  }
  return XAMG_OK;
}

int xamg_level_info(const xamg_hier *h, int32_t level, int32_t *n, int64_t *nnz_a, int64_t *nnz_p) {
  if (!h || level < 0 || level >= (int)h->host.lv.size()) return XAMG_ERR_INVALID_ARG;
  const HostLevel &L = h->host.lv[level];
  if (n) *n = L.A.n;
  if (nnz_a) *nnz_a = L.A.nnz();
  if (nnz_p) *nnz_p = L.P.nnz();
  return XAMG_OK;
}

int xamg_level_export(const xamg_hier *h, int32_t level, int32_t *rowptr, int32_t *col, double *val,
                      int32_t *p_rowptr, int32_t *p_col, double *p_val, int32_t *cf, double *cheb) {
  if (!h || level < 0 || level >= (int)h->host.lv.size()) return XAMG_ERR_INVALID_ARG;
  const HostLevel &L = h->host.lv[level];
  if (rowptr) std::memcpy(rowptr, L.A.rowptr.data(), L.A.rowptr.size() * sizeof(int32_t));
  if (col) std::memcpy(col, L.A.col.data(), L.A.col.size() * sizeof(int32_t));
  if (val) std::memcpy(val, L.A.val.data(), L.A.val.size() * sizeof(double));
  if (!L.P.rowptr.empty()) {
    if (p_rowptr) std::memcpy(p_rowptr, L.P.rowptr.data(), L.P.rowptr.size() * sizeof(int32_t));
    if (p_col) std::memcpy(p_col, L.P.col.data(), L.P.col.size() * sizeof(int32_t));
    if (p_val) std::memcpy(p_val, L.P.val.data(), L.P.val.size() * sizeof(double));
  }
  if (cf && !L.cf.empty()) std::memcpy(cf, L.cf.data(), L.cf.size() * sizeof(int32_t));
  if (cheb) {
    cheb[0] = L.lo;
    cheb[1] = L.hi;
    cheb[2] = L.lam;
    cheb[3] = L.gersh;
  }
  return XAMG_OK;
}

int xamg_coarse_export(const xamg_hier *h, int32_t *nc, double *lu, int32_t *piv) {
  if (!h) return XAMG_ERR_INVALID_ARG;
  if (nc) *nc = h->host.nc;
  if (lu) std::memcpy(lu, h->host.lu.data(), h->host.lu.size() * sizeof(double));
  if (piv) std::memcpy(piv, h->host.piv.data(), h->host.piv.size() * sizeof(int32_t));
  return XAMG_OK;
}

int xamg_workspace_bytes(const xamg_hier *h, int32_t m, int32_t method, int32_t precond,
                         size_t *bytes) {
  if (!h || !bytes || m < 1 || m > XAMG_MAX_RHS || (method < XAMG_PCG || method > XAMG_BICGSTAB_PIPELINED) ||
      precond < XAMG_PREC_FP64 || precond > XAMG_PREC_BF16)
    return XAMG_ERR_INVALID_ARG;
  *bytes = plan(h, pad_nv(m), method, precond, nullptr, nullptr);
  return XAMG_OK;
}

int xamg_solve(xamg_hier *h, const double *B, double *X, int32_t m, double tol, int32_t maxit,
               const xamg_solve_opts *opts, xamg_stats *stats) {
  return solve_impl(h, B, X, m, tol, maxit, opts, stats);
}

// The device address of host memory that the GPU can reach directly
// (page-locked memory registered with CUDA), else nullptr.
static const void *device_view(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the query's error
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int xamg_solve_host(xamg_hier *h, const double *B, double *X, int32_t m, double tol, int32_t maxit,
                    const xamg_solve_opts *opts, xamg_stats *stats) {
  if (!h || !h->on_device || !B || !X || m < 1 || m > XAMG_MAX_RHS) return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  // page-locked buffers: the solve's first pass reads B, and its last pass
  // writes X, over the host link, with no staging copies (the solve reads B
  // once and writes X once; it synchronizes the stream before returning)
  const double *dB = static_cast<const double *>(device_view(B));
  double *dX = static_cast<double *>(const_cast<void *>(device_view(X)));
  if (dB && dX) return solve_impl(h, dB, dX, m, tol, maxit, opts, stats);
  const size_t bytes = (size_t)h->host.lv[0].A.n * m * sizeof(double);
  if (h->hb_bytes < 2 * align256(bytes)) {
    if (h->hb) cudaFree(h->hb);
    h->hb = nullptr;
    h->hb_bytes = 0;
    XCK(cudaMalloc((void **)&h->hb, 2 * align256(bytes)));
    h->hb_bytes = 2 * align256(bytes);
  }
  double *db = h->hb, *dx = (double *)((char *)h->hb + align256(bytes));
  cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
  XCK(cudaMemcpyAsync(db, B, bytes, cudaMemcpyHostToDevice, st));
  if (opts && opts->x0_given) XCK(cudaMemcpyAsync(dx, X, bytes, cudaMemcpyHostToDevice, st));
  int rc = solve_impl(h, db, dx, m, tol, maxit, opts, stats);
  if (rc < 0) return rc;
  XCK(cudaMemcpyAsync(X, dx, bytes, cudaMemcpyDeviceToHost, st));
  XCK(cudaStreamSynchronize(st));
  return rc;
}

int xamg_level_spmm(xamg_hier *h, int32_t level, int32_t which, const double *X, double *Y,
                    int32_t m, void *stream) {
  if (!h || !h->on_device || !X || !Y || m < 1 || m > XAMG_MAX_RHS || level < 0 ||
      level >= (int)h->lv.size() || which < 0 || which > 2)
    return XAMG_ERR_INVALID_ARG;
  if (which > 0 && level + 1 >= (int)h->lv.size()) return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  DevLevel &D = h->lv[level];
  const DevCsr &M = which == 0 ? D.A : which == 1 ? D.P : D.R;
  cudaStream_t st = (cudaStream_t)stream;
  const int nv = pad_nv(m);
  const double *src = X;
  double *dst = Y;
  Work W;
  if (nv != m) {
    int rc = ensure_workspace(h, nv, XAMG_PCG, XAMG_PREC_FP64, nullptr, W);
    if (rc != XAMG_OK) return rc;
    src = W.Bn;
    dst = W.X;
    launch_pad_in(nv, M.ncols, X, m, W.Bn, elem_grid(M.ncols, nv), st);
  }
  RowOp o = blank<double>();
  o.src = src;
  o.y = dst;
  if (rows<double>(h, level, which, XAMG_PREC_FP64, o, nv, false, EPI_Y, st) < 0) return XAMG_ERR_CUDA;
  if (nv != m) launch_copy_out(nv, M.n, W.X, Y, m, elem_grid(M.n, nv), st);
  XCK(cudaStreamSynchronize(st));
  XCK(cudaGetLastError());
  if (h->timing) flush_timing(h);
  return XAMG_OK;
}

int xamg_level_spmm_precond(xamg_hier *h, int32_t precond, int32_t level, int32_t which, const double *X,
                            double *Y, int32_t m, void *stream) {
  if (!h || !h->on_device || !X || !Y || m < 1 || m > XAMG_MAX_RHS || level < 0 ||
      level >= (int)h->lv.size() || which < 0 || which > 2)
    return XAMG_ERR_INVALID_ARG;
  if (which > 0 && level + 1 >= (int)h->lv.size()) return XAMG_ERR_INVALID_ARG;
  if (precond != XAMG_PREC_FP32 && precond != XAMG_PREC_BF16) return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int nv = pad_nv(m);
  Work W;
  // the level-0 FP32 blocks of the workspace hold the operand and the result
  // (every level's operators have at most n_0 rows and columns)
  int rc = ensure_workspace(h, nv, XAMG_PCG, precond, nullptr, W);
  if (rc != XAMG_OK) return rc;
  DevLevel &D = h->lv[level];
  const DevCsr &M = which == 0 ? D.A : which == 1 ? D.P : D.R;
  launch_pad_in(nv, M.ncols, X, m, W.Bn, elem_grid(M.ncols, nv), st);
  launch_to_f32(nv, M.ncols, W.Bn, W.R32, nullptr, nullptr, elem_grid(M.ncols, nv), st);
  RowOpF o = blank<float>();
  o.src = W.R32;
  o.y = W.Z32;
  if (rows<float>(h, level, which, precond, o, nv, false, EPI_Y, st) < 0) return XAMG_ERR_CUDA;
  launch_to_f64(nv, M.n, W.Z32, W.X, elem_grid(M.n, nv), st);
  launch_copy_out(nv, M.n, W.X, Y, m, elem_grid(M.n, nv), st);
  XCK(cudaStreamSynchronize(st));
  XCK(cudaGetLastError());
  if (h->timing) flush_timing(h);
  return XAMG_OK;
}

int xamg_set_tail(xamg_hier *h, int64_t max_elems, double wait_limit_s, int32_t extra_arrivals) {
  if (!h || max_elems < 0 || !(wait_limit_s > 0.0) || wait_limit_s > 60.0 || extra_arrivals < 0)
    return XAMG_ERR_INVALID_ARG;
  clear_graphs(h);  // the captured tail launches hold the old settings
  h->tail_elems = max_elems;
  h->tail_limit_s = wait_limit_s;
  h->tail_extra = extra_arrivals;
  return XAMG_OK;
}

int xamg_tail_info(const xamg_hier *h, int32_t m, int32_t *first_level) {
  if (!h || !h->on_device || !first_level || m < 1 || m > XAMG_MAX_RHS) return XAMG_ERR_INVALID_ARG;
  *first_level = tail_start(h, pad_nv(m));
  return XAMG_OK;
}

int xamg_set_index16(xamg_hier *h, int32_t enable) {
  if (!h) return XAMG_ERR_INVALID_ARG;
  if (h->use_idx16 != (enable != 0)) clear_graphs(h);
  h->use_idx16 = enable != 0;
  return XAMG_OK;
}

int xamg_index16_info(xamg_hier *h, int32_t level, int32_t *mask) {
  if (!h || !h->on_device || !mask || level < 0 || level >= (int)h->lv.size()) return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  int rc = upload_lowp(h);
  if (rc != XAMG_OK) return rc;
  const DevLevel &D = h->lv[level];
  *mask = (D.w16[0] ? 1 : 0) | (D.w16[1] ? 2 : 0) | (D.w16[2] ? 4 : 0);
  return XAMG_OK;
}

int xamg_smooth(xamg_hier *h, int32_t level, const double *B, double *X, double *R, int32_t x_zero,
                int32_t m, void *stream) {
  if (!h || !h->on_device || !B || !X || m < 1 || m > XAMG_MAX_RHS || level < 0 ||
      level + 1 >= (int)h->lv.size() || (!x_zero && R))
    return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int nv = pad_nv(m);
  Work W;
  int rc = ensure_workspace(h, nv, XAMG_PCG, XAMG_PREC_FP64, nullptr, W);
  if (rc != XAMG_OK) return rc;
  DevLevel &D = h->lv[level];
  const int64_t n = D.A.n;
  const int ge = elem_grid(n, nv);
  // padded copies of B and X in Bn / X, residual in vr, directions in vd/vd2
  launch_pad_in(nv, n, B, m, W.Bn, ge, st);
  double *x = W.X, *r = W.vr[level];
  if (x_zero) {
    launch_scale_rows(nv, n, D.w[0], W.Bn, x, ge, st);
    if ((rc = presmooth<double>(h, W, XAMG_PREC_FP64, level, W.Bn, x, r, st)) != XAMG_OK) return rc;
    if (R) launch_copy_out(nv, n, r, R, m, ge, st);
  } else {
    launch_pad_in(nv, n, X, m, x, ge, st);
    if ((rc = postsmooth_first<double>(h, W, XAMG_PREC_FP64, level, W.Bn, x, r, st)) != XAMG_OK ||
        (rc = postsmooth_rest<double>(h, W, XAMG_PREC_FP64, level, x, r, st, Dots())) != XAMG_OK)
      return rc;
  }
  launch_copy_out(nv, n, x, X, m, ge, st);
  XCK(cudaStreamSynchronize(st));
  XCK(cudaGetLastError());
  if (h->timing) flush_timing(h);
  return XAMG_OK;
}

int xamg_vcycle(xamg_hier *h, const double *B, double *X, int32_t m, void *stream) {
  if (!h || !h->on_device || !B || !X || m < 1 || m > XAMG_MAX_RHS) return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  h->flags_h->tail_err = 0;
  cudaStream_t st = (cudaStream_t)stream;
  const int nv = pad_nv(m);
  Work W;
  int rc = ensure_workspace(h, nv, XAMG_PCG, XAMG_PREC_FP64, nullptr, W);
  if (rc != XAMG_OK) return rc;
  const int64_t n = h->lv[0].A.n;
  const int ge = elem_grid(n, nv);
  launch_pad_in(nv, n, B, m, W.Bn, ge, st);
  if (h->lv.size() > 1) launch_scale_rows(nv, n, h->lv[0].w[0], W.Bn, W.X, ge, st);
  if ((rc = vcycle<double>(h, W, XAMG_PREC_FP64, 0, W.Bn, W.X, st, Dots())) != XAMG_OK) return rc;
  launch_copy_out(nv, n, W.X, X, m, ge, st);
  XCK(cudaStreamSynchronize(st));
  XCK(cudaGetLastError());
  if (h->flags_h->tail_err) {  // a grid-barrier wait of the fused tail ran out
    h->flags_h->tail_err = 0;
    return XAMG_ERR_TIMEOUT;
  }
  if (h->timing) flush_timing(h);
  return XAMG_OK;
}

int xamg_vcycle_precond(xamg_hier *h, int32_t precond, const double *B, double *X, int32_t m,
                        void *stream) {
  if (!h || !h->on_device || !B || !X || m < 1 || m > XAMG_MAX_RHS) return XAMG_ERR_INVALID_ARG;
  if (precond == XAMG_PREC_FP64) return xamg_vcycle(h, B, X, m, stream);
  if (precond != XAMG_PREC_FP32 && precond != XAMG_PREC_BF16) return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  h->flags_h->tail_err = 0;
  cudaStream_t st = (cudaStream_t)stream;
  const int nv = pad_nv(m);
  Work W;
  int rc = ensure_workspace(h, nv, XAMG_PCG, precond, nullptr, W);
  if (rc != XAMG_OK) return rc;
  const int64_t n = h->lv[0].A.n;
  const int ge = elem_grid(n, nv);
  launch_pad_in(nv, n, B, m, W.Bn, ge, st);
  launch_to_f32(nv, n, W.Bn, W.R32, h->lv.size() > 1 ? h->lv[0].w32[0] : nullptr, W.Z32, ge, st);
  if ((rc = vcycle<float>(h, W, precond, 0, W.R32, W.Z32, st, Dots())) != XAMG_OK) return rc;
  launch_to_f64(nv, n, W.Z32, W.X, ge, st);
  launch_copy_out(nv, n, W.X, X, m, ge, st);
  XCK(cudaStreamSynchronize(st));
  XCK(cudaGetLastError());
  if (h->flags_h->tail_err) {  // a grid-barrier wait of the fused tail ran out
    h->flags_h->tail_err = 0;
    return XAMG_ERR_TIMEOUT;
  }
  if (h->timing) flush_timing(h);
  return XAMG_OK;
}

int xamg_coarse_solve(xamg_hier *h, const double *B, double *X, int32_t m, void *stream) {
  if (!h || !h->on_device || !B || !X || m < 1 || m > XAMG_MAX_RHS) return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int nv = pad_nv(m);
  Work W;
  int rc = ensure_workspace(h, nv, XAMG_PCG, XAMG_PREC_FP64, nullptr, W);
  if (rc != XAMG_OK) return rc;
  const int nc = h->host.nc;
  const int ge = elem_grid(nc, nv);
  launch_pad_in(nv, nc, B, m, W.Bn, ge, st);
  launch_coarse(nv, nc, h->ainv, W.Bn, W.X, st);
  launch_copy_out(nv, nc, W.X, X, m, ge, st);
  XCK(cudaStreamSynchronize(st));
  XCK(cudaGetLastError());
  return XAMG_OK;
}

int xamg_coldot(const double *U, const double *V, int64_t n, int32_t m, double *out, void *stream) {
  if (!U || !V || !out || n < 0 || m < 1 || m > XAMG_MAX_RHS) return XAMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = coldot_rt_grid(n, m);
  double *part = nullptr;
  XCK(cudaMallocAsync((void **)&part, (size_t)grid * m * sizeof(double), st));
  launch_coldot_rt(n, m, U, V, part, grid, st);
  launch_reduce_rt(m, part, grid, out, st);
  cudaError_t e1 = cudaGetLastError();
  cudaError_t e2 = cudaFreeAsync(part, st);
  cudaError_t e3 = cudaStreamSynchronize(st);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return XAMG_ERR_CUDA;
  return XAMG_OK;
}

int xamg_autotune(xamg_hier *h, int32_t m, int32_t precond, void *stream, int32_t *ops_tuned,
                  int32_t *ops_wide) {
  if (!h || !h->on_device || m < 1 || m > XAMG_MAX_RHS ||
      (precond != XAMG_PREC_FP64 && precond != XAMG_PREC_FP32 && precond != XAMG_PREC_BF16))
    return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  const int nv = pad_nv(m);
  Work W;
  int rc = ensure_workspace(h, nv, XAMG_PCG, precond, nullptr, W);
  if (rc != XAMG_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int lg = 0;
  while ((1 << lg) < nv) ++lg;
  const int pc = precond == XAMG_PREC_BF16 ? 1 : precond == XAMG_PREC_FP32 ? 0 : 2;
  const bool timing = h->timing;
  h->timing = false;
  clear_graphs(h);  // captured iterations use the splits about to change
  cudaEvent_t e0, e1;
  XCK(cudaEventCreate(&e0));
  XCK(cudaEventCreate(&e1));
  int tuned = 0, wide = 0;
  const int L = (int)h->lv.size();
  for (int l = 0; l + 1 < L && rc == XAMG_OK; ++l) {
    for (int which = 0; which < 3 && rc == XAMG_OK; ++which) {
      signed char &slot = h->lv[l].split[pc][which][lg];
      if (precond == XAMG_PREC_FP64) {
        // y = M x on this level's FP64 work blocks
        RowOpT<double> o = blank<double>();
        double *x_l = l == 0 ? W.R : W.vx[l];
        if (which == 0) {
          o.src = x_l; o.y = W.vr[l];
        } else if (which == 1) {
          o.src = W.vx[l + 1]; o.y = W.vr[l];
        } else {
          o.src = W.vr[l]; o.y = W.vb[l + 1];
        }
        rc = tune_product<double>(h, l, which, precond, o, nv, slot, st, e0, e1, &wide);
      } else {
        RowOpT<float> o = blank<float>();
        if (which == 0) {
          o.src = W.fx[l]; o.y = W.fr[l];
        } else if (which == 1) {
          o.src = W.fx[l + 1]; o.y = W.fr[l];
        } else {
          o.src = W.fr[l]; o.y = W.fb[l + 1];
        }
        rc = tune_product<float>(h, l, which, precond, o, nv, slot, st, e0, e1, &wide);
      }
      ++tuned;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->timing = timing;
  if (rc != XAMG_OK) return rc;
  if (ops_tuned) *ops_tuned = tuned;
  if (ops_wide) *ops_wide = wide;
  return XAMG_OK;
}

int xamg_set_split(xamg_hier *h, int32_t m, int32_t precond, int32_t level, int32_t which,
                   int32_t candidate) {
  if (!h || !h->on_device || m < 1 || m > XAMG_MAX_RHS ||
      (precond != XAMG_PREC_FP64 && precond != XAMG_PREC_FP32 && precond != XAMG_PREC_BF16))
    return XAMG_ERR_INVALID_ARG;
  const int L = (int)h->lv.size();
  if (level < 0 || level >= L || which < 0 || which > 2 || (which > 0 && level + 1 >= L))
    return XAMG_ERR_INVALID_ARG;
  const int nv = pad_nv(m);
  if (candidate < -1 || candidate >= split_candidates(nv, precond != XAMG_PREC_FP64)) return XAMG_ERR_INVALID_ARG;
  int lg = 0;
  while ((1 << lg) < nv) ++lg;
  const int pc = precond == XAMG_PREC_BF16 ? 1 : precond == XAMG_PREC_FP32 ? 0 : 2;
  h->lv[level].split[pc][which][lg] = (signed char)candidate;
  clear_graphs(h);  // captured iterations used the previous split
  return XAMG_OK;
}

int xamg_set_graphs(xamg_hier *h, int32_t enable) {
  if (!h || !h->on_device) return XAMG_ERR_INVALID_ARG;
  XCK(cudaSetDevice(h->device));
  h->use_graphs = enable != 0;
  if (!h->use_graphs) clear_graphs(h);
  return XAMG_OK;
}

int64_t xamg_kernel_launches(void) { return g_launches.load(); }

int xamg_timing_enable(xamg_hier *h, int32_t enable) {
  if (!h || !h->on_device) return XAMG_ERR_INVALID_ARG;
  h->timing = enable != 0;
  if (h->timing) h->tacc.assign(h->lv.size() * 6, TimeAcc());
  return XAMG_OK;
}

int xamg_timing_read(const xamg_hier *h, int32_t level, int32_t which, int64_t *launches,
                     double *total_ms, double *flops, double *bytes) {
  if (!h || !h->on_device || level < 0 || level >= (int)h->lv.size() || which < 0 || which > 5)
    return XAMG_ERR_INVALID_ARG;
  const TimeAcc &t = h->tacc[(size_t)level * 6 + which];
  if (launches) *launches = t.launches;
  if (total_ms) *total_ms = t.ms;
  if (flops) *flops = t.flops;
  if (bytes) *bytes = t.bytes;
  return XAMG_OK;
}

}  // extern "C"
