// batch.cu -- batched solve of many independent systems A_s X_s = B_s of
// uneven size n_s and column count m_s: flexible PCG in FP64 around the FP32
// V(1,1) Chebyshev preconditioner of each system's own hierarchy, all systems
// advanced in lockstep.  Every stage of the cycle and of the Krylov loop is
// one persistent launch for all systems (batch_stage*.cu); one iteration is
// replayed as a CUDA graph; the row split of every operator can be chosen by
// timing (autotuner).  The paper solves one system at a time; this is the
// batched form added for many small systems, where single-system launches
// are latency-bound.  Each system computes exactly the steps of
// xamg_solve with precond = XAMG_PREC_FP32 (capi.cu, solve_fpcg).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/xamg_gpu.h"
#include "batch.h"
#include "batch_stage.cuh"
#include "elem.cuh"

namespace xamg {

int launch_bk_g1(int kind, int nv, int opt, const void *params, const int *sel, int grid, cudaStream_t st);
int launch_bk_g2(int kind, int nv, int opt, const void *params, const int *sel, int grid, cudaStream_t st);
int launch_bk_g3(int kind, int nv, int opt, const void *params, const int *sel, int grid, cudaStream_t st);

int launch_bk(int kind, int nv, int opt, const void *params, const int *sel, int grid, cudaStream_t st) {
  int r = launch_bk_g1(kind, nv, opt, params, sel, grid, st);
  if (r != -2) return r;
  r = launch_bk_g2(kind, nv, opt, params, sel, grid, st);
  if (r != -2) return r;
  return launch_bk_g3(kind, nv, opt, params, sel, grid, st);
}

// kernel of each stage
int stage_kind(int st) {
  switch (st) {
    case BS_PRE1: return BK_F_YDN;
    case BS_PRE2: return BK_F_YXDP;
    case BS_RESTRICT: return BK_F_D0_POS;
    case BS_RESTRICT_C: case BS_PROLONG: case BS_TUNE_A: case BS_TUNE_P: case BS_TUNE_R: return BK_F_Y_POS;
    case BS_POST1: return BK_F_D0_NEG;
    case BS_POST2: return BK_F_XLAST;
    case BS_POST2_DOT2: return BK_F_XLAST_DOT2;
    case BS_AP: return BK_D_YDOT;
    default: return BK_D_YDOT2;
  }
}

int bstage_max_grid(int st) { return launch_bk(stage_kind(st), 0, 0, nullptr, nullptr, 0, nullptr); }

int bstage_rows_per_block(int st, int nv, int opt) {
  const int kind = stage_kind(st);
  const bool fp64 = kind == BK_D_YDOT || kind == BK_D_YDOT2;
  if (kind == BK_F_XLAST_DOT2 || fp64) opt = 0;
#define XAMG_RPB(V) \
  case V: return fp64 ? rows_per_block<double, V>(opt) : rows_per_block<float, V>(opt);
  switch (nv) {
    XAMG_RPB(1)
    XAMG_RPB(2)
    XAMG_RPB(4)
    XAMG_RPB(8)
    XAMG_RPB(16)
    XAMG_RPB(32)
    default: return kWarps;
  }
#undef XAMG_RPB
}

#define XAMG_BNV(nv, CALL)                           \
  switch (nv) {                                      \
    case 1: { constexpr int NV = 1; CALL; } break;   \
    case 2: { constexpr int NV = 2; CALL; } break;   \
    case 4: { constexpr int NV = 4; CALL; } break;   \
    case 8: { constexpr int NV = 8; CALL; } break;   \
    case 16: { constexpr int NV = 16; CALL; } break; \
    case 32: { constexpr int NV = 32; CALL; } break; \
    default: break;                                  \
  }

// ---- batched elementwise steps: blocks walk the selected systems in order,
// each with the single-system element loop (elem.cuh) ----
__global__ void __launch_bounds__(kBlock) k_b_init(const BSys *__restrict__ sys, int ns, const int *__restrict__ sel) {
  for (int s = 0; s < ns; ++s) {
    if (!sel[s]) continue;
    const BSys &S = sys[s];
    XAMG_BNV(S.nv, (d_init_fpcg<NV>(S.n0, S.B, S.m, S.Bn, S.R, S.X, S.R32, S.Z32, S.w0, S.part[0])));
    // Q is read (as the second dot operand) by the first V-cycle's last step
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < S.n0 * S.nv; e += (int64_t)gridDim.x * kBlock)
      S.Q[e] = 0.0;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kBlock) k_b_xr(const BSys *__restrict__ sys, int ns, const int *__restrict__ sel) {
  for (int s = 0; s < ns; ++s) {
    if (!sel[s]) continue;
    const BSys &S = sys[s];
    XAMG_BNV(S.nv, (d_fpcg_xr<NV>(S.n0, S.X, S.R, S.P, S.Q, S.cs, S.w0, S.R32, S.Z32, S.part[1])));
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kBlock) k_b_p(const BSys *__restrict__ sys, int ns, const int *__restrict__ sel) {
  for (int s = 0; s < ns; ++s) {
    if (!sel[s]) continue;
    const BSys &S = sys[s];
    XAMG_BNV(S.nv, (d_fpcg_p<NV>(S.n0, S.P, S.Z32, S.cs)));
  }
}

// restarted columns after a confirmation: R = Q (the true residual), then
// the FP32 copy and the first smoother iterate (same elements per thread)
__global__ void __launch_bounds__(kBlock) k_b_restart(const BSys *__restrict__ sys, int ns, const int *__restrict__ sel) {
  for (int s = 0; s < ns; ++s) {
    if (!sel[s]) continue;
    const BSys &S = sys[s];
    XAMG_BNV(S.nv, (d_copy_cols<NV>(S.n0, S.R, S.Q, S.cs), d_to_f32<NV>(S.n0, S.R, S.R32, S.w0, S.Z32)));
  }
}

__global__ void __launch_bounds__(kBlock) k_b_copy_out(const BSys *__restrict__ sys, int ns, const int *__restrict__ sel) {
  for (int s = 0; s < ns; ++s) {
    if (!sel[s]) continue;
    const BSys &S = sys[s];
    XAMG_BNV(S.nv, (d_copy_out<NV>(S.n0, S.X, S.Xu, S.m)));
  }
}

// one block per system: the coarsest-level solve of the FP32 block (FP64
// product with the inverse on the tensor cores)
__global__ void __launch_bounds__(kBlock) k_b_coarse(const BSys *__restrict__ sys, int ns, const int *__restrict__ sel) {
  const int s = blockIdx.x;
  if (s >= ns || !sel[s]) return;
  const BSys &S = sys[s];
  const BLevel &C = S.lv[S.L - 1];
  XAMG_BNV(S.nv, (d_coarse_mma<NV, float, float>(S.nc, S.ainv, C.b, C.x)));
}

// one 1024-thread block per system: the per-column scalar step of the
// Krylov loop; the alpha step advances the system's iteration counter
__global__ void __launch_bounds__(1024) k_b_scalar(const BSys *__restrict__ sys, int ns, const int *__restrict__ sel,
                                                   int mode, int i0, int i1, int nblk, double tol) {
  const int s = blockIdx.x;
  if (s >= ns || !sel[s]) return;
  const BSys &S = sys[s];
  int k = 0;
  if (mode == SM_PCG_ALPHA) k = *S.kiter + 1;
  XAMG_BNV(S.nv, (d_scalar<NV>(mode, S.cs, S.part[i0], i1 >= 0 ? S.part[i1] : nullptr, nblk, tol, k, S.flags)));
  if (threadIdx.x == 0) {
    if (mode == SM_PCG_ALPHA) *S.kiter = k;
    if (mode == SM_INIT) *S.kiter = 0;
  }
}

void launch_b_init(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st) {
  k_b_init<<<grid, kBlock, 0, st>>>(sys, ns, sel);
  g_launches++;
}
void launch_b_xr(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st) {
  k_b_xr<<<grid, kBlock, 0, st>>>(sys, ns, sel);
  g_launches++;
}
void launch_b_p(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st) {
  k_b_p<<<grid, kBlock, 0, st>>>(sys, ns, sel);
  g_launches++;
}
void launch_b_restart(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st) {
  k_b_restart<<<grid, kBlock, 0, st>>>(sys, ns, sel);
  g_launches++;
}
void launch_b_copy_out(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st) {
  k_b_copy_out<<<grid, kBlock, 0, st>>>(sys, ns, sel);
  g_launches++;
}
void launch_b_coarse(const BSys *sys, int ns, const int *sel, cudaStream_t st) {
  k_b_coarse<<<ns, kBlock, 0, st>>>(sys, ns, sel);
  g_launches++;
}
void launch_b_scalar(const BSys *sys, int ns, const int *sel, int mode, int i0, int i1, int nblk,
                     double tol, cudaStream_t st) {
  k_b_scalar<<<ns, 1024, 0, st>>>(sys, ns, sel, mode, i0, i1, nblk, tol);
  g_launches++;
}

}  // namespace xamg

using namespace xamg;

struct xamg_batch {
  int device = 0, ns = 0, Lmax = 0;
  bool use_graph = true;
  std::vector<xamg_hier *> h;
  std::vector<HierView> views;
  std::vector<int> m, nv, L;
  std::vector<BSys> sys_h;
  std::vector<BLevel> lv_h;  // ns x kBatchMaxLevels
  BSys *sys_d = nullptr;
  BLevel *lv_d = nullptr;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  // selection masks on the device: 0 = running systems, 1 = systems being
  // confirmed, 2 = systems restarting columns, 3 = systems needing the final
  // true residual, 4 = one system (autotuner); host copies in pinned memory
  int *sel_d = nullptr;
  int *sel_h = nullptr;
  Flags *flags_h = nullptr, *flags_d = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_launches = 0;
  std::vector<int> gA, gP, gR;  // grids per level of the A, P and R stages
  int g_ap = 0, g_tr = 0, g_post0 = 0, g_elem = 0;
  int launches_per_iter = 0;
  int ops_tuned = 0, ops_wide = 0;
  // host staging of one launch's parameter block (the larger of the FP32 and
  // FP64 forms)
  std::vector<char> params = std::vector<char>(std::max(sizeof(StageParams<float>), sizeof(StageParams<double>)));
};

namespace {

#define BCK(call)                                                             \
  do {                                                                        \
    cudaError_t e__ = (call);                                                 \
    if (e__ != cudaSuccess)                                                   \
      return e__ == cudaErrorMemoryAllocation ? XAMG_ERR_OOM : XAMG_ERR_CUDA; \
  } while (0)

#define BRET(expr)                  \
  do {                              \
    const int r__ = (expr);         \
    if (r__ != XAMG_OK) return r__; \
  } while (0)

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

int pad_to_nv(int m) {
  int v = 1;
  while (v < m) v <<= 1;
  return v;
}

int *sel_dev(xamg_batch *b, int which) { return b->sel_d + (size_t)which * b->ns; }
int *sel_host(xamg_batch *b, int which) { return b->sel_h + (size_t)which * b->ns; }

int upload_sel(xamg_batch *b, int which) {
  BCK(cudaMemcpyAsync(sel_dev(b, which), sel_host(b, which), b->ns * sizeof(int), cudaMemcpyHostToDevice, b->st));
  return XAMG_OK;
}

int upload_tables(xamg_batch *b) {
  BCK(cudaMemcpyAsync(b->lv_d, b->lv_h.data(), b->lv_h.size() * sizeof(BLevel), cudaMemcpyHostToDevice, b->st));
  BCK(cudaMemcpyAsync(b->sys_d, b->sys_h.data(), b->sys_h.size() * sizeof(BSys), cudaMemcpyHostToDevice, b->st));
  BCK(cudaStreamSynchronize(b->st));
  return XAMG_OK;
}

BLevel &blev(xamg_batch *b, int s, int l) { return b->lv_h[(size_t)s * kBatchMaxLevels + l]; }

// grid of stage st on level l: enough blocks for the largest selected system
// (its rows over the rows one block takes), at most the persistent grid
int stage_grid(xamg_batch *b, int st, int l) {
  int64_t need = 1;
  for (int s = 0; s < b->ns; ++s) {
    const BSys &S = b->sys_h[s];
    int64_t rows;
    int opt;
    if (st == BS_AP || st == BS_TRUERES) {
      rows = S.n0;
      opt = S.optA0;
    } else {
      if (l >= S.L - 1) continue;
      const BLevel &V = blev(b, s, l);
      if (st == BS_RESTRICT || st == BS_RESTRICT_C || st == BS_TUNE_R) {
        rows = V.nc;
        opt = V.optR;
      } else if (st == BS_PROLONG || st == BS_TUNE_P) {
        rows = V.n;
        opt = V.optP;
      } else {
        rows = V.n;
        opt = V.optA;
      }
    }
    const int rpb = bstage_rows_per_block(st, S.nv, opt);
    need = std::max<int64_t>(need, (rows + rpb - 1) / rpb);
  }
  return (int)std::min<int64_t>(need, bstage_max_grid(st));
}

void compute_grids(xamg_batch *b) {
  const int Lm = std::max(1, b->Lmax - 1);
  b->gA.assign(Lm, 1);
  b->gP.assign(Lm, 1);
  b->gR.assign(Lm, 1);
  for (int l = 0; l + 1 < b->Lmax; ++l) {
    b->gA[l] = stage_grid(b, BS_PRE1, l);
    b->gP[l] = stage_grid(b, BS_PROLONG, l);
    b->gR[l] = stage_grid(b, BS_RESTRICT, l);
  }
  b->g_ap = stage_grid(b, BS_AP, 0);
  b->g_tr = stage_grid(b, BS_TRUERES, 0);
  b->g_post0 = stage_grid(b, BS_POST2_DOT2, 0);
  int64_t emax = 1;
  for (const BSys &S : b->sys_h) emax = std::max<int64_t>(emax, S.n0 * S.nv);
  b->g_elem = (int)std::max<int64_t>(1, std::min<int64_t>((emax + kBlock - 1) / kBlock, std::min<int64_t>((int64_t)device_sm_count() * 8, kMaxGrid)));
}

template <class TB>
RowOpT<TB> blank_row() {
  RowOpT<TB> o;
  std::memset(&o, 0, sizeof(o));
  return o;
}

// The row operation of stage st on level l of system s, or false if the
// stage does not apply to it (mirrors presmooth / postsmooth / vcycle and the
// Krylov steps of the single-system solve with the FP32 preconditioner).
bool stage_op_f(xamg_batch *b, int st, int s, int l, RowOpF &o, int &opt) {
  const BSys &S = b->sys_h[s];
  if (l >= S.L - 1) return false;
  const BLevel &V = blev(b, s, l);
  const BLevel *C = l + 1 < S.L ? &blev(b, s, l + 1) : nullptr;
  o = blank_row<float>();
  auto A = [&]() { o.n = V.n; o.rowptr = V.Arp; o.col = V.Aci; o.val = V.Av; opt = V.optA; };
  auto P = [&]() { o.n = V.n; o.rowptr = V.Prp; o.col = V.Pci; o.val = V.Pv; opt = V.optP; };
  auto R = [&]() { o.n = V.nc; o.rowptr = V.Rrp; o.col = V.Rci; o.val = V.Rv; opt = V.optR; };
  switch (st) {
    case BS_PRE1:
      A(); o.init = V.b; o.src = V.x; o.y = V.r; o.dp = V.x; o.w = V.w[1]; o.c1 = V.c1[1]; o.dnext = V.d;
      return true;
    case BS_PRE2:
      A(); o.init = V.r; o.src = V.d; o.y = V.r; o.dp = V.d; o.x = V.x;
      return true;
    case BS_RESTRICT:
      if (l + 2 >= S.L) return false;
      R(); o.src = V.r; o.y = C->b; o.w = C->w[0]; o.dnext = C->x;
      return true;
    case BS_RESTRICT_C:
      if (l + 2 != S.L) return false;
      R(); o.src = V.r; o.y = C->b;
      return true;
    case BS_PROLONG:
      P(); o.init = V.x; o.src = C->x; o.y = V.x;
      return true;
    case BS_POST1:
      A(); o.init = V.b; o.src = V.x; o.y = V.r; o.w = V.w[0]; o.dnext = V.d;
      return true;
    case BS_POST2:
    case BS_POST2_DOT2:
      A(); o.init = V.r; o.src = V.d; o.dp = V.d; o.w = V.w[1]; o.c1 = V.c1[1]; o.x = V.x;
      if (st == BS_POST2_DOT2) {
        o.dot_u = S.R; o.partials = S.part[1]; o.dot_u2 = S.Q; o.partials2 = S.part[2];
        opt = 0;
      }
      return true;
    case BS_TUNE_A:
      A(); o.src = V.x; o.y = V.r;
      return true;
    case BS_TUNE_P:
      P(); o.src = C->x; o.y = V.r;
      return true;
    case BS_TUNE_R:
      R(); o.src = V.r; o.y = C->b;
      return true;
    default:
      return false;
  }
}

bool stage_op_d(xamg_batch *b, int st, int s, RowOp &o, int &opt) {
  const BSys &S = b->sys_h[s];
  o = blank_row<double>();
  o.n = (int)S.n0; o.rowptr = S.A0rp; o.col = S.A0ci; o.val = S.A0v;
  opt = 0;
  if (st == BS_AP) {
    o.src = S.P; o.y = S.Q; o.dot_u = S.P; o.partials = S.part[0];
  } else {
    o.init = S.Bn; o.src = S.X; o.y = S.Q; o.partials2 = S.part[2];
  }
  return true;
}

// Stage st on level l for the systems of selection mask `sel` to which the
// stage applies: one launch per (block width, row split) present, and per
// kStageOps systems of that pair; `only` >= 0 restricts the list to that
// system (autotuner).  With `count` set, nothing is launched and *count
// receives the number of launches.
template <class TB>
int stage_t(xamg_batch *b, int st, int sel, int l, int grid, int only, int *count) {
  StageParams<TB> &P = *reinterpret_cast<StageParams<TB> *>(b->params.data());
  const int kind = stage_kind(st);
  // the kernels without a wide split run every entry narrow
  const bool has_wide = kind != BK_F_XLAST_DOT2 && kind != BK_D_YDOT && kind != BK_D_YDOT2;
  if (count) *count = 0;
  for (int nv = 1; nv <= XAMG_MAX_RHS; nv <<= 1) {
    for (int split = 0; split < (has_wide ? 2 : 1); ++split) {
      P.count = 0;
      auto flush = [&]() -> int {
        if (!P.count) return XAMG_OK;
        if (count) {
          ++*count;
          P.count = 0;
          return XAMG_OK;
        }
        const int r = launch_bk(kind, nv, split, &P, sel_dev(b, sel), grid, b->st);
        P.count = 0;
        return r < 0 ? XAMG_ERR_CUDA : XAMG_OK;
      };
      for (int s = 0; s < b->ns; ++s) {
        if ((only >= 0 && s != only) || b->sys_h[s].nv != nv) continue;
        RowOpT<TB> o;
        int opt = 0;
        bool on;
        if constexpr (sizeof(TB) == 8) on = stage_op_d(b, st, s, o, opt);
        else on = stage_op_f(b, st, s, l, o, opt);
        if (!on || (has_wide && (opt != 0) != (split != 0))) continue;
        const int i = P.count++;
        P.sys[i] = s;
        P.op[i] = o;
        if (P.count == kStageOps) BRET(flush());
      }
      BRET(flush());
    }
  }
  return XAMG_OK;
}

int stage(xamg_batch *b, int st, int sel, int l, int grid, int only = -1, int *count = nullptr) {
  if (st == BS_AP || st == BS_TRUERES) return stage_t<double>(b, st, sel, l, grid, only, count);
  return stage_t<float>(b, st, sel, l, grid, only, count);
}

// Launches of one steady iteration (iteration_b) for every system together.
int count_iteration_launches(xamg_batch *b) {
  int total = 0, c = 0;
  auto add = [&](int st, int l) {
    stage(b, st, 0, l, 1, -1, &c);
    total += c;
  };
  for (int l = 0; l + 1 < b->Lmax; ++l) {
    add(BS_PRE1, l);
    add(BS_PRE2, l);
    add(BS_RESTRICT, l);
    add(BS_RESTRICT_C, l);
    add(BS_PROLONG, l);
    add(BS_POST1, l);
    add(l == 0 ? BS_POST2_DOT2 : BS_POST2, l);
  }
  add(BS_AP, 0);
  // coarsest solve, flexible beta, p update, alpha, x/r update, convergence test
  return total + 6;
}

// the FP32 V(1,1) cycle of every system selected by mask `sel`: on entry each
// system's level-0 x holds w0 .* b; the last step on level 0 writes the FP64
// partials z.R (part[1]) and z.Q (part[2]) over g_post0 blocks
int vcycle_b(xamg_batch *b, int sel) {
  for (int l = 0; l + 1 < b->Lmax; ++l) {
    BRET(stage(b, BS_PRE1, sel, l, b->gA[l]));
    BRET(stage(b, BS_PRE2, sel, l, b->gA[l]));
    BRET(stage(b, BS_RESTRICT, sel, l, b->gR[l]));
    BRET(stage(b, BS_RESTRICT_C, sel, l, b->gR[l]));
  }
  launch_b_coarse(b->sys_d, b->ns, sel_dev(b, sel), b->st);
  for (int l = b->Lmax - 2; l >= 0; --l) {
    BRET(stage(b, BS_PROLONG, sel, l, b->gP[l]));
    BRET(stage(b, BS_POST1, sel, l, b->gA[l]));
    BRET(stage(b, l == 0 ? BS_POST2_DOT2 : BS_POST2, sel, l, l == 0 ? b->g_post0 : b->gA[l]));
  }
  BCK(cudaPeekAtLastError());
  return XAMG_OK;
}

// A p (pT q), alpha, x/r update (|r|^2), convergence test
int krylov_b(xamg_batch *b, double tol) {
  const int *sel = sel_dev(b, 0);
  BRET(stage(b, BS_AP, 0, 0, b->g_ap));
  launch_b_scalar(b->sys_d, b->ns, sel, SM_PCG_ALPHA, 0, -1, b->g_ap, tol, b->st);
  launch_b_xr(b->sys_d, b->ns, sel, b->g_elem, b->st);
  launch_b_scalar(b->sys_d, b->ns, sel, SM_PCG_CONV, 1, -1, b->g_elem, tol, b->st);
  BCK(cudaPeekAtLastError());
  return XAMG_OK;
}

// the steady iteration: preconditioner, flexible beta, p update, then the
// next A p .. convergence test
int iteration_b(xamg_batch *b, double tol) {
  const int *sel = sel_dev(b, 0);
  BRET(vcycle_b(b, 0));
  launch_b_scalar(b->sys_d, b->ns, sel, SM_FPCG_BETA, 1, 2, b->g_post0, tol, b->st);
  launch_b_p(b->sys_d, b->ns, sel, b->g_elem, b->st);
  return krylov_b(b, tol);
}

int plan_workspace(xamg_batch *b, bool alloc) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char * {
    char *p = alloc ? b->ws + off : nullptr;
    off += al256(bytes);
    return p;
  };
  const int part_rows = std::max(std::max(b->g_elem, b->g_ap), std::max(b->g_post0, b->g_tr));
  for (int s = 0; s < b->ns; ++s) {
    BSys &S = b->sys_h[s];
    const HierView &H = b->views[s];
    const size_t n0 = (size_t)S.n0, nv = (size_t)S.nv;
    const size_t d = n0 * nv * sizeof(double), f = n0 * nv * sizeof(float);
    S.Bn = (double *)take(d);
    S.X = (double *)take(d);
    S.R = (double *)take(d);
    S.P = (double *)take(d);
    S.Q = (double *)take(d);
    S.R32 = (float *)take(f);
    S.Z32 = (float *)take(f);
    for (int l = 0; l < S.L; ++l) {
      BLevel &V = blev(b, s, l);
      const size_t fb = (size_t)H.lv[l].n * nv * sizeof(float);
      if (l == 0) {
        V.b = S.R32;
        V.x = S.Z32;
      } else {
        V.b = (float *)take(fb);
        V.x = (float *)take(fb);
      }
      if (l + 1 < S.L) {
        V.r = (float *)take(fb);
        V.d = (float *)take(fb);
      }
    }
    for (int i = 0; i < 3; ++i) S.part[i] = (double *)take((size_t)part_rows * nv * sizeof(double));
    S.cs = (ColState *)take(sizeof(ColState));
    S.kiter = (int *)take(sizeof(int));
  }
  if (!alloc) {
    b->ws_bytes = off;
    BCK(cudaMalloc((void **)&b->ws, off));
    BCK(cudaMemset(b->ws, 0, off));
  }
  return XAMG_OK;
}

// Times y = M x for one system's operator under both row splits and keeps
// the faster one.
int autotune(xamg_batch *b) {
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  int *one = sel_host(b, 4);
  int rc = XAMG_OK;
  for (int s = 0; s < b->ns && rc == XAMG_OK; ++s) {
    std::fill(one, one + b->ns, 0);
    one[s] = 1;
    if ((rc = upload_sel(b, 4)) != XAMG_OK) break;
    for (int l = 0; l + 1 < b->sys_h[s].L && rc == XAMG_OK; ++l) {
      for (int op = 0; op < 3 && rc == XAMG_OK; ++op) {
        const int st = op == 0 ? BS_TUNE_A : op == 1 ? BS_TUNE_P : BS_TUNE_R;
        BLevel &V = blev(b, s, l);
        int &opt = op == 0 ? V.optA : op == 1 ? V.optP : V.optR;
        float best = 1e30f;
        int best_opt = 0;
        for (int o = 0; o < 2; ++o) {
          opt = o;
          // the grid this system alone needs under this split
          const int64_t rows = op == 2 ? V.nc : V.n;
          const int rpb = bstage_rows_per_block(st, b->sys_h[s].nv, o);
          const int grid = (int)std::min<int64_t>((rows + rpb - 1) / rpb, bstage_max_grid(st));
          if ((rc = stage(b, st, 4, l, grid, s)) != XAMG_OK) break;
          cudaEventRecord(e0, b->st);
          for (int r = 0; r < 3; ++r) stage(b, st, 4, l, grid, s);
          cudaEventRecord(e1, b->st);
          if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = XAMG_ERR_CUDA;
            break;
          }
          float ms = 0.0f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best) {
            best = ms;
            best_opt = o;
          }
        }
        opt = best_opt;
        b->ops_tuned++;
        b->ops_wide += best_opt;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BRET(rc);
  return upload_tables(b);
}

void destroy(xamg_batch *b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ws) cudaFree(b->ws);
  if (b->sys_d) cudaFree(b->sys_d);
  if (b->lv_d) cudaFree(b->lv_d);
  if (b->sel_d) cudaFree(b->sel_d);
  if (b->sel_h) cudaFreeHost(b->sel_h);
  if (b->flags_h) cudaFreeHost(b->flags_h);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

}  // namespace

extern "C" {

void xamg_batch_opts_default(xamg_batch_opts *o) {
  if (!o) return;
  o->autotune = 1;
  o->use_graph = 1;
}

int xamg_batch_create(xamg_hier *const *h, const int32_t *m, int32_t count, const xamg_batch_opts *opts,
                      xamg_batch **out) {
  if (!out) return XAMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!h || !m || count < 1) return XAMG_ERR_INVALID_ARG;
  xamg_batch_opts o;
  xamg_batch_opts_default(&o);
  if (opts) o = *opts;
  xamg_batch *b = new (std::nothrow) xamg_batch();
  if (!b) return XAMG_ERR_OOM;
  b->ns = count;
  b->use_graph = o.use_graph != 0;
  b->h.assign(h, h + count);
  b->views.resize(count);
  b->sys_h.resize(count);
  b->lv_h.assign((size_t)count * kBatchMaxLevels, BLevel());
  int rc = XAMG_OK;
  auto fail = [&](int code) {
    destroy(b);
    return code;
  };
  for (int s = 0; s < count; ++s) {
    if (!h[s] || m[s] < 1 || m[s] > XAMG_MAX_RHS) return fail(XAMG_ERR_INVALID_ARG);
    if ((rc = hier_view(h[s], &b->views[s])) != XAMG_OK) return fail(rc);
    const HierView &H = b->views[s];
    if (s == 0) b->device = H.device;
    // each system needs at least two levels and the default two Chebyshev steps
    if (H.device != b->device || H.L < 2 || H.cheb_steps != 2) return fail(XAMG_ERR_INVALID_ARG);
  }
  if (cudaSetDevice(b->device) != cudaSuccess) return fail(XAMG_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) return fail(XAMG_ERR_CUDA);
  if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) return fail(XAMG_ERR_CUDA);
  for (int s = 0; s < count; ++s) {
    const HierView &H = b->views[s];
    BSys &S = b->sys_h[s];
    S.nv = pad_to_nv(m[s]);
    S.m = m[s];
    S.L = H.L;
    S.nc = H.nc;
    S.n0 = H.lv[0].n;
    S.ainv = H.ainv;
    S.A0rp = H.lv[0].Arp;
    S.A0ci = H.lv[0].Aci;
    S.A0v = H.lv[0].A64;
    S.w0 = H.lv[0].w32[0];
    b->Lmax = std::max(b->Lmax, H.L);
    for (int l = 0; l < H.L; ++l) {
      BLevel &V = blev(b, s, l);
      const HierLevelView &W = H.lv[l];
      V.n = W.n;
      V.nc = W.nc;
      V.Arp = W.Arp; V.Aci = W.Aci; V.Av = W.Av;
      V.Prp = W.Prp; V.Pci = W.Pci; V.Pv = W.Pv;
      V.Rrp = W.Rrp; V.Rci = W.Rci; V.Rv = W.Rv;
      for (int k = 0; k < 4; ++k) {
        V.w[k] = W.w32[k];
        V.c1[k] = W.c1f[k];
      }
      // untuned split: the single-system rule (long FP32 rows of wide blocks,
      // or one column with long rows, split over the warp)
      auto rule = [&](int64_t nnz, int rows) {
        const double avg = rows ? (double)nnz / rows : 0.0;
        return (S.nv == 1 && avg >= 24.0) || (S.nv >= 16 && avg >= 64.0) ? 1 : 0;
      };
      V.optA = rule(W.nnzA, W.n);
      V.optP = rule(W.nnzP, W.n);
      V.optR = rule(W.nnzR, W.nc);
    }
  }
  if (cudaMalloc((void **)&b->lv_d, b->lv_h.size() * sizeof(BLevel)) != cudaSuccess ||
      cudaMalloc((void **)&b->sys_d, b->sys_h.size() * sizeof(BSys)) != cudaSuccess ||
      cudaMalloc((void **)&b->sel_d, (size_t)5 * count * sizeof(int)) != cudaSuccess ||
      cudaHostAlloc((void **)&b->sel_h, (size_t)5 * count * sizeof(int), cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void **)&b->flags_h, (size_t)count * sizeof(Flags), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void **)&b->flags_d, b->flags_h, 0) != cudaSuccess)
    return fail(XAMG_ERR_OOM);
  for (int s = 0; s < count; ++s) {
    BSys &S = b->sys_h[s];
    S.lv = b->lv_d + (size_t)s * kBatchMaxLevels;
    S.flags = b->flags_d + s;
  }
  compute_grids(b);
  if ((rc = plan_workspace(b, false)) != XAMG_OK) return fail(rc);
  if ((rc = plan_workspace(b, true)) != XAMG_OK) return fail(rc);
  if ((rc = upload_tables(b)) != XAMG_OK) return fail(rc);
  if (o.autotune) {
    if ((rc = autotune(b)) != XAMG_OK) return fail(rc);
    // grids follow the chosen splits; the partial arrays were sized for the
    // persistent grid bound of every dot stage, which does not depend on them
    const int pr0 = std::max(std::max(b->g_elem, b->g_ap), std::max(b->g_post0, b->g_tr));
    compute_grids(b);
    const int pr1 = std::max(std::max(b->g_elem, b->g_ap), std::max(b->g_post0, b->g_tr));
    if (pr1 > pr0) return fail(XAMG_ERR_CUDA);
  }
  b->launches_per_iter = count_iteration_launches(b);
  *out = b;
  return XAMG_OK;
}

int xamg_batch_destroy(xamg_batch *b) {
  if (!b) return XAMG_ERR_INVALID_ARG;
  cudaSetDevice(b->device);
  destroy(b);
  return XAMG_OK;
}

int xamg_batch_info(const xamg_batch *b, int32_t *launches_per_iteration, int32_t *ops_tuned, int32_t *ops_wide,
                    int64_t *workspace_bytes) {
  if (!b) return XAMG_ERR_INVALID_ARG;
  if (launches_per_iteration) *launches_per_iteration = b->launches_per_iter;
  if (ops_tuned) *ops_tuned = b->ops_tuned;
  if (ops_wide) *ops_wide = b->ops_wide;
  if (workspace_bytes) *workspace_bytes = (int64_t)b->ws_bytes;
  return XAMG_OK;
}

int xamg_batch_solve(xamg_batch *b, const double *const *B, double *const *X, double tol, int32_t maxit,
                     void *stream, xamg_stats *stats) {
  if (!b || !B || !X || !(tol > 0.0) || maxit < 0) return XAMG_ERR_INVALID_ARG;
  for (int s = 0; s < b->ns; ++s)
    if (!B[s] || !X[s]) return XAMG_ERR_INVALID_ARG;
  BCK(cudaSetDevice(b->device));
  const int ns = b->ns;
  cudaStream_t user = (cudaStream_t)stream;
  // order after the caller's earlier work on its stream
  BCK(cudaEventRecord(b->ev, user));
  BCK(cudaStreamWaitEvent(b->st, b->ev, 0));
  for (int s = 0; s < ns; ++s) {
    b->sys_h[s].B = B[s];
    b->sys_h[s].Xu = X[s];
  }
  BRET(upload_tables(b));
  int *run = sel_host(b, 0);
  std::vector<int> confirmed(ns, 0), vcycles(ns, 0), iterations(ns, 0);
  std::fill(run, run + ns, 1);
  BRET(upload_sel(b, 0));
  launch_b_init(b->sys_d, ns, sel_dev(b, 0), b->g_elem, b->st);
  launch_b_scalar(b->sys_d, ns, sel_dev(b, 0), SM_INIT, 0, -1, b->g_elem, tol, b->st);
  BCK(cudaStreamSynchronize(b->st));
  BCK(cudaGetLastError());
  for (int s = 0; s < ns; ++s) {
    if (b->flags_h[s].breakdown < 0) return XAMG_ERR_NONFINITE;
    run[s] = b->flags_h[s].active > 0;
  }
  BRET(upload_sel(b, 0));
  bool any = std::any_of(run, run + ns, [](int v) { return v != 0; });
  if (any) {
    // first preconditioner application and direction, then the first A p
    BRET(vcycle_b(b, 0));
    launch_b_scalar(b->sys_d, ns, sel_dev(b, 0), SM_PCG_BETA, 1, -1, b->g_post0, tol, b->st);
    launch_b_p(b->sys_d, ns, sel_dev(b, 0), b->g_elem, b->st);
    for (int s = 0; s < ns; ++s) vcycles[s] += run[s];
  }
  for (int k = 1; k <= maxit && any; ++k) {
    if (k == 1) {
      BRET(krylov_b(b, tol));
    } else if (b->use_graph) {
      if (!b->gexec) {
        // capture the steady iteration once; its launches read the masks and
        // tables from device memory, so one graph serves every solve
        const int64_t before = g_launches.load();
        BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
        const int rc = iteration_b(b, tol);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(b->st, &g);
        BRET(rc);
        BCK(ce);
        b->graph = g;
        BCK(cudaGraphInstantiate(&b->gexec, b->graph, 0));
        b->graph_launches = g_launches.load() - before;
        g_launches -= b->graph_launches;  // counted per replay below
      }
      BCK(cudaGraphLaunch(b->gexec, b->st));
      g_launches += b->graph_launches;
    } else {
      BRET(iteration_b(b, tol));
    }
    if (k > 1)
      for (int s = 0; s < ns; ++s) vcycles[s] += run[s];
    for (int s = 0; s < ns; ++s) iterations[s] += run[s];
    BCK(cudaStreamSynchronize(b->st));
    BCK(cudaGetLastError());
    // systems whose columns all stopped: confirm with the true residual
    int *conf = sel_host(b, 1);
    bool anyc = false;
    for (int s = 0; s < ns; ++s) {
      conf[s] = run[s] && b->flags_h[s].active == 0;
      anyc |= conf[s] != 0;
    }
    if (anyc) {
      BRET(upload_sel(b, 1));
      BRET(stage(b, BS_TRUERES, 1, 0, b->g_tr));
      launch_b_scalar(b->sys_d, ns, sel_dev(b, 1), SM_CONFIRM, 2, -1, b->g_tr, tol, b->st);
      BCK(cudaStreamSynchronize(b->st));
      BCK(cudaGetLastError());
      int *rs = sel_host(b, 2);
      bool anyr = false;
      for (int s = 0; s < ns; ++s) {
        rs[s] = 0;
        if (!conf[s]) continue;
        if (b->flags_h[s].reactivated == 0) {
          run[s] = 0;
          confirmed[s] = 1;
        } else {
          rs[s] = 1;
          anyr = true;
        }
      }
      if (anyr) {
        BRET(upload_sel(b, 2));
        launch_b_restart(b->sys_d, ns, sel_dev(b, 2), b->g_elem, b->st);
      }
      BRET(upload_sel(b, 0));
    }
    any = std::any_of(run, run + ns, [](int v) { return v != 0; });
  }
  // true residual of the systems that did not end on a confirmation
  int *fin = sel_host(b, 3);
  bool anyf = false;
  for (int s = 0; s < ns; ++s) {
    fin[s] = !confirmed[s];
    anyf |= fin[s] != 0;
  }
  if (anyf) {
    BRET(upload_sel(b, 3));
    BRET(stage(b, BS_TRUERES, 3, 0, b->g_tr));
    launch_b_scalar(b->sys_d, ns, sel_dev(b, 3), SM_FINAL, 2, -1, b->g_tr, tol, b->st);
  }
  std::fill(run, run + ns, 1);
  BRET(upload_sel(b, 0));
  launch_b_copy_out(b->sys_d, ns, sel_dev(b, 0), b->g_elem, b->st);
  std::vector<ColState> cs(ns);
  for (int s = 0; s < ns; ++s)
    BCK(cudaMemcpyAsync(&cs[s], b->sys_h[s].cs, sizeof(ColState), cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  BCK(cudaGetLastError());
  // later work on the caller's stream sees the solution
  BCK(cudaEventRecord(b->ev, b->st));
  BCK(cudaStreamWaitEvent(user, b->ev, 0));
  int rc = XAMG_OK;
  for (int s = 0; s < ns; ++s) {
    int maxits = 0;
    for (int j = 0; j < b->sys_h[s].m; ++j) {
      int status;
      double rel = 0.0;
      if (cs[s].state[j] == 4) {
        status = XAMG_COL_CONVERGED;
      } else {
        rel = cs[s].tn[j] / cs[s].nb[j];
        if (cs[s].state[j] == 3) status = XAMG_COL_BREAKDOWN;
        else status = rel <= tol ? XAMG_COL_CONVERGED : XAMG_COL_NOT_CONVERGED;
      }
      if (status == XAMG_COL_BREAKDOWN) rc = XAMG_BREAKDOWN;
      else if (status == XAMG_COL_NOT_CONVERGED && rc == XAMG_OK) rc = XAMG_NOT_CONVERGED;
      maxits = std::max(maxits, (int)cs[s].iters[j]);
      if (stats) {
        if (stats[s].iters) stats[s].iters[j] = cs[s].iters[j];
        if (stats[s].relres) stats[s].relres[j] = rel;
        if (stats[s].status) stats[s].status[j] = status;
      }
    }
    if (stats) {
      stats[s].iterations = maxits;
      stats[s].vcycles = vcycles[s];
    }
  }
  return rc;
}

}  // extern "C"
