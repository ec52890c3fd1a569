// batch.h -- internal interface of the batched solve (many independent
// systems of uneven size and column count advanced in lockstep, one launch per
// V-cycle stage for all of them of a block width and row split).  Internal to
// the library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "launch.h"

struct xamg_hier;

namespace xamg {

constexpr int kBatchMaxLevels = 32;

// Read-only device view of one frozen hierarchy (FP64 fine operator, FP32
// copies of every operator, Chebyshev weights and coefficients in FP32).
struct HierLevelView {
  int n = 0;       // rows of A_l
  int nc = 0;      // rows of the next level (rows of R_l, columns of P_l)
  int64_t nnzA = 0, nnzP = 0, nnzR = 0;
  const int32_t *Arp = nullptr, *Aci = nullptr, *Prp = nullptr, *Pci = nullptr, *Rrp = nullptr,
                *Rci = nullptr;
  const float *Av = nullptr, *Pv = nullptr, *Rv = nullptr;
  const double *A64 = nullptr;  // FP64 values of A_l
  const float *w32[4] = {nullptr, nullptr, nullptr, nullptr};
  float c1f[4] = {0, 0, 0, 0};
};

struct HierView {
  int L = 0, nc = 0, cheb_steps = 0, device = 0;
  const double *ainv = nullptr;  // inverse of the coarsest operator (nc x nc)
  HierLevelView lv[kBatchMaxLevels];
};

// Fills v for a hierarchy on the device (uploading its FP32 copies if they are
// not there yet).  Returns an XAMG status.
int hier_view(xamg_hier *h, HierView *v);

// ---- device tables of the batched solve ----

// One system's level l (FP32 blocks n x nv row-major).
struct BLevel {
  int n = 0, nc = 0;
  const int32_t *Arp = nullptr, *Aci = nullptr, *Prp = nullptr, *Pci = nullptr, *Rrp = nullptr,
                *Rci = nullptr;
  const float *Av = nullptr, *Pv = nullptr, *Rv = nullptr;
  const float *w[4] = {nullptr, nullptr, nullptr, nullptr};
  float c1[4] = {0, 0, 0, 0};
  float *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr;
  // row split of each operator's product: 0 = narrow (rows per warp as in the
  // single-system kernel), 1 = wide (one row per warp, entries split over
  // the warp's lanes); chosen by the autotuner
  int optA = 0, optP = 0, optR = 0;
};

struct BSys {
  int nv = 0, m = 0, L = 0, nc = 0;
  int64_t n0 = 0;
  const double *ainv = nullptr;  // inverse of the coarsest operator (nc x nc)
  const int32_t *A0rp = nullptr, *A0ci = nullptr;
  const double *A0v = nullptr;  // FP64 fine operator
  int optA0 = 0;                // row split of the FP64 fine products
  const double *B = nullptr;    // caller's right-hand sides (n0 x m)
  double *Xu = nullptr;         // caller's solution block (n0 x m)
  double *Bn = nullptr, *X = nullptr, *R = nullptr, *P = nullptr, *Q = nullptr;
  float *R32 = nullptr, *Z32 = nullptr;
  const float *w0 = nullptr;    // level-0 first Chebyshev weights (FP32)
  ColState *cs = nullptr;
  Flags *flags = nullptr;       // device address of the mapped host counters
  double *part[3] = {nullptr, nullptr, nullptr};
  int *kiter = nullptr;         // iteration counter (advanced by the alpha step)
  const BLevel *lv = nullptr;   // L entries
};

// Stages of the batched V-cycle and Krylov loop.  FP32 stages act on level l
// of every selected system that has a finer-than-coarsest level l.
enum BStage : int {
  BS_PRE1 = 0,     // r = b - A x, d = c1 x + w1 r          (x holds w0 b on entry)
  BS_PRE2,         // r = r - A d, x += d
  BS_RESTRICT,     // b_{l+1} = R r, x_{l+1} = w0_{l+1} b_{l+1}   (level l+1 not coarsest)
  BS_RESTRICT_C,   // b_{l+1} = R r                                 (level l+1 coarsest)
  BS_PROLONG,      // x += P x_{l+1}
  BS_POST1,        // r = b - A x, d = w0 r
  BS_POST2,        // x += d + (c1 d + w1 (r - A d))
  BS_POST2_DOT2,   // the same on level 0 with FP64 partials z.R and z.Q
  BS_AP,           // FP64: Q = A P, partials P.Q
  BS_TRUERES,      // FP64: Q = Bn - A X, partials |Q|^2
  BS_TUNE_A,       // FP32: r = A x (autotuner)
  BS_TUNE_P,       // FP32: x = P x_{l+1}
  BS_TUNE_R,       // FP32: b_{l+1} = R r
  BS_COUNT
};

// Rows per block of stage st's product for a system of nv columns and row
// split opt, and the stage kernel's persistent grid bound.
int bstage_rows_per_block(int st, int nv, int opt);
int bstage_max_grid(int st);

// Batched elementwise steps (grid-stride over each selected system's blocks).
void launch_b_init(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st);
void launch_b_xr(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st);
void launch_b_p(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st);
void launch_b_restart(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st);
void launch_b_copy_out(const BSys *sys, int ns, const int *sel, int grid, cudaStream_t st);
void launch_b_coarse(const BSys *sys, int ns, const int *sel, cudaStream_t st);
// Scalar step `mode` for every selected system (one 1024-thread block per
// system): partial arrays part[i0] (and part[i1] if i1 >= 0) with nblk rows.
void launch_b_scalar(const BSys *sys, int ns, const int *sel, int mode, int i0, int i1, int nblk,
                     double tol, cudaStream_t st);

}  // namespace xamg
