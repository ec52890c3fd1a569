// vtail.cuh -- the coarse tail of the V(1,1) cycle as one cooperative kernel.
//
// Below a size threshold the levels of a V-cycle are bound by the latency of
// their launches, not by their work: every stage (a Chebyshev step, the
// restriction, the prolongation) is a short dependent chain of loads, and a
// kernel boundary costs several microseconds on top.  The tail kernel runs
// all stages of the levels from l0 down to the coarsest and back up to the
// first post-smoothing step of l0 in one launch, with a grid-wide barrier
// between stages (paper Sec. 2.1: the V-cycle of the MultiGrid preconditioner;
// the fusion is this implementation's).  Each stage runs exactly the row body
// of its single-launch counterpart (rows_vec with the same block width, split,
// sign and epilogue), so results are bitwise those of the launch-per-stage
// path.  Internal to the library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace xamg {

constexpr int kTailMaxStages = 64;  // stages of one tail program

// Stage kinds: the operator (A with the precision's values; P or R with the
// block scalar's values), the sign of the product, and the epilogue.
enum TailKind : int {
  TK_A_YDN = 0,    // A, negated, EPI_Y_DN   (first pre-smoothing step)
  TK_A_YXDP = 1,   // A, negated, EPI_Y_XDP  (last pre-smoothing step)
  TK_A_YD0 = 2,    // A, negated, EPI_Y_D0   (first post-smoothing step)
  TK_A_XLAST = 3,  // A, negated, EPI_XLAST  (last post-smoothing step)
  TK_PR_Y = 4,     // P or R, EPI_Y          (prolongation with init; restriction to the coarsest)
  TK_PR_YD0 = 5,   // R, EPI_Y_D0            (restriction and the next level's first iterate)
  TK_KINDS = 6,
  TK_COARSE = 100  // coarsest solve: op.n = n_c, op.val = A_c^-1, op.src = b, op.y = x
};

template <class TB>
struct TailStage {
  RowOpT<TB> op;
  int kind;
  int wide;  // 1: the one-row-per-warp split (k_rows with slices > 1)
};

// Barrier words in device memory, zeroed before every launch.
struct TailSync {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

template <class TB>
struct TailProg {
  int nstages;
  int extra;                    // added to the barrier's expected arrivals (fault injection; 0)
  unsigned long long limit_ns;  // bound on one barrier wait
  TailSync *sync;
  int32_t *err_host;            // mapped host word, set to 1 when a wait runs out
  TailStage<TB> st[kTailMaxStages];
};

// Launch of the tail program on blocks of nv columns (2..32); vt: 0 = the
// block scalar's values for A, 1 = bf16 values of A with row scales (FP32
// blocks).  Returns the grid size, or -1 on a launch error.
int launch_vtail_f64(const TailProg<double> &p, int nv, cudaStream_t st);
int launch_vtail_f32(const TailProg<float> &p, int nv, int vt, cudaStream_t st);

}  // namespace xamg
