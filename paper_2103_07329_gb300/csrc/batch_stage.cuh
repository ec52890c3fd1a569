// batch_stage.cuh -- the batched row stages: one persistent launch applies
// one step of the V-cycle (or of the Krylov loop) to a list of systems.  The
// host builds each system's row operation (as for a single-system launch) and
// passes the whole list as one kernel parameter block, so every field is read
// from the constant bank where it is used, as in the single-system kernel.
// Blocks walk the list in order; within a system the warps take the rows in
// the single-system grid-stride order (rows_vec / rows_sliced of
// kernels.cuh), so each system's products and partial dot sums are computed
// exactly as a single-system launch with the same grid computes them.  The
// column count NV and the row split of each entry are runtime values: a
// switch selects the compile-time body.  Included by batch.cu and
// batch_stage*.cu (one group of kernels per unit).
#pragma once
#include <algorithm>

#include "batch.h"
#include "kernels.cuh"

namespace xamg {

template <class TB, class TV, int NV, int S, bool NEG, int EPI>
__device__ __forceinline__ void row_body(const RowOpT<TB> &op) {
  if constexpr (S == 1) {
    rows_vec<TB, TV, NV, row_vec<TB, NV>(), 1, NEG, EPI>(op);
  } else if constexpr (NV > 1) {
    rows_vec<TB, TV, NV, row_vec<TB, NV>(), S, NEG, EPI>(op);
  } else {
    rows_sliced<TB, TV, NV, S, NEG, EPI>(op);
  }
}

// Row splits: narrow = the single-system kernel's default (4 lanes per row
// for one column, else one group of NV/VEC lanes per row); wide = one row per
// warp, its entries split into slices over the warp.
template <class TB, int NV>
__host__ __device__ constexpr int narrow_s() { return NV == 1 ? 4 : 1; }
template <class TB, int NV>
__host__ __device__ constexpr int wide_s() { return NV == 1 ? 16 : 32 / (NV / row_vec<TB, NV>()); }

template <class TB, int NV>
__host__ __device__ constexpr int rows_per_block(int opt) {
  return kWarps * (32 / ((NV == 1 ? 1 : NV / row_vec<TB, NV>()) * (opt ? wide_s<TB, NV>() : narrow_s<TB, NV>())));
}

// WIDE: whether the wide split is compiled for this kernel (the kernels that
// only act on the fine level, a short-row stencil, keep the narrow one).
template <class TB, class TV, bool NEG, int EPI, bool WIDE>
__device__ __forceinline__ void row_dispatch(int nv, int opt, const RowOpT<TB> &op) {
#define XAMG_RD(V)                                                       \
  case V:                                                                \
    if (WIDE && opt)                                                     \
      row_body<TB, TV, V, wide_s<TB, V>(), NEG, EPI>(op);                \
    else                                                                 \
      row_body<TB, TV, V, narrow_s<TB, V>(), NEG, EPI>(op);              \
    break;
  switch (nv) {
    XAMG_RD(1)
    XAMG_RD(2)
    XAMG_RD(4)
    XAMG_RD(8)
    XAMG_RD(16)
    XAMG_RD(32)
    default: break;
  }
#undef XAMG_RD
}

// Entries per launch: the parameter block stays below the 32 KB limit of
// kernel parameters.
constexpr int kStageOps = 96;

template <class TB>
struct StageParams {
  int count;
  int sys[kStageOps];              // system index (selection mask)
  unsigned char nv[kStageOps];     // block width
  unsigned char opt[kStageOps];    // row split
  RowOpT<TB> op[kStageOps];
};

// The (block scalar, sign, epilogue, wide split) combinations the batched
// solve uses.
enum BKind : int {
  BK_F_YDN = 0,     // FP32 first pre-smoothing step
  BK_F_YXDP,        // FP32 last pre-smoothing step
  BK_F_D0_POS,      // FP32 restriction writing the next level's first iterate
  BK_F_Y_POS,       // FP32 plain product (restriction to the coarsest, prolongation, tuning)
  BK_F_D0_NEG,      // FP32 first post-smoothing step
  BK_F_XLAST,       // FP32 last post-smoothing step
  BK_F_XLAST_DOT2,  // the same on level 0 with two FP64 partial dots
  BK_D_YDOT,        // FP64 A p with p.q
  BK_D_YDOT2,       // FP64 true residual with |r|^2
  BK_COUNT
};

template <int K> struct KD;
template <> struct KD<BK_F_YDN> { using TB = float; static constexpr bool NEG = true, WIDE = true; static constexpr int EPI = EPI_Y_DN; };
template <> struct KD<BK_F_YXDP> { using TB = float; static constexpr bool NEG = true, WIDE = true; static constexpr int EPI = EPI_Y_XDP; };
template <> struct KD<BK_F_D0_POS> { using TB = float; static constexpr bool NEG = false, WIDE = true; static constexpr int EPI = EPI_Y_D0; };
template <> struct KD<BK_F_Y_POS> { using TB = float; static constexpr bool NEG = false, WIDE = true; static constexpr int EPI = EPI_Y; };
template <> struct KD<BK_F_D0_NEG> { using TB = float; static constexpr bool NEG = true, WIDE = true; static constexpr int EPI = EPI_Y_D0; };
template <> struct KD<BK_F_XLAST> { using TB = float; static constexpr bool NEG = true, WIDE = true; static constexpr int EPI = EPI_XLAST; };
template <> struct KD<BK_F_XLAST_DOT2> { using TB = float; static constexpr bool NEG = true, WIDE = false; static constexpr int EPI = EPI_XLAST_DOT2; };
template <> struct KD<BK_D_YDOT> { using TB = double; static constexpr bool NEG = false, WIDE = false; static constexpr int EPI = EPI_Y_DOT; };
template <> struct KD<BK_D_YDOT2> { using TB = double; static constexpr bool NEG = true, WIDE = false; static constexpr int EPI = EPI_Y_DOT2; };

template <int K>
__global__ void __launch_bounds__(kBlock, 4) k_bstage(const __grid_constant__ StageParams<typename KD<K>::TB> P,
                                                      const int *__restrict__ sel) {
  using D = KD<K>;
  using TB = typename D::TB;
  for (int i = 0; i < P.count; ++i) {
    if (!sel[P.sys[i]]) continue;
    row_dispatch<TB, TB, D::NEG, D::EPI, D::WIDE>(P.nv[i], P.opt[i], P.op[i]);
    // the dot epilogues reuse the block's shared reduction buffers
    if constexpr (epi_has_dot<D::EPI>()) __syncthreads();
  }
}

// Launches kernel K with the parameter block `params` (a StageParams of the
// kernel's block scalar); grid <= 0 returns the persistent grid bound.
template <int K>
int bk_launch_t(const void *params, const int *sel, int grid, cudaStream_t st) {
  static int max_grid = 0;
  if (!max_grid) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bstage<K>, kBlock, 0) != cudaSuccess || b < 1) b = 1;
    max_grid = std::min(kMaxGrid, b * device_sm_count());
  }
  if (grid <= 0) return max_grid;
  grid = std::min(grid, max_grid);
  k_bstage<K><<<grid, kBlock, 0, st>>>(*static_cast<const StageParams<typename KD<K>::TB> *>(params), sel);
  g_launches++;
  return cudaPeekAtLastError() == cudaSuccess ? grid : -1;
}

}  // namespace xamg
