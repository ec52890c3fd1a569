// batch_stage.cuh -- the batched row stages: one persistent launch applies
// one step of the V-cycle (or of the Krylov loop) to a list of systems.  The
// host builds each system's row operation (as for a single-system launch) and
// passes the whole list as one kernel parameter block, so every field is read
// from the constant bank where it is used, as in the single-system kernel.
// Blocks walk the list in order; within a system the warps take the rows in
// the single-system grid-stride order (rows_vec / rows_sliced of
// kernels.cuh), so each system's products and partial dot sums are computed
// exactly as a single-system launch with the same grid computes them.  A
// launch serves the systems of one block width NV and one row split, both
// compile-time parameters of the kernel.  Included by batch.cu and
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

// Entries per launch: the parameter block stays below the 32 KB limit of
// kernel parameters.
constexpr int kStageOps = 96;

template <class TB>
struct StageParams {
  int count;
  int sys[kStageOps];              // system index (selection mask)
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

// One launch: every listed system of block width NV under row split WIDE
// (both compile-time, so that each kernel holds one body and its registers).
template <int K, int NV, bool WIDE>
__global__ void __launch_bounds__(kBlock, 4) k_bstage(const __grid_constant__ StageParams<typename KD<K>::TB> P,
                                                      const int *__restrict__ sel) {
  using D = KD<K>;
  using TB = typename D::TB;
  constexpr int S = WIDE ? wide_s<TB, NV>() : narrow_s<TB, NV>();
  for (int i = 0; i < P.count; ++i) {
    if (!sel[P.sys[i]]) continue;
    row_body<TB, TB, NV, S, D::NEG, D::EPI>(P.op[i]);
    // the dot epilogues reuse the block's shared reduction buffers
    if constexpr (epi_has_dot<D::EPI>()) __syncthreads();
  }
}

template <int K, int NV, bool WIDE>
int bk_launch_nv(const void *params, const int *sel, int grid, cudaStream_t st) {
  static int max_grid = 0;
  if (!max_grid) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bstage<K, NV, WIDE>, kBlock, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    max_grid = std::min(kMaxGrid, b * device_sm_count());
  }
  if (grid <= 0) return max_grid;
  grid = std::min(grid, max_grid);
  k_bstage<K, NV, WIDE><<<grid, kBlock, 0, st>>>(*static_cast<const StageParams<typename KD<K>::TB> *>(params),
                                                  sel);
  g_launches++;
  return cudaPeekAtLastError() == cudaSuccess ? grid : -1;
}

template <int K, int NV>
int bk_launch_split(int opt, const void *params, const int *sel, int grid, cudaStream_t st) {
  if constexpr (KD<K>::WIDE) {
    if (opt) return bk_launch_nv<K, NV, true>(params, sel, grid, st);
  }
  return bk_launch_nv<K, NV, false>(params, sel, grid, st);
}

template <int K, int NV>
int bk_bound(int g) {
  g = std::min(g, bk_launch_nv<K, NV, false>(nullptr, nullptr, 0, nullptr));
  if constexpr (KD<K>::WIDE) g = std::min(g, bk_launch_nv<K, NV, true>(nullptr, nullptr, 0, nullptr));
  return g;
}

// Launches kernel K for block width nv and row split opt (0 narrow, 1 wide;
// kernels without the wide split take the narrow one) with the parameter
// block `params` (a StageParams of the kernel's block scalar).  grid <= 0
// returns the persistent grid bound of that kernel; nv = 0 returns the
// smallest bound over every width and split (the dot stages' partial arrays
// have that many rows whatever the width).
template <int K>
int bk_launch_t(int nv, int opt, const void *params, const int *sel, int grid, cudaStream_t st) {
  switch (nv) {
    case 1: return bk_launch_split<K, 1>(opt, params, sel, grid, st);
    case 2: return bk_launch_split<K, 2>(opt, params, sel, grid, st);
    case 4: return bk_launch_split<K, 4>(opt, params, sel, grid, st);
    case 8: return bk_launch_split<K, 8>(opt, params, sel, grid, st);
    case 16: return bk_launch_split<K, 16>(opt, params, sel, grid, st);
    case 32: return bk_launch_split<K, 32>(opt, params, sel, grid, st);
    case 0: {
      int g = kMaxGrid;
      g = bk_bound<K, 1>(g);
      g = bk_bound<K, 2>(g);
      g = bk_bound<K, 4>(g);
      g = bk_bound<K, 8>(g);
      g = bk_bound<K, 16>(g);
      return bk_bound<K, 32>(g);
    }
    default: return -1;
  }
}

}  // namespace xamg
