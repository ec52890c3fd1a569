// rows_inst.cuh -- instantiations and launcher of the fused row kernel for one
// NV (XAMG_NV), included by rows_nv*.cu so that the NVs compile in parallel.
#include <algorithm>

#include "launch.h"

#ifndef XAMG_NV
#error "define XAMG_NV before including rows_inst.cuh"
#endif

namespace xamg {
namespace {

template <int NV, int S, bool NEG, int EPI>
int rows_t(const RowOp &op, cudaStream_t st) {
  static int max_grid = 0;
  if (!max_grid) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_rows<NV, S, NEG, EPI>, kBlock, 0) !=
            cudaSuccess ||
        b < 1)
      b = 1;
    max_grid = std::min(kMaxGrid, b * device_sm_count());
  }
  constexpr int rows_per_block = kWarps * (32 / (NV * S));
  const int64_t need = ((int64_t)op.n + rows_per_block - 1) / rows_per_block;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, max_grid));
  k_rows<NV, S, NEG, EPI><<<grid, kBlock, 0, st>>>(op);
  g_launches++;
  return cudaPeekAtLastError() == cudaSuccess ? grid : -1;
}

// The (sign, epilogue) pairs the solver uses.
template <int NV, int S>
int rows_e(const RowOp &op, bool neg, int epi, cudaStream_t st) {
  if (neg) {
    switch (epi) {
      case EPI_Y: return rows_t<NV, S, true, EPI_Y>(op, st);
      case EPI_Y_D0: return rows_t<NV, S, true, EPI_Y_D0>(op, st);
      case EPI_Y_DN: return rows_t<NV, S, true, EPI_Y_DN>(op, st);
      case EPI_Y_XDP: return rows_t<NV, S, true, EPI_Y_XDP>(op, st);
      case EPI_MID: return rows_t<NV, S, true, EPI_MID>(op, st);
      case EPI_XLAST: return rows_t<NV, S, true, EPI_XLAST>(op, st);
      case EPI_XLAST_DOT: return rows_t<NV, S, true, EPI_XLAST_DOT>(op, st);
      case EPI_Y_DOT2: return rows_t<NV, S, true, EPI_Y_DOT2>(op, st);
      default: return -1;
    }
  }
  switch (epi) {
    case EPI_Y: return rows_t<NV, S, false, EPI_Y>(op, st);
    case EPI_Y_D0: return rows_t<NV, S, false, EPI_Y_D0>(op, st);
    case EPI_Y_DOT: return rows_t<NV, S, false, EPI_Y_DOT>(op, st);
    case EPI_Y_DOT2: return rows_t<NV, S, false, EPI_Y_DOT2>(op, st);
    default: return -1;
  }
}

}  // namespace

#define XAMG_CAT2(a, b) a##b
#define XAMG_CAT(a, b) XAMG_CAT2(a, b)

// m = 1 splits rows over 4 or 16 lanes; wider blocks use one lane per column.
int XAMG_CAT(launch_rows_nv, XAMG_NV)(const RowOp &op, int slices, bool neg, int epi,
                                       cudaStream_t st) {
#if XAMG_NV == 1
  if (slices >= 16) return rows_e<1, 16>(op, neg, epi, st);
  return rows_e<1, 4>(op, neg, epi, st);
#else
  (void)slices;
  return rows_e<XAMG_NV, 1>(op, neg, epi, st);
#endif
}

}  // namespace xamg
