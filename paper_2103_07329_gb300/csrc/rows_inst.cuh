// rows_inst.cuh -- instantiations and launcher of the fused row kernel for one
// block width NV (XAMG_NV) and one block scalar (XAMG_FLOAT: float blocks with
// float or bf16 values; otherwise double blocks and values).  Included by the
// rows_nv*.cu / rowsf_nv*.cu units so that the variants compile in parallel.
#include <algorithm>

#include "launch.h"

#ifndef XAMG_NV
#error "define XAMG_NV before including rows_inst.cuh"
#endif

namespace xamg {
namespace {

#if XAMG_FLOAT
using TBx = float;
#else
using TBx = double;
#endif

// S < 0: an m = 1 stream-kernel variant (StreamCfg<S>).
template <class TV, int NV, int S, bool NEG, int EPI>
int rows_t(const RowOpT<TBx> &op, cudaStream_t st) {
  if constexpr (S == kStreamV256 || S == kStreamV1024) {
    constexpr int R = S == kStreamV256 ? 256 : 1024;
    constexpr int smem = kWarps * stream_warp_bytes<TV, R>();
    auto kern = k_rows_stream_v<TBx, TV, NV, R, NEG, EPI>;
    static int max_grid = 0;
    if (!max_grid) {
      int b = 0;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kBlock, smem) != cudaSuccess || b < 1)
        b = 1;
      max_grid = std::min(kMaxGrid, b * device_sm_count());
    }
    constexpr int rows_per_block = kWarps * 32;
    const int64_t need = ((int64_t)op.n + rows_per_block - 1) / rows_per_block;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, max_grid));
    kern<<<grid, kBlock, smem, st>>>(op);
    g_launches++;
    return cudaPeekAtLastError() == cudaSuccess ? grid : -1;
  } else if constexpr (S == kAsyncNarrow) {
    constexpr int smem = kWarps * async_warp_bytes<TV, NV>();
    auto kern = k_rows_async<TBx, TV, NV, NEG, EPI>;
    static int max_grid = 0;
    if (!max_grid) {
      int b = 0;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kBlock, smem) != cudaSuccess || b < 1)
        b = 1;
      max_grid = std::min(kMaxGrid, b * device_sm_count());
    }
    constexpr int rows_per_block = kWarps * async_rows_per_warp<NV>();
    const int64_t need = ((int64_t)op.n + rows_per_block - 1) / rows_per_block;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, max_grid));
    kern<<<grid, kBlock, smem, st>>>(op);
    g_launches++;
    return cudaPeekAtLastError() == cudaSuccess ? grid : -1;
  } else if constexpr (S < 0 && NV == 1) {
    constexpr int LPR = StreamCfg<S>::LPR, R = StreamCfg<S>::R;
    constexpr int smem = kWarps * stream_warp_bytes<TV, R>();
    auto kern = k_rows_stream<TBx, TV, LPR, R, NEG, EPI>;
    static int max_grid = 0;
    if (!max_grid) {
      int b = 0;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kBlock, smem) != cudaSuccess || b < 1)
        b = 1;
      max_grid = std::min(kMaxGrid, b * device_sm_count());
    }
    constexpr int rows_per_block = kWarps * (32 / LPR);
    const int64_t need = ((int64_t)op.n + rows_per_block - 1) / rows_per_block;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, max_grid));
    kern<<<grid, kBlock, smem, st>>>(op);
    g_launches++;
    return cudaPeekAtLastError() == cudaSuccess ? grid : -1;
  } else {
    static int max_grid = 0;
    if (!max_grid) {
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_rows<TBx, TV, NV, S, NEG, EPI>, kBlock,
                                                        0) != cudaSuccess ||
          b < 1)
        b = 1;
      max_grid = std::min(kMaxGrid, b * device_sm_count());
    }
    // S < 0 (NV > 1): -S warps per row; kPipeNarrow, kNarrow2, kPipeNarrow2:
    // the narrow split (with split_vec columns per lane)
    constexpr int SS = (S == kPipeNarrow || S == kNarrow2 || S == kPipeNarrow2) ? 1 : S;
    constexpr int lanes_per_row = NV == 1 ? SS : (NV / split_vec<TBx, NV, S>()) * (SS > 0 ? SS : 1);
    constexpr int rows_per_block = SS < 0 ? kWarps / -SS : kWarps * (32 / lanes_per_row);
    const int64_t need = ((int64_t)op.n + rows_per_block - 1) / rows_per_block;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, max_grid));
    k_rows<TBx, TV, NV, S, NEG, EPI><<<grid, kBlock, 0, st>>>(op);
    g_launches++;
    return cudaPeekAtLastError() == cudaSuccess ? grid : -1;
  }
}

// The (sign, epilogue) pairs the solver uses.
template <class TV, int NV, int S>
int rows_e(const RowOpT<TBx> &op, bool neg, int epi, cudaStream_t st) {
  if (neg) {
    switch (epi) {
      case EPI_Y: return rows_t<TV, NV, S, true, EPI_Y>(op, st);
      case EPI_Y_D0: return rows_t<TV, NV, S, true, EPI_Y_D0>(op, st);
      case EPI_Y_DN: return rows_t<TV, NV, S, true, EPI_Y_DN>(op, st);
      case EPI_Y_XDP: return rows_t<TV, NV, S, true, EPI_Y_XDP>(op, st);
      case EPI_MID: return rows_t<TV, NV, S, true, EPI_MID>(op, st);
      case EPI_XLAST: return rows_t<TV, NV, S, true, EPI_XLAST>(op, st);
      case EPI_XLAST_DOT: return rows_t<TV, NV, S, true, EPI_XLAST_DOT>(op, st);
#if XAMG_FLOAT
      case EPI_XLAST_DOT2: return rows_t<TV, NV, S, true, EPI_XLAST_DOT2>(op, st);
#else
      case EPI_Y_DOT2: return rows_t<TV, NV, S, true, EPI_Y_DOT2>(op, st);
#endif
      default: return -1;
    }
  }
  switch (epi) {
    case EPI_Y: return rows_t<TV, NV, S, false, EPI_Y>(op, st);
    case EPI_Y_D0: return rows_t<TV, NV, S, false, EPI_Y_D0>(op, st);
#if !XAMG_FLOAT
    case EPI_Y_DOT: return rows_t<TV, NV, S, false, EPI_Y_DOT>(op, st);
    case EPI_Y_DOT2: return rows_t<TV, NV, S, false, EPI_Y_DOT2>(op, st);
#endif
    default: return -1;
  }
}

// m = 1 takes the stream kernel (short or long window) or 16 lanes per row;
// wider blocks give each lane VEC columns and may split long rows over the
// whole warp (slices: one row per warp).
template <class TV>
int rows_any(const RowOpT<TBx> &op, int slices, bool neg, int epi, cudaStream_t st) {
#if XAMG_NV == 1
  if constexpr (ValueLoad<TV>::idx16) {
    // 16-bit indices are a wide-block format; m = 1 reads the 32-bit ones
    (void)op; (void)slices; (void)neg; (void)epi; (void)st;
    return -1;
  } else {
    switch (slices) {
      case kStreamShort: return rows_e<TV, 1, kStreamShort>(op, neg, epi, st);
      case kStreamLong: return rows_e<TV, 1, kStreamLong>(op, neg, epi, st);
      case kStreamQuad: return rows_e<TV, 1, kStreamQuad>(op, neg, epi, st);
      case kStreamWarp: return rows_e<TV, 1, kStreamWarp>(op, neg, epi, st);
      case kStreamMid: return rows_e<TV, 1, kStreamMid>(op, neg, epi, st);
      case kStreamPair: return rows_e<TV, 1, kStreamPair>(op, neg, epi, st);
      default: return rows_e<TV, 1, kSliced16>(op, neg, epi, st);
    }
  }
#else
#if XAMG_NV == 2 || XAMG_NV == 4
  // one lane per row over the warp's staged entries (8- to 32-byte block rows)
  if constexpr (!ValueLoad<TV>::idx16) {
    if (slices == kStreamV256) return rows_e<TV, XAMG_NV, kStreamV256>(op, neg, epi, st);
    if (slices == kStreamV1024) return rows_e<TV, XAMG_NV, kStreamV1024>(op, neg, epi, st);
  }
#endif
  if (slices == kStreamV256 || slices == kStreamV1024) slices = 1;
#if XAMG_FLOAT && XAMG_NV >= 8
  // the narrow split with operand rows staged through shared memory
  if constexpr (!ValueLoad<TV>::idx16) {
    if (slices == kAsyncNarrow) return rows_e<TV, XAMG_NV, kAsyncNarrow>(op, neg, epi, st);
  }
#endif
  if (slices == kAsyncNarrow) slices = 1;
#if !XAMG_FLOAT && XAMG_NV >= 8
  // the narrow split with its row loop software-pipelined, and both with two
  // columns per lane
  if (slices == kPipeNarrow) return rows_e<TV, XAMG_NV, kPipeNarrow>(op, neg, epi, st);
  if (slices == kNarrow2) return rows_e<TV, XAMG_NV, kNarrow2>(op, neg, epi, st);
  if (slices == kPipeNarrow2) return rows_e<TV, XAMG_NV, kPipeNarrow2>(op, neg, epi, st);
#endif
  if (slices == kPipeNarrow || slices == kNarrow2 || slices == kPipeNarrow2) slices = 1;
  // long rows: every group of the warp takes a slice of one row (one row per
  // warp; with 32 FP64 columns a row already fills the warp)
  constexpr int WS = 32 / (XAMG_NV / row_vec<TBx, XAMG_NV>());
  if constexpr (WS > 1) {
#if !XAMG_FLOAT && XAMG_NV == 16
    // 16 FP64 columns: the row's two slices in each of kWarpsPerRow warps
    if (slices > 1) return rows_e<TV, XAMG_NV, -kWarpsPerRow>(op, neg, epi, st);
#endif
    if (slices > 1) return rows_e<TV, XAMG_NV, WS>(op, neg, epi, st);
  } else {
    // a row already fills the warp: the wide split gives it kWarpsPerRow warps
    if (slices > 1) return rows_e<TV, XAMG_NV, -kWarpsPerRow>(op, neg, epi, st);
  }
  return rows_e<TV, XAMG_NV, 1>(op, neg, epi, st);
#endif
}

}  // namespace

#define XAMG_CAT2(a, b) a##b
#define XAMG_CAT(a, b) XAMG_CAT2(a, b)

#if XAMG_FLOAT
// vt: 0 = float values, 1 = bf16 values with per-row scale, 2 = the same with
// 16-bit column indices, 3 = float values with 16-bit column indices
int XAMG_CAT(launch_rowsf_nv, XAMG_NV)(const RowOpF &op, int slices, bool neg, int epi, int vt,
                                        cudaStream_t st) {
  if (vt == 3) return rows_any<F32Idx16>(op, slices, neg, epi, st);
  if (vt == 2) return rows_any<Bf16Idx16>(op, slices, neg, epi, st);
  return vt == 1 ? rows_any<__nv_bfloat16>(op, slices, neg, epi, st)
                 : rows_any<float>(op, slices, neg, epi, st);
}
#else
int XAMG_CAT(launch_rows_nv, XAMG_NV)(const RowOp &op, int slices, bool neg, int epi,
                                       cudaStream_t st) {
  return rows_any<double>(op, slices, neg, epi, st);
}
#endif

}  // namespace xamg
