// vtail_kern.cuh -- device code and launcher of the cooperative coarse-tail
// kernel (vtail.cuh), instantiated per block scalar by vtail_f64.cu and
// vtail_f32.cu.  Internal to the library.
#pragma once
#include <algorithm>
#include <type_traits>

#include "elem.cuh"
#include "vtail.cuh"

namespace xamg {

__device__ __forceinline__ unsigned long long tail_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of the cooperative tail launch.  Thread 0 of each block
// arrives on the counter; the last of `expected` arrivals resets it and
// advances the generation word, on which the others wait.  Every wait is
// bounded: after limit_ns (or as soon as another block has given up) the
// block records the failure (sync->err, and *err_host for the host) and
// returns false, and the kernel returns; nothing else is in flight at that
// point (the row bodies issue only plain loads and stores).
__device__ __forceinline__ bool tail_barrier(TailSync *sync, unsigned int expected,
                                             unsigned long long limit_ns, int32_t *err_host) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int *gen = &sync->gen;
    volatile int *err = &sync->err;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(&sync->count, 1u) + 1u == expected) {
      atomicExch(&sync->count, 0u);
      __threadfence();
      atomicAdd(&sync->gen, 1u);
    } else {
      const unsigned long long t0 = tail_clock_ns();
      while (*gen == g) {
        if (*err) {
          ok = 0;
          break;
        }
        if (tail_clock_ns() - t0 > limit_ns) {
          ok = 0;
          atomicExch(&sync->err, 1);
          if (err_host) *(volatile int32_t *)err_host = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// One stage's row body: the split, sign and epilogue of its single-launch
// counterpart (k_rows with slices 1, or the wide split), reading the operand
// block through the coherent path.
template <class TB, class TVA, int NV, int KIND, bool WIDE>
__device__ __forceinline__ void tail_rows(const RowOpT<TB> &op) {
  constexpr int VEC = row_vec<TB, NV>();
  constexpr int G = NV / VEC;
  constexpr bool isA = KIND <= TK_A_XLAST;
  using TV = typename std::conditional<isA, TVA, TB>::type;
  constexpr bool NEG = isA;
  constexpr int EPI = KIND == TK_A_YDN    ? EPI_Y_DN
                      : KIND == TK_A_YXDP ? EPI_Y_XDP
                      : KIND == TK_A_YD0  ? EPI_Y_D0
                      : KIND == TK_A_XLAST ? EPI_XLAST
                      : KIND == TK_PR_Y   ? EPI_Y
                                          : EPI_Y_D0;
  if constexpr (!WIDE) {
    rows_vec<TB, TV, NV, VEC, 1, NEG, EPI, 1, true>(op);
  } else if constexpr (sizeof(TB) == 8 && NV >= 16) {
    rows_vec<TB, TV, NV, VEC, 32 / G, NEG, EPI, kWarpsPerRow, true>(op);
  } else {
    rows_vec<TB, TV, NV, VEC, 32 / G, NEG, EPI, 1, true>(op);
  }
}

template <class TB, class TVA, int NV>
__device__ __forceinline__ void tail_stage(const TailStage<TB> &t) {
  switch (t.kind * 2 + t.wide) {
    case TK_A_YDN * 2: tail_rows<TB, TVA, NV, TK_A_YDN, false>(t.op); break;
    case TK_A_YDN * 2 + 1: tail_rows<TB, TVA, NV, TK_A_YDN, true>(t.op); break;
    case TK_A_YXDP * 2: tail_rows<TB, TVA, NV, TK_A_YXDP, false>(t.op); break;
    case TK_A_YXDP * 2 + 1: tail_rows<TB, TVA, NV, TK_A_YXDP, true>(t.op); break;
    case TK_A_YD0 * 2: tail_rows<TB, TVA, NV, TK_A_YD0, false>(t.op); break;
    case TK_A_YD0 * 2 + 1: tail_rows<TB, TVA, NV, TK_A_YD0, true>(t.op); break;
    case TK_A_XLAST * 2: tail_rows<TB, TVA, NV, TK_A_XLAST, false>(t.op); break;
    case TK_A_XLAST * 2 + 1: tail_rows<TB, TVA, NV, TK_A_XLAST, true>(t.op); break;
    case TK_PR_Y * 2: tail_rows<TB, TVA, NV, TK_PR_Y, false>(t.op); break;
    case TK_PR_Y * 2 + 1: tail_rows<TB, TVA, NV, TK_PR_Y, true>(t.op); break;
    case TK_PR_YD0 * 2: tail_rows<TB, TVA, NV, TK_PR_YD0, false>(t.op); break;
    case TK_PR_YD0 * 2 + 1: tail_rows<TB, TVA, NV, TK_PR_YD0, true>(t.op); break;
    default:
      if (t.kind == TK_COARSE && blockIdx.x == 0)
        d_coarse_mma<NV, TB, TB>(t.op.n, static_cast<const double *>(t.op.val), t.op.src, t.op.y);
      break;
  }
}

// The tail program: its stages in order, a grid barrier between two stages.
template <class TB, class TVA, int NV>
__global__ void __launch_bounds__(kBlock, 2) k_vtail(const __grid_constant__ TailProg<TB> p) {
  const unsigned int expected = gridDim.x + (unsigned int)p.extra;
  for (int s = 0; s < p.nstages; ++s) {
    tail_stage<TB, TVA, NV>(p.st[s]);
    if (s + 1 < p.nstages && !tail_barrier(p.sync, expected, p.limit_ns, p.err_host)) return;
  }
}

// Cooperative launch with every block resident: the grid is the kernel's
// occupancy times the SM count (at most kMaxGrid).
template <class TB, class TVA, int NV>
int vtail_launch(const TailProg<TB> &p, cudaStream_t st) {
  auto kern = k_vtail<TB, TVA, NV>;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kBlock, 0) != cudaSuccess || b < 1) return -1;
  const int grid = std::min(kMaxGrid, b * device_sm_count());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, p);
  g_launches++;
  return e == cudaSuccess ? grid : -1;
}

}  // namespace xamg
