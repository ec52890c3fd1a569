// batch_stage.cuh -- the batched row stages: one persistent launch applies
// one step of the V-cycle (or of the Krylov loop) to every selected system.
// Blocks walk the systems in order; within a system the warps take the rows
// in the same grid-stride order as the single-system row kernel (rows_vec /
// rows_sliced of kernels.cuh), so each system's products and partial dot
// sums are computed exactly as a single-system launch with the same grid
// would compute them.  The column count NV and the row split of every
// system's operator are runtime values: a switch selects the compile-time
// body.  Included by batch_stage*.cu (one group of stages per unit).
#pragma once
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

// WIDE: whether the wide split is compiled for this stage (the stages that
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

template <class TB>
__device__ __forceinline__ RowOpT<TB> blank_op() {
  RowOpT<TB> o;
  o.n = 0;
  o.rowptr = nullptr;
  o.col = nullptr;
  o.val = nullptr;
  o.rscale = nullptr;
  o.colw = nullptr;
  o.rowmeta = nullptr;
  o.src = nullptr;
  o.init = nullptr;
  o.y = nullptr;
  o.dp = nullptr;
  o.w = nullptr;
  o.c1 = 0;
  o.dnext = nullptr;
  o.x = nullptr;
  o.dot_u = nullptr;
  o.dot_u2 = nullptr;
  o.partials = nullptr;
  o.partials2 = nullptr;
  return o;
}

// Stage definitions: block scalar, sign, epilogue; whether it applies to
// system S at level l; the operation; the operator's row split.
template <int ST>
struct SD;

__device__ __forceinline__ void op_A(RowOpT<float> &o, const BLevel &V) {
  o.n = V.n;
  o.rowptr = V.Arp;
  o.col = V.Aci;
  o.val = V.Av;
}

template <>
struct SD<BS_PRE1> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = true;
  static constexpr int EPI = EPI_Y_DN;
  __device__ static bool on(const BSys &S, int l) { return l < S.L - 1; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optA; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l];
    RowOpT<float> o = blank_op<float>();
    op_A(o, V);
    o.init = V.b; o.src = V.x; o.y = V.r; o.dp = V.x; o.w = V.w[1]; o.c1 = V.c1[1]; o.dnext = V.d;
    return o;
  }
};
template <>
struct SD<BS_PRE2> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = true;
  static constexpr int EPI = EPI_Y_XDP;
  __device__ static bool on(const BSys &S, int l) { return l < S.L - 1; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optA; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l];
    RowOpT<float> o = blank_op<float>();
    op_A(o, V);
    o.init = V.r; o.src = V.d; o.y = V.r; o.dp = V.d; o.x = V.x;
    return o;
  }
};
template <>
struct SD<BS_RESTRICT> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = false;
  static constexpr int EPI = EPI_Y_D0;
  __device__ static bool on(const BSys &S, int l) { return l + 2 < S.L; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optR; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l], &C = S.lv[l + 1];
    RowOpT<float> o = blank_op<float>();
    o.n = V.nc; o.rowptr = V.Rrp; o.col = V.Rci; o.val = V.Rv;
    o.src = V.r; o.y = C.b; o.w = C.w[0]; o.dnext = C.x;
    return o;
  }
};
template <>
struct SD<BS_RESTRICT_C> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = false;
  static constexpr int EPI = EPI_Y;
  __device__ static bool on(const BSys &S, int l) { return l + 2 == S.L; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optR; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l], &C = S.lv[l + 1];
    RowOpT<float> o = blank_op<float>();
    o.n = V.nc; o.rowptr = V.Rrp; o.col = V.Rci; o.val = V.Rv;
    o.src = V.r; o.y = C.b;
    return o;
  }
};
template <>
struct SD<BS_PROLONG> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = false;
  static constexpr int EPI = EPI_Y;
  __device__ static bool on(const BSys &S, int l) { return l < S.L - 1; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optP; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l], &C = S.lv[l + 1];
    RowOpT<float> o = blank_op<float>();
    o.n = V.n; o.rowptr = V.Prp; o.col = V.Pci; o.val = V.Pv;
    o.init = V.x; o.src = C.x; o.y = V.x;
    return o;
  }
};
template <>
struct SD<BS_POST1> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = true;
  static constexpr int EPI = EPI_Y_D0;
  __device__ static bool on(const BSys &S, int l) { return l < S.L - 1; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optA; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l];
    RowOpT<float> o = blank_op<float>();
    op_A(o, V);
    o.init = V.b; o.src = V.x; o.y = V.r; o.w = V.w[0]; o.dnext = V.d;
    return o;
  }
};
template <>
struct SD<BS_POST2> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = true;
  static constexpr int EPI = EPI_XLAST;
  __device__ static bool on(const BSys &S, int l) { return l < S.L - 1; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optA; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l];
    RowOpT<float> o = blank_op<float>();
    op_A(o, V);
    o.init = V.r; o.src = V.d; o.dp = V.d; o.w = V.w[1]; o.c1 = V.c1[1]; o.x = V.x;
    return o;
  }
};
template <>
struct SD<BS_POST2_DOT2> {
  using TB = float;
  static constexpr bool WIDE = false;
  static constexpr bool NEG = true;
  static constexpr int EPI = EPI_XLAST_DOT2;
  __device__ static bool on(const BSys &S, int l) { return l < S.L - 1; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optA; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    RowOpT<float> o = SD<BS_POST2>::make(S, l);
    o.dot_u = S.R; o.partials = S.part[1];
    o.dot_u2 = S.Q; o.partials2 = S.part[2];
    return o;
  }
};
template <>
struct SD<BS_AP> {
  using TB = double;
  static constexpr bool WIDE = false;
  static constexpr bool NEG = false;
  static constexpr int EPI = EPI_Y_DOT;
  __device__ static bool on(const BSys &, int) { return true; }
  __device__ static int opt(const BSys &S, const BLevel &) { return S.optA0; }
  __device__ static RowOpT<double> make(const BSys &S, int) {
    RowOpT<double> o = blank_op<double>();
    o.n = (int)S.n0; o.rowptr = S.A0rp; o.col = S.A0ci; o.val = S.A0v;
    o.src = S.P; o.y = S.Q; o.dot_u = S.P; o.partials = S.part[0];
    return o;
  }
};
template <>
struct SD<BS_TRUERES> {
  using TB = double;
  static constexpr bool WIDE = false;
  static constexpr bool NEG = true;
  static constexpr int EPI = EPI_Y_DOT2;
  __device__ static bool on(const BSys &, int) { return true; }
  __device__ static int opt(const BSys &S, const BLevel &) { return S.optA0; }
  __device__ static RowOpT<double> make(const BSys &S, int) {
    RowOpT<double> o = blank_op<double>();
    o.n = (int)S.n0; o.rowptr = S.A0rp; o.col = S.A0ci; o.val = S.A0v;
    o.init = S.Bn; o.src = S.X; o.y = S.Q; o.partials2 = S.part[2];
    return o;
  }
};
template <>
struct SD<BS_TUNE_A> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = false;
  static constexpr int EPI = EPI_Y;
  __device__ static bool on(const BSys &S, int l) { return l < S.L - 1; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optA; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l];
    RowOpT<float> o = blank_op<float>();
    op_A(o, V);
    o.src = V.x; o.y = V.r;
    return o;
  }
};
template <>
struct SD<BS_TUNE_P> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = false;
  static constexpr int EPI = EPI_Y;
  __device__ static bool on(const BSys &S, int l) { return l < S.L - 1; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optP; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l], &C = S.lv[l + 1];
    RowOpT<float> o = blank_op<float>();
    o.n = V.n; o.rowptr = V.Prp; o.col = V.Pci; o.val = V.Pv;
    o.src = C.x; o.y = V.r;
    return o;
  }
};
template <>
struct SD<BS_TUNE_R> {
  using TB = float;
  static constexpr bool WIDE = true;
  static constexpr bool NEG = false;
  static constexpr int EPI = EPI_Y;
  __device__ static bool on(const BSys &S, int l) { return l < S.L - 1; }
  __device__ static int opt(const BSys &, const BLevel &V) { return V.optR; }
  __device__ static RowOpT<float> make(const BSys &S, int l) {
    const BLevel &V = S.lv[l], &C = S.lv[l + 1];
    RowOpT<float> o = blank_op<float>();
    o.n = V.nc; o.rowptr = V.Rrp; o.col = V.Rci; o.val = V.Rv;
    o.src = V.r; o.y = C.b;
    return o;
  }
};

// One launch of stage ST on level `level` for every system s with sel[s]:
// blocks take the systems in order and, inside one, the rows in the
// single-system grid-stride order.
template <int ST>
__global__ void __launch_bounds__(kBlock, 3) k_bstage(const BSys *__restrict__ sys, int ns,
                                                      const int *__restrict__ sel, int level) {
  using D = SD<ST>;
  using TB = typename D::TB;
  for (int s = 0; s < ns; ++s) {
    if (!sel[s]) continue;
    const BSys &S = sys[s];
    if (!D::on(S, level)) continue;
    const RowOpT<TB> op = D::make(S, level);
    const int opt = D::opt(S, S.lv[level]);
    row_dispatch<TB, TB, D::NEG, D::EPI, D::WIDE>(S.nv, opt, op);
    // the dot epilogues reuse the block's shared reduction buffers
    if constexpr (epi_has_dot<D::EPI>()) __syncthreads();
  }
}

template <int ST>
int bstage_launch_t(const BSys *sys, int ns, const int *sel, int level, int grid, cudaStream_t st) {
  static int max_grid = 0;
  if (!max_grid) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bstage<ST>, kBlock, 0) != cudaSuccess || b < 1) b = 1;
    max_grid = std::min(kMaxGrid, b * device_sm_count());
  }
  if (grid <= 0) return max_grid;  // query
  grid = std::min(grid, max_grid);
  k_bstage<ST><<<grid, kBlock, 0, st>>>(sys, ns, sel, level);
  g_launches++;
  return cudaPeekAtLastError() == cudaSuccess ? grid : -1;
}

}  // namespace xamg
