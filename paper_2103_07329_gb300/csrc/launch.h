// launch.h -- host-side launchers of the solve-phase kernels (runtime NV
// dispatch onto the compile-time NV kernels of kernels.cu).  Internal.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "kernels.cuh"

namespace xamg {

constexpr int kMaxGrid = 4096;  // upper bound on blocks of any reducing launch

// Per-column solver state on the device (NV <= 32 columns are used).
struct ColState {
  double nb[32];       // ||b_j||
  double rho[32];      // PCG: r.z ; BiCGStab: rhat.r of the last iteration
  double alpha[32];
  double beta[32];
  double omega[32];
  double tn[32];       // true residual norms
  double rho_old[32];  // reordered BiCGStab: rho of the previous iteration
  int32_t state[32];   // 0 active, 1 frozen by the residual test, 2 confirmed,
                       // 3 breakdown, 4 zero right-hand side
  int32_t restart[32]; // next direction update starts afresh
  int32_t iters[32];
  int32_t reac[32];    // 1: column restarted by the last confirmation
  int32_t kdev;        // iteration number of the last alpha step (graph replays read it)
};

// Host-visible counters written by the scalar kernels (mapped pinned memory).
struct Flags {
  int32_t active;       // columns still iterating
  int32_t frozen;       // columns frozen by the recursive residual test
  int32_t reactivated;  // columns restarted by the last confirmation
  int32_t breakdown;
  int32_t tail_err;     // 1: a grid-barrier wait of the fused coarse tail ran out
};

enum ScalarMode : int {
  SM_INIT = 0,       // p0: ||b||^2 partials -> nb, state, restart = 1
  SM_PCG_ALPHA = 1,  // p0: p.q -> alpha, iters = k
  SM_PCG_CONV = 2,   // p0: r.r -> freeze
  SM_PCG_BETA = 3,   // p0: r.z -> beta, rho
  SM_CONFIRM = 4,    // p0: true residual^2 -> confirm or restart
  SM_FINAL = 5,      // p0: true residual^2 -> tn
  SM_BI_RHO = 6,     // p0: rhat.r -> beta, rho
  SM_BI_ALPHA = 7,   // p0: rhat.v -> alpha
  SM_BI_HALF = 8,    // p0: s.s -> iters = k, half-step freeze
  SM_BI_OMEGA = 9,   // p0: t.s, p1: t.t -> omega
  SM_BI_CONV = 10,   // p0: r.r -> freeze
  SM_FPCG_BETA = 11, // p0: r.z, p1: q.z -> flexible beta, rho
};

// Scalar steps of the BiCGStab variants (k_vscalar): the partial-sum arrays
// and their block counts.
enum VScalarMode : int {
  VS_RHO0 = 0,     // p0: rhat.r -> rho of every column that starts afresh
  VS_RB_BETA = 1,  // reordered: beta of the direction update
  VS_RB_OMEGA = 2, // reordered: p0 t.s, p1 t.t, p2 s.s -> omega, iters, freeze
  VS_RB_RHO = 3,   // reordered: p0 rhat.s, p1 rhat.t -> rho' = rhat.s - omega rhat.t
  VS_PB_INIT = 4,  // pipelined: p0 rhat.r, p1 rhat.w -> rho, alpha (fresh columns)
  VS_PB_OMEGA = 5, // pipelined: p0 q.y, p1 y.y -> omega, iters
  VS_PB_ALPHA = 6, // pipelined: p0..p4 rhat.r, rhat.w, rhat.s, rhat.z, r.r -> freeze, beta, rho, alpha
};
struct VParts {
  const double *p[5];
  int nblk[5];
};

// Row splits at m = 1 (the `slices` argument of the row launchers at nv = 1):
// the stream kernel with lanes per row / window entries per warp of 1 / 256
// (kStreamShort), 1 / 512 (kStreamMid), 2 / 512 (kStreamPair), 1 / 1024
// (kStreamLong), 4 / 1024 (kStreamQuad) or 32 / 1024 (kStreamWarp), or 16
// lanes per row with the row's entries dealt round-robin (kSliced16).
// Warps sharing one row in the wide split of blocks whose row already fills a
// warp (32 FP64 columns): the dense Galerkin levels have too few rows to
// fill the GPU one row per warp.
constexpr int kWarpsPerRow = 4;

constexpr int kStreamShort = -1, kStreamLong = -2, kStreamQuad = -3, kStreamWarp = -4, kStreamMid = -5,
              kStreamPair = -6, kSliced16 = 16;
// FP32 blocks of 8 or more columns: the narrow split with operand rows staged
// through shared memory (rows_async); the `slices` code of the row launchers.
constexpr int kAsyncNarrow = 100;
// Blocks of 2 or 4 columns (8 or 16 bytes per block row): the stream kernel
// with one lane per row and a 256- or 1024-entry window (rows_stream_v).
constexpr int kStreamV256 = 200, kStreamV1024 = 201;
// (kPipeNarrow, kNarrow2 and kPipeNarrow2, the other narrow splits of FP64
// blocks of 8 or more columns, are defined with the row kernel in
// kernels.cuh.)

int device_sm_count();
extern std::atomic<int64_t> g_launches;  // kernels launched by the library

// Fused row operation with epilogue `epi` (enum Epi); returns the grid size
// used (needed to reduce op.partials), or -1 on a launch error or an
// unsupported combination.  One translation unit per NV (rows_nv*.cu).
int launch_rows(const RowOp &op, int nv, int slices, bool neg, int epi, cudaStream_t st);
int launch_rows_nv1(const RowOp &op, int slices, bool neg, int epi, cudaStream_t st);
int launch_rows_nv2(const RowOp &op, int slices, bool neg, int epi, cudaStream_t st);
int launch_rows_nv4(const RowOp &op, int slices, bool neg, int epi, cudaStream_t st);
int launch_rows_nv8(const RowOp &op, int slices, bool neg, int epi, cudaStream_t st);
int launch_rows_nv16(const RowOp &op, int slices, bool neg, int epi, cudaStream_t st);
int launch_rows_nv32(const RowOp &op, int slices, bool neg, int epi, cudaStream_t st);
// FP32 blocks; vt 0 = float values, 1 = bf16 values with per-row FP32 scale,
// 2 = bf16 values with 16-bit column indices, 3 = float values with 16-bit
// column indices.
int launch_rows_f(const RowOpF &op, int nv, int slices, bool neg, int epi, int vt, cudaStream_t st);
int launch_rowsf_nv1(const RowOpF &op, int slices, bool neg, int epi, int vt, cudaStream_t st);
int launch_rowsf_nv2(const RowOpF &op, int slices, bool neg, int epi, int vt, cudaStream_t st);
int launch_rowsf_nv4(const RowOpF &op, int slices, bool neg, int epi, int vt, cudaStream_t st);
int launch_rowsf_nv8(const RowOpF &op, int slices, bool neg, int epi, int vt, cudaStream_t st);
int launch_rowsf_nv16(const RowOpF &op, int slices, bool neg, int epi, int vt, cudaStream_t st);
int launch_rowsf_nv32(const RowOpF &op, int slices, bool neg, int epi, int vt, cudaStream_t st);

void launch_rb_s(int nv, int64_t n, double *S, const double *R, const double *V, const double *RH,
                 const ColState *cs, const double *w0, double *SH, double *part_ss, double *part_rs, int grid,
                 cudaStream_t st);
void launch_rb_xr(int nv, int64_t n, double *X, double *R, const double *S, const double *T, const double *PH,
                  const double *SH, const double *RH, const ColState *cs, double *part_rt, int grid,
                  cudaStream_t st);
void launch_pb_psz(int nv, int64_t n, double *P, double *S, double *Z, const double *R, const double *W,
                   const double *T, const double *V, const ColState *cs, int grid, cudaStream_t st);
void launch_pb_qy(int nv, int64_t n, double *Q, double *Y, const double *R, const double *S, const double *W,
                  const double *Z, const ColState *cs, double *part_qy, double *part_yy, int grid,
                  cudaStream_t st);
void launch_pb_urw(int nv, int64_t n, double *U, double *R, double *W, const double *P, const double *Q,
                   const double *Y, const double *T, const double *V, const double *S, const double *Z,
                   const double *RH, const ColState *cs, double *const part[5], int grid, cudaStream_t st);
void launch_pb_form_x(int nv, int64_t n, double *X, const double *X0, const double *D, int grid, cudaStream_t st);
void launch_pb_restart(int nv, int64_t n, const double *X, double *X0, double *U, double *RH, const double *R,
                       const ColState *cs, int grid, cudaStream_t st);
void launch_vscalar(int nv, int mode, ColState *cs, const VParts &P, double tol, int k, Flags *flags,
                    cudaStream_t st);

// Elementwise grid size for n rows of nv columns.
int elem_grid(int64_t n, int nv);

void launch_init_pcg(int nv, int64_t n, const double *B, int m, double *Bn, double *R, double *X,
                     double *Z, const double *w0, double *part, int grid, cudaStream_t st);
void launch_init_bicg(int nv, int64_t n, const double *B, int m, double *Bn, double *R, double *RH,
                      double *X, double *P, double *V, double *part, int grid, cudaStream_t st);
void launch_pcg_xr(int nv, int64_t n, double *X, double *R, const double *P, const double *Q,
                   const ColState *cs, const double *w0, double *Z, double *part, int grid,
                   cudaStream_t st);
void launch_pcg_p(int nv, int64_t n, double *P, const double *Z, const ColState *cs, int grid,
                  cudaStream_t st);
void launch_bicg_p(int nv, int64_t n, double *P, const double *R, const double *V,
                   const ColState *cs, const double *w0, double *PH, int grid, cudaStream_t st);
void launch_bicg_s(int nv, int64_t n, double *S, const double *R, const double *V,
                   const ColState *cs, const double *w0, double *SH, double *part, int grid,
                   cudaStream_t st);
void launch_bicg_xr(int nv, int64_t n, double *X, double *R, const double *S, const double *T,
                    const double *PH, const double *SH, const double *RH, const ColState *cs,
                    double *part_rr, double *part_rhr, int grid, cudaStream_t st);
void launch_copy_cols(int nv, int64_t n, double *dst, const double *src, const ColState *cs,
                      int grid, cudaStream_t st);
void launch_copy_out(int nv, int64_t n, const double *Xin, double *Xuser, int m, int grid,
                     cudaStream_t st);
void launch_pad_in(int nv, int64_t n, const double *Xuser, int m, double *Xp, int grid,
                   cudaStream_t st);
void launch_scale_rows(int nv, int64_t n, const double *w, const double *B, double *X, int grid,
                       cudaStream_t st);
void launch_axpy_dot(int nv, int64_t n, double *X, const double *D, const double *U, double *part,
                     int grid, cudaStream_t st);
void launch_coldot(int nv, int64_t n, const double *U, const double *V, double *part, int grid,
                   cudaStream_t st);
void launch_scalar(int nv, int mode, ColState *cs, const double *p0, const double *p1, int nblk,
                   double tol, int k, Flags *flags, cudaStream_t st);
// Coarsest solve X = Ainv B (Ainv: nc x nc inverse of the coarsest operator).
void launch_coarse(int nv, int nc, const double *Ainv, const double *B, double *X, cudaStream_t st);
// Outer FP64 loop around an FP32-block preconditioner.
void launch_init_fpcg(int nv, int64_t n, const double *B, int m, double *Bn, double *R, double *X,
                      float *R32, float *Z32, const float *w0, double *part, int grid,
                      cudaStream_t st);
void launch_fpcg_xr(int nv, int64_t n, double *X, double *R, const double *P, const double *Q,
                    const ColState *cs, const float *w0, float *R32, float *Z32, double *part,
                    int grid, cudaStream_t st);
void launch_fpcg_p(int nv, int64_t n, double *P, const float *Z32, const ColState *cs, int grid,
                   cudaStream_t st);
void launch_to_f32(int nv, int64_t n, const double *X, float *Y32, const float *w0, float *Z32,
                   int grid, cudaStream_t st);
void launch_to_f64(int nv, int64_t n, const float *X32, double *Y, int grid, cudaStream_t st);
void launch_axpy_dot_f(int nv, int64_t n, float *X, const float *D, const double *U,
                       const double *U2, double *part, double *part2, int grid, cudaStream_t st);
void launch_coarse_f(int nv, int nc, const double *Ainv, const float *B, float *X, cudaStream_t st);
void launch_zero_rhs_cols(int nv, int64_t n, double *X, const ColState *cs, int grid, cudaStream_t st);
// Runtime-m column dots for the public entry point: partials then reduce.
int coldot_rt_grid(int64_t n, int m);
void launch_coldot_rt(int64_t n, int m, const double *U, const double *V, double *part, int grid,
                      cudaStream_t st);
void launch_reduce_rt(int m, const double *part, int nblk, double *out, cudaStream_t st);

}  // namespace xamg
