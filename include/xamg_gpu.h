/*
 * xamg_gpu.h -- C ABI of the GB300 (sm_103a) solve-phase library for sparse
 * systems A X = B with m right-hand sides (paper Sec. 1: A is n x n, X and B
 * are n x m with m << n).
 *
 * The library builds a classical algebraic-multigrid hierarchy once on the
 * host (the paper's MultiGrid setup, Sec. 2.3) and then runs the solve phase
 * on one GPU: multi-column sparse products (the paper's "blas2" group,
 * Sec. 2.2-2.3), Chebyshev smoothing, restriction, prolongation, the
 * coarsest direct solve and the PCG / BiCGStab Krylov loops (Sec. 2.1,
 * Tab. 1) with per-column status flags.
 *
 * Conventions shared by every entry point:
 *   - Blocks of m columns are stored n x m ROW-MAJOR: element (i, j) of X is
 *     X[i*m + j] (the columns of one row are adjacent).
 *   - Return value 0 = success; negative = error (nothing usable written);
 *     positive = numerical outcome of a solve (results written).
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device (e.g. from torch.empty(..., device="cuda").data_ptr()); "host"
 *     pointers are ordinary process memory.  Pointers named const are only
 *     read.  The library never frees memory it did not allocate.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Every entry point that takes a stream enqueues its
 *     device work there and returns only after that work has finished.
 *   - Input and output blocks of one call must not overlap.
 *   - The handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef XAMG_GPU_H
#define XAMG_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define XAMG_OK 0
#define XAMG_ERR_INVALID_ARG (-1) /* bad size, pointer, layout or option       */
#define XAMG_ERR_CUDA (-2)        /* a CUDA runtime call failed                 */
#define XAMG_ERR_OOM (-3)         /* host or device allocation failed           */
#define XAMG_ERR_NONFINITE (-4)   /* NaN or Inf in the matrix or in B           */
#define XAMG_ERR_TIMEOUT (-5)     /* a bounded device wait ran out              */
#define XAMG_ERR_SETUP (-6)       /* hierarchy could not be built (zero pivot,
                                     zero diagonal, coarsest level too large)   */
#define XAMG_NOT_CONVERGED 1      /* some column missed tol within maxit        */
#define XAMG_BREAKDOWN 2          /* some column hit a Krylov breakdown         */

/* per-column status written to xamg_stats.status[j] */
#define XAMG_COL_CONVERGED 0
#define XAMG_COL_NOT_CONVERGED 1
#define XAMG_COL_BREAKDOWN 2

/* solver methods (paper Tab. 1: CG and BiCGStab as solvers, MultiGrid as
 * preconditioner, Chebyshev as pre-/post-smoother, Direct on the coarsest
 * level) */
#define XAMG_PCG 0
#define XAMG_BICGSTAB 1
/* BiCGStab variants (paper Sec. 2.1: "Reordered BiCGStab", "Pipelined
 * BiCGStab" and their merged formulations), the same right-preconditioned
 * method in exact arithmetic:
 *   REORDERED: the dot products of an iteration in two groups, (rhat, v) and
 *     (t, s), (t, t), (rhat, s), (rhat, t), (s, s), with rho and ||r|| of the
 *     next iteration from recurrences (Krasnopolsky 2010): one host read per
 *     iteration instead of two (no test between the two halves).
 *   PIPELINED: auxiliary products w = B r, s = B p, z = B s, t = B w, v = B z
 *     of B = A M, so that each group of dot products can run beside one
 *     application of B (Cools and Vanroose 2017); the solution is formed as
 *     x = x0 + M u when the columns stop.  Its recurrences assume a linear
 *     M: XAMG_PREC_FP64 only (XAMG_ERR_INVALID_ARG otherwise).
 * Vector updates carry their dot products in both (merged formulation). */
#define XAMG_BICGSTAB_REORDERED 2
#define XAMG_BICGSTAB_PIPELINED 3

/* preconditioner precision (paper Sec. 2.3, "mixed-precision": reduced
 * precision in the multigrid hierarchy only, basic precision for the result)
 *   XAMG_PREC_FP64  V-cycle in FP64, standard PCG / BiCGStab
 *   XAMG_PREC_FP32  V-cycle on FP32 blocks with FP32 values of A, P, R and
 *                   FP32 accumulation; FP64 coarsest solve; PCG becomes
 *                   flexible PCG (FP64 outer loop, FP64 dots and residuals)
 *   XAMG_PREC_BF16  as FP32, but A's values are bf16 relative to a per-row
 *                   FP32 scale s_i = max_j |a_ij|: a_ij ~ s_i bf16(a_ij / s_i);
 *                   where every row's columns lie in two consecutive windows
 *                   of 65536 columns, A's column indices are also stored as
 *                   uint16 (low 16 bits plus one per-row window word), read
 *                   by the products on blocks of two or more columns (m = 1
 *                   reads the 32-bit indices) */
#define XAMG_PREC_FP64 0
#define XAMG_PREC_FP32 1
#define XAMG_PREC_BF16 2

/* largest m accepted by the solve entry points */
#define XAMG_MAX_RHS 32

typedef struct xamg_hier xamg_hier; /* opaque, owned by the library */

/* A square sparse matrix in CSR form in HOST memory, read-only, owned by the
 * caller: rowptr[n+1] (rowptr[0] = 0, non-decreasing), col[nnz] strictly
 * ascending within each row and in [0, n), val[nnz].  Each row must hold a
 * nonzero diagonal entry. */
typedef struct {
  int32_t n;
  int64_t nnz;
  const int32_t *rowptr;
  const int32_t *col;
  const double *val;
} xamg_csr;

/* AMG setup parameters (fill with xamg_amg_params_default first).
 *   theta         strength threshold of classical Ruge-Stueben coarsening (0.25)
 *   max_coarse    a level with at most this many rows is the coarsest (64)
 *   max_levels    hard cap on the number of levels (25)
 *   cheb_steps    Chebyshev recurrence steps per smoothing = polynomial
 *                 order (2; paper Fig. 3 "polynomial_order 2"), in [1, 4]
 *   power_iters   power iterations for the largest eigenvalue of D^-1 A (20)
 *   cheb_lo_frac  lower end of the Chebyshev interval as a fraction of the
 *                 upper end (0.3)
 *   cheb_hi_safety  factor on the power-iteration estimate (1.1); the upper
 *                 end is min(cheb_hi_safety * estimate, Gershgorin bound)
 *   max_dense     largest coarsest level accepted for the dense LU (1024)
 *   nthreads      host threads for the setup (0 = all hardware threads)
 *   device_upload 1 (default): upload the hierarchy to the current CUDA
 *                 device; 0: build the host-side hierarchy only (no CUDA
 *                 call is made; only the xamg_*info, xamg_level_export,
 *                 xamg_coarse_export and xamg_hier_save entry points accept
 *                 such a handle) */
typedef struct {
  double theta;
  int32_t max_coarse;
  int32_t max_levels;
  int32_t cheb_steps;
  int32_t power_iters;
  double cheb_lo_frac;
  double cheb_hi_safety;
  int32_t max_dense;
  int32_t nthreads;
  int32_t device_upload;
} xamg_amg_params;

/* Solve options (fill with xamg_solve_opts_default first).
 *   method       XAMG_PCG, XAMG_BICGSTAB, XAMG_BICGSTAB_REORDERED or
 *                XAMG_BICGSTAB_PIPELINED
 *   precond      XAMG_PREC_FP64 (default), XAMG_PREC_FP32 or XAMG_PREC_BF16
 *   x0_given     0 (default): start from X = 0; 1: X holds the initial guess
 *                X0 on entry (a warm start, e.g. a learned prediction); the
 *                stopping test stays ||b_j - A x_j|| <= tol ||b_j||, and a
 *                zero column b_j still returns x_j = 0
 *   stream       cudaStream_t as void*, NULL = legacy default stream
 *   workspace    optional caller-owned DEVICE buffer of workspace_bytes bytes
 *                (at least xamg_workspace_bytes(); 256-byte aligned); NULL
 *                makes the library allocate and cache one inside the handle
 *   workspace_bytes  size of `workspace` */
typedef struct {
  int32_t method;
  int32_t precond;
  int32_t x0_given;
  void *stream;
  void *workspace;
  size_t workspace_bytes;
} xamg_solve_opts;

/* Per-solve statistics (paper Fig. 2, "solver->stats").  The three arrays are
 * caller-owned HOST arrays of length m; any of them may be NULL.
 *   iters[j]   Krylov iterations of column j (one preconditioner application
 *              per PCG iteration, two per BiCGStab iteration)
 *   relres[j]  true relative residual ||b_j - A x_j|| / ||b_j|| at exit
 *              (0 for a zero column)
 *   status[j]  XAMG_COL_* code
 *   iterations total loop iterations the call ran (max over columns)
 *   vcycles    preconditioner applications the call ran */
typedef struct {
  int32_t *iters;
  double *relres;
  int32_t *status;
  int32_t iterations;
  int32_t vcycles;
} xamg_stats;

/* Human-readable text for a status code (static storage). */
const char *xamg_strerror(int code);

void xamg_amg_params_default(xamg_amg_params *p);
void xamg_solve_opts_default(xamg_solve_opts *o);

/* Builds the AMG hierarchy of A on the host (classical Ruge-Stueben
 * coarsening, classical interpolation, Galerkin R A P with R = P^T, Chebyshev
 * interval per level, dense LU of the coarsest level; paper Sec. 2.3: the
 * MultiGrid setup()) and uploads it to the current CUDA device.  A is read
 * only during the call.  On success *out holds a new handle owned by the
 * caller, to be released with xamg_destroy.  Errors: INVALID_ARG (bad CSR,
 * missing diagonal), NONFINITE, SETUP, OOM, CUDA. */
int xamg_setup_hierarchy(const xamg_csr *A, const xamg_amg_params *p, xamg_hier **out);

/* Releases the handle and every device buffer it owns.  NULL is accepted. */
int xamg_destroy(xamg_hier *h);

/* The frozen hierarchy as a byte blob (the "hierarchy as input" of the
 * solve phase): the setup parameters and every level's A, P, R, coarse /
 * fine flags, inverse diagonal and Chebyshev interval, plus the coarsest
 * LU factors, written field by field in this host's byte order behind a
 * magic string and a format version.  *bytes receives the blob's size; with
 * blob = NULL nothing else happens (size query), else the blob is written to
 * the caller's buffer of `capacity` bytes (XAMG_ERR_INVALID_ARG if smaller).
 * Host only. */
int xamg_hier_save(const xamg_hier *h, void *blob, size_t capacity, size_t *bytes);

/* A hierarchy from a blob of xamg_hier_save, uploaded to the current device
 * when its saved parameters ask for it (device_upload), exactly as after
 * xamg_setup_hierarchy: solves on it equal those on the saved hierarchy bit
 * for bit.  XAMG_ERR_INVALID_ARG if the blob is not a complete, well-formed
 * hierarchy of this format (every length, offset and index is checked).
 * The caller's blob is only read. */
int xamg_hier_load(const void *blob, size_t bytes, xamg_hier **out);

/* Number of levels and the row count, nnz of A, nnz of P of level `level`
 * (nnz_p = 0 on the coarsest level).  Any output pointer may be NULL. */
int xamg_hier_info(const xamg_hier *h, int32_t *levels, double *op_complexity);
int xamg_level_info(const xamg_hier *h, int32_t level, int32_t *n, int64_t *nnz_a,
                    int64_t *nnz_p);

/* Copies the host-side setup results of one level into caller-owned HOST
 * arrays (any may be NULL): rowptr[n+1], col[nnz_a], val[nnz_a] of A;
 * p_rowptr[n+1], p_col[nnz_p], p_val[nnz_p] of P; cf[n] (1 = coarse point);
 * cheb[4] = {lower, upper, power estimate, Gershgorin bound}. */
int xamg_level_export(const xamg_hier *h, int32_t level, int32_t *rowptr, int32_t *col,
                      double *val, int32_t *p_rowptr, int32_t *p_col, double *p_val,
                      int32_t *cf, double *cheb);

/* Copies the coarsest level's dense LU factors (row-major nc x nc, unit lower
 * L below the diagonal, U on and above it) and pivot rows (row k was swapped
 * with row piv[k]) into caller-owned HOST arrays; *nc receives the size. */
int xamg_coarse_export(const xamg_hier *h, int32_t *nc, double *lu, int32_t *piv);

/* Bytes of device workspace a solve of m columns with `method` and
 * preconditioner precision `precond` needs. */
int xamg_workspace_bytes(const xamg_hier *h, int32_t m, int32_t method, int32_t precond,
                         size_t *bytes);

/* Solves A X = B to ||b_j - A x_j|| <= tol ||b_j|| for every column
 * (paper Sec. 1 and 2.1; PCG or BiCGStab preconditioned by one V(1,1)
 * Chebyshev cycle, paper Fig. 3).  B and X are DEVICE n x m row-major
 * blocks, 1 <= m <= XAMG_MAX_RHS, caller-owned; X0 = 0 unless
 * opts->x0_given.  Each column stops
 * on its own (status flags); X always holds the last iterate.  Returns 0 when
 * every column converged, XAMG_NOT_CONVERGED / XAMG_BREAKDOWN otherwise, or
 * a negative error (NONFINITE if B holds NaN/Inf: X is then untouched).
 * `stats` may be NULL. */
int xamg_solve(xamg_hier *h, const double *B, double *X, int32_t m, double tol, int32_t maxit,
               const xamg_solve_opts *opts, xamg_stats *stats);

/* As xamg_solve with B and X in HOST memory, all on opts->stream.  When both
 * are page-locked memory registered with CUDA (cudaHostAlloc,
 * cudaHostRegister, a pinned torch tensor), the solve's first pass reads B
 * and its last pass writes X directly over the host link; otherwise the call
 * copies B to a device buffer, solves, and copies X back. */
int xamg_solve_host(xamg_hier *h, const double *B, double *X, int32_t m, double tol,
                    int32_t maxit, const xamg_solve_opts *opts, xamg_stats *stats);

/* ---- single steps of the solve phase, for testing and measurement ---- */

/* Y = M X on level `level` for M = A (which = 0), P (which = 1, level <
 * levels-1, X has n_{level+1} rows) or R = P^T (which = 2, Y has n_{level+1}
 * rows): the multi-column sparse product of paper Sec. 2.2.  X, Y: DEVICE
 * row-major blocks with m columns, 1 <= m <= XAMG_MAX_RHS. */
int xamg_level_spmm(xamg_hier *h, int32_t level, int32_t which, const double *X, double *Y,
                    int32_t m, void *stream);

/* Y = M X on level `level` in the reduced precision `precond`
 * (XAMG_PREC_FP32: FP32 values of M; XAMG_PREC_BF16: for M = A the bf16
 * values with their FP32 row scales, y_i = s_i (sum_k q_ik x_k), and FP32
 * values of P and R): the product of the preconditioner's V-cycle (paper
 * Sec. 2.3, "mixed-precision" and index compression), with the same split and
 * 16-bit index choice the V-cycle makes for blocks of pad(m) columns.  X is
 * rounded to FP32 (exactly, when it holds FP32 values), every term is added
 * to the FP32 row sum with one rounding, and the FP32 result is widened into
 * Y.  which, level, X and Y as for xamg_level_spmm: DEVICE FP64 row-major
 * blocks with m columns, 1 <= m <= XAMG_MAX_RHS, caller-owned.  The first
 * reduced-precision call uploads the FP32/bf16 copies of the hierarchy.
 * Errors: INVALID_ARG (bad level, operator, m or precond), CUDA, OOM. */
int xamg_level_spmm_precond(xamg_hier *h, int32_t precond, int32_t level, int32_t which,
                            const double *X, double *Y, int32_t m, void *stream);

/* Fused coarse tail of the V(1,1) cycle (off by default; max_elems = 131072
 * is the tested setting).  The levels whose n x pad(m) blocks hold at most
 * max_elems elements -- from
 * the first such level down to the coarsest and back up to its first
 * post-smoothing step, at most ten levels, blocks of two or more columns,
 * two Chebyshev steps -- run as one cooperative kernel launch with a
 * grid-wide barrier between stages (paper Sec. 2.1: the V-cycle; the fusion
 * is this library's).  Each stage computes exactly what its separate launch
 * would, so results are bitwise those of the unfused cycle.  On GB300 it
 * measured slower than the separate launches replayed from a CUDA graph
 * (a stage with its grid barrier took about 12 us against about 5 us per
 * launch: the barrier itself costs 2 us, and the cooperative kernel holds
 * only two blocks per SM), hence off by default.  max_elems = 0 turns the
 * fusion off.  Every barrier wait is bounded by wait_limit_s
 * seconds (0 < wait_limit_s <= 60; default 2): a wait that runs out ends the
 * kernel, and the solve or V-cycle returns XAMG_ERR_TIMEOUT (X then holds no
 * meaningful result; the device stays usable).  extra_arrivals > 0 adds
 * arrivals that never come to every barrier: fault injection for testing
 * the bounded waits (0 in normal use).  Drops the cached CUDA graphs.  Host
 * only.  Errors: INVALID_ARG. */
int xamg_set_tail(xamg_hier *h, int64_t max_elems, double wait_limit_s, int32_t extra_arrivals);

/* First level of the fused coarse tail for blocks of pad(m) columns, or -1
 * when the cycle runs unfused, written to *first_level.  Host only.
 * Errors: INVALID_ARG. */
int xamg_tail_info(const xamg_hier *h, int32_t m, int32_t *first_level);

/* 16-bit column indices of the reduced-precision products (paper Sec. 2.3:
 * CSR index types reduced to uint16_t), off by default: on GB300 the decode
 * lengthens each row's index -> operand-gather chain by more than the two
 * bytes per entry it saves, measured at every block width.  Each operator that
 * fits the segmented form -- rows cut into tiles of 32, each tile with at
 * most four segment bases that cover every column of its rows within 65535
 * -- stores its columns as 16-bit offsets and is read that way by blocks of
 * two or more columns; decoding is exact, so results do not depend on the
 * setting.  enable = 0 reads the 32-bit indices everywhere (it drops the
 * cached CUDA graphs).  Host only.  No counterpart of the switch in the
 * paper. */
int xamg_set_index16(xamg_hier *h, int32_t enable);

/* Which operators of level `level` have 16-bit column indices: bit 0 = A,
 * bit 1 = P, bit 2 = R, written to *mask.  Uploads the reduced-precision
 * copies of the hierarchy on first use.  Errors: INVALID_ARG, CUDA, OOM. */
int xamg_index16_info(xamg_hier *h, int32_t level, int32_t *mask);

/* Chebyshev smoothing on level `level` (< levels-1): cheb_steps steps on X
 * for right-hand side B.  x_zero = 1 takes X = 0 on entry (pre-smoothing)
 * and then, if R is not NULL, writes the residual B - A X after the last
 * step to R; x_zero = 0 smooths the given X (post-smoothing; R must be
 * NULL).  DEVICE row-major blocks with m columns. */
int xamg_smooth(xamg_hier *h, int32_t level, const double *B, double *X, double *R,
                int32_t x_zero, int32_t m, void *stream);

/* One V(1,1) cycle from X = 0 for right-hand side B (the preconditioner
 * application z = M^-1 r of paper Fig. 3, MultiGrid with max_iters 1).
 * DEVICE row-major blocks n x m. */
int xamg_vcycle(xamg_hier *h, const double *B, double *X, int32_t m, void *stream);

/* One V(1,1) cycle in preconditioner precision `precond` (XAMG_PREC_*): B is
 * rounded to the FP32 block, the cycle runs on FP32 blocks (FP64 coarsest
 * solve) and its result is widened into X.  DEVICE FP64 row-major blocks
 * n x m.  XAMG_PREC_FP64 is xamg_vcycle.  The first reduced-precision call
 * uploads the FP32/bf16 copies of the hierarchy (kept until xamg_destroy). */
int xamg_vcycle_precond(xamg_hier *h, int32_t precond, const double *B, double *X, int32_t m,
                        void *stream);

/* Coarsest-level direct solve X = A_L^-1 B (paper Tab. 1, Direct): the
 * setup's LU factors (partial pivoting) give the explicit inverse once, at
 * upload, and every solve is the dense FP64 product A_L^-1 B on the tensor
 * cores (mma.sync m8n8k4 .f64).  DEVICE row-major blocks n_L x m. */
int xamg_coarse_solve(xamg_hier *h, const double *B, double *X, int32_t m, void *stream);

/* Column dot products out[j] = sum_i U[i*m + j] * V[i*m + j] of two DEVICE
 * n x m row-major blocks (the paper's "blas" dot products, Sec. 2.3), into the
 * DEVICE array out[m].  The sum is reduced in a fixed order, so repeated
 * calls give identical bits.  Allocates (and frees) its own device scratch
 * for the per-block partial sums.  A CUDA error that earlier work left
 * pending in the runtime is reported as XAMG_ERR_CUDA (and cleared). */
int xamg_coldot(const double *U, const double *V, int64_t n, int32_t m, double *out,
                void *stream);

/* Column dot products like xamg_coldot, for callers that must not allocate
 * device memory during the call: for example a host framework that has
 * reserved all device memory for its own pool (so cudaMalloc would fail), or
 * a latency-critical loop that must not enter the CUDA allocator, which may
 * synchronize the device.  There is no counterpart in the paper.
 *
 * U, V: DEVICE n x m row-major blocks; out: DEVICE array of m doubles; all
 * caller-owned.  The per-block partial sums live in one file-scope device
 * array of the library (1024 blocks x 32 columns of doubles, 256 KiB), which
 * every GPU that loads the library keeps until the process exits; the call
 * uses at most 1024 blocks, so any n >= 0 is accepted, and m must be in
 * [1, XAMG_MAX_RHS] (else XAMG_ERR_INVALID_ARG, nothing launched).  The call
 * makes no cudaMalloc, cudaFree or other allocating call.  Its first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.  The
 * address is kept for the life of the process, so the library must not be
 * used across a cudaDeviceReset of that device.  A CUDA error that earlier
 * work left pending in the runtime is reported by this call as
 * XAMG_ERR_CUDA (and cleared), like any launch error of its own.  All
 * calls share the array and it keeps the last call's contents: calls whose
 * device work overlaps (other streams, other threads) race on it and must be
 * serialised by the caller.  Results are reduced in a fixed order; they may
 * differ from xamg_coldot's in the last bits because the block count differs.
 * Returns after the work on `stream` has finished. */
int xamg_coldot_noalloc(const double *U, const double *V, int64_t n, int32_t m, double *out,
                        void *stream);

/* Autotuner of the preconditioner's sparse products: for every level's A, P
 * and R, times y = M x on blocks of pad(m) columns (m in [1, XAMG_MAX_RHS])
 * of the precision `precond` selects (XAMG_PREC_FP64: FP64 blocks;
 * XAMG_PREC_FP32 / XAMG_PREC_BF16: FP32 blocks with FP32 / bf16 values of A)
 * under every row split -- for m > 1 the default (a group of lanes per row,
 * several rows per warp), one row per warp with its entries split over the
 * lanes (16 and 32 FP64 columns: four warps per row) and the third
 * candidate where xamg_set_split lists one; for m = 1 the stream kernel (the
 * warp's entries staged in shared memory) with one lane per row and a 256-,
 * 512- or 1024-entry window, 2, 4 or 32 lanes per row, and 16 lanes per row
 * without staging -- and keeps the fastest in the hierarchy; later solves
 * and V-cycles of that block width and precision use it.  Results do not
 * depend on the split beyond the order of each row's sums.  ops_tuned /
 * ops_wide (may be NULL): products tuned and how many chose a split other
 * than the first candidate.  Uses the hierarchy's cached
 * workspace; synchronizes `stream`.  No counterpart in the paper. */
int xamg_autotune(xamg_hier *h, int32_t m, int32_t precond, void *stream, int32_t *ops_tuned,
                  int32_t *ops_wide);

/* Sets the row split of one sparse product by hand (what xamg_autotune sets
 * by timing): operator `which` (0 = A, 1 = P, 2 = R; P and R exist below the
 * coarsest level) of level `level`, blocks of pad(m) columns of precision
 * `precond`.  candidate: -1 = the default rule; otherwise the index of a
 * tuning candidate -- m = 1: 0 = stream kernel, one lane per row, 256-entry
 * window; 1 = 16 lanes per row; 2, 3, 4 = stream kernel with a 1024-entry
 * window and 1 lane, 4 lanes or a warp per row; 5, 6 = stream kernel with a
 * 512-entry window and 1 or 2 lanes per row; m > 1: 0 = a
 * group of lanes per row, 1 = one row per warp (for FP64 blocks of 16 and
 * 32 columns: four warps per row), and for FP32 blocks of 8 or more columns
 * 2 = a group of lanes per row with the operand rows staged through shared
 * memory by asynchronous copies (the sums of candidate 0, bit for bit; an
 * operator whose warp row groups exceed the staging window takes 0), for
 * blocks of 2 or 4 columns 2 = the stream kernel of m = 1 with one lane
 * per row holding the row's columns (the sums of candidate 0), and for FP64
 * blocks of 8, 16 or 32 columns 2 = candidate 0 with its row loop
 * software-pipelined (the next rows' column indices and row pointers
 * loaded while a row's operand rows are gathered; the sums of candidate 0),
 * 3 = candidate 0 and 4 = candidate 2 with two adjacent columns per lane,
 * so that a warp works on two rows at once (the sums of candidate 0).
 * Results do not depend on the split beyond the order of each row's sums.  XAMG_ERR_INVALID_ARG for any other
 * value.  Host only.  No counterpart in the paper. */
int xamg_set_split(xamg_hier *h, int32_t m, int32_t precond, int32_t level, int32_t which,
                   int32_t candidate);

/* CUDA graphs of the steady PCG iteration (on by default).  With graphs on,
 * the PCG solves (XAMG_PCG, every precond) replay the fixed launch sequence
 * between two host reads of an iteration -- preconditioner, beta, direction
 * update, A p, alpha, x/r update, convergence test -- as one captured graph,
 * cached per (block width, precond, workspace, tol) on the hierarchy and
 * dropped when the workspace or a row split changes.  Results are bitwise
 * those of the uncaptured launches; small systems, whose solves are bound by
 * launch latency, gain the most.  Timing (xamg_timing_enable) bypasses them.
 * enable = 0 turns them off and frees the cache.  No counterpart in the
 * paper. */
int xamg_set_graphs(xamg_hier *h, int32_t enable);

/* ---- batched solve of many independent systems ----
 *
 * Solves count independent systems A_s X_s = B_s (A_s n_s x n_s with its own
 * frozen hierarchy h[s], B_s and X_s n_s x m[s] row-major DEVICE blocks) to
 * the relative residual tol per column.  Each system runs exactly the steps
 * of xamg_solve with method XAMG_PCG and precond XAMG_PREC_FP32 (flexible PCG
 * in FP64 around the FP32 V(1,1) Chebyshev preconditioner, FP64 coarsest
 * solve), and all systems advance in lockstep: every stage of the V-cycle
 * and of the Krylov loop is one launch for all of them (one per block width
 * and row split present, for the row stages), whatever their sizes and
 * hierarchy depths.  A system leaves the lockstep when all
 * its columns are confirmed converged.  The paper solves one system at a
 * time; this form serves many small systems, whose single-system launches are
 * latency-bound.
 *
 * Requirements: every hierarchy on the same device with at least two levels
 * and cheb_steps = 2 (the default); 1 <= m[s] <= XAMG_MAX_RHS.  Otherwise
 * XAMG_ERR_INVALID_ARG. */
typedef struct xamg_batch xamg_batch;

typedef struct {
  int32_t autotune;  /* 1 (default): at creation, time both row splits (rows per warp: the
                        single-system default, or one row per warp with its entries split over
                        the lanes) of every FP32 operator of every level and keep the faster */
  int32_t use_graph; /* 1 (default): replay the steady iteration as one CUDA graph */
} xamg_batch_opts;

void xamg_batch_opts_default(xamg_batch_opts *o);

/* Plans the batch: device tables of the systems, one workspace for all of
 * them (allocated here and owned by the batch), launch grids, autotuning.
 * The hierarchies must outlive the batch. */
int xamg_batch_create(xamg_hier *const *h, const int32_t *m, int32_t count, const xamg_batch_opts *opts,
                      xamg_batch **out);
int xamg_batch_destroy(xamg_batch *b);

/* Launches per steady iteration (for every system together), operators
 * autotuned and how many of them chose the one-row-per-warp split, bytes of
 * the batch's workspace.  Output pointers may be NULL. */
int xamg_batch_info(const xamg_batch *b, int32_t *launches_per_iteration, int32_t *ops_tuned, int32_t *ops_wide,
                    int64_t *workspace_bytes);

/* B, X: HOST arrays of count DEVICE pointers.  stats: NULL or a HOST array of
 * count xamg_stats (their per-column arrays sized m[s]).  Work runs on the
 * batch's own stream, ordered after earlier work on `stream` and before later
 * work on it; returns when the solutions are written.  Return code as
 * xamg_solve's, over all systems. */
int xamg_batch_solve(xamg_batch *b, const double *const *B, double *const *X, double tol, int32_t maxit,
                     void *stream, xamg_stats *stats);

/* ---- learned initial guess ----
 *
 * A 3-D convolutional encoder-decoder that predicts a first iterate X0 of the
 * solve from (B, log coefficient) on an N^3 grid, trained on the GPU on
 * solutions this library computes; the solve then starts from X0
 * (xamg_solve_opts.x0_given) instead of X0 = 0.  The paper has no learned
 * component.  Architecture, four grid levels of edge N, N/2, N/4, N/8 (all
 * convolutions 3x3x3, stride 1, zero padding, ReLU after all but the last):
 *   e0a 2->8, e0b 8->8 | avg-pool 2, e1a 8->16, e1b 16->16 | pool, e2a, e2b
 *   16->16 | pool, e3a, e3b 16->16 | nearest-upsample + skip(e2b), d2 16->16 |
 *   up + skip(e1b), d1a 16->16, d1b 16->8 | up + skip(e0b), d0a 8->8, d0b 8->1.
 * The flat FP32 parameter vector (xamg_net_param_count() floats) holds, per
 * layer in the order above, W[cout][27][cin] (tap t = 9(dz+1) + 3(dy+1) +
 * (dx+1), a cross-correlation) then b[cout]; e0a is stored with cin = 8 (input
 * channels 2..7 are zero) and d0b with cout = 8 (only output channel 0 is
 * used), so their extra weights receive zero gradient.  Activations and
 * gradients are BF16, products accumulate in FP32 on the tensor cores,
 * parameters and Adam moments are FP32.  One handle serves one device and
 * one stream at a time. */
typedef struct xamg_net xamg_net;

typedef struct {
  float lr, beta1, beta2, eps; /* Adam step size and decay rates; eps > 0 */
} xamg_adam;

int64_t xamg_net_param_count(void);

/* Allocates a network for N^3 grids (N a multiple of 8, 8 <= N <= 1024) and
 * batches of up to max_batch samples on the current device; parameters start
 * at zero (set them with xamg_net_set_params). */
int xamg_net_create(int32_t N, int32_t max_batch, xamg_net **out);
void xamg_net_destroy(xamg_net *net);

/* HOST flat parameter vectors (layout above); set also resets Adam. */
int xamg_net_set_params(xamg_net *net, const float *params);
int xamg_net_get_params(const xamg_net *net, float *params);

/* out[b][v] = network output (FP32 channel 0 of the last layer) for the
 * DEVICE input inp[b][v][2] (FP32 pairs: normalised right-hand side, log
 * coefficient), v = (z N + y) N + x; out is a DEVICE [batch][N^3] array.
 * Returns after the work on `stream` has finished. */
int xamg_net_forward(xamg_net *net, const float *inp, float *out, int32_t batch, void *stream);

/* Training loss.  With e_b = out_b - target_b for sample b of a batch and
 * w_b = sample_weight[row of b] (1 if sample_weight is NULL):
 *   XAMG_NET_LOSS_MSE:    L = sum_b w_b |e_b|^2 / (batch N^3)
 *   XAMG_NET_LOSS_ENERGY: L = sum_b w_b e_b^T A_b e_b / batch, with A_b the
 *     cell-centred diffusion operator on the N^3 grid of unit cells whose log
 *     coefficient is the sample's input channel 1 (face transmissibility
 *     2 k_a k_c / (k_a + k_c) between cells, 2 k_c on a boundary face).
 * The energy norm is the norm in which PCG's error decreases, so it weighs
 * the parts of e that the solve would otherwise have to remove. */
#define XAMG_NET_LOSS_MSE 0
#define XAMG_NET_LOSS_ENERGY 1
typedef struct {
  int32_t kind;                /* XAMG_NET_LOSS_MSE or XAMG_NET_LOSS_ENERGY */
  const float *sample_weight;  /* DEVICE, one per sample row, or NULL */
} xamg_net_loss;

/* Loss L (lo NULL: unweighted MSE) of the DEVICE batch inp[batch][N^3][2],
 * target[batch][N^3] (FP32) into *loss and, if grad != NULL, dL/dparams into
 * the HOST array grad (flat layout); sample_weight is indexed by b.
 * XAMG_ERR_NONFINITE if L is not finite. */
int xamg_net_loss_grad(xamg_net *net, const float *inp, const float *target, int32_t batch,
                       const xamg_net_loss *lo, float *loss, float *grad, void *stream);

/* One Adam step on the loss of the samples idx[0..batch) (DEVICE int32
 * indices into the DEVICE arrays inp[nsamples][N^3][2] and
 * target[nsamples][N^3]; sample_weight is indexed by idx[b]); *loss (may be
 * NULL) receives the loss before the step.  The indices are copied to the
 * host and checked (each in [0, nsamples), else XAMG_ERR_INVALID_ARG and
 * nothing is launched), so the call synchronizes `stream` once before its
 * kernels. */
int xamg_net_train_step(xamg_net *net, const float *inp, const float *target, int64_t nsamples,
                        const int32_t *idx, int32_t batch, const xamg_net_loss *lo, const xamg_adam *opt,
                        float *loss, void *stream);

/* Initial guess for the DEVICE n x m row-major block B (n = N^3, m <=
 * min(max_batch, XAMG_MAX_RHS)) and DEVICE FP32 log coefficient logk[n]:
 * column j is fed as B[:, j] / s_j with s_j = ||B[:, j]||_2 / sqrt(n), and
 * X0[v][j] = out_j[v] * s_j * out_scale (a zero column gives X0 = 0).
 * X0 is a DEVICE n x m row-major block.  Asynchronous on `stream`. */
int xamg_net_predict_x0(xamg_net *net, const double *B, const float *logk, double out_scale, double *X0,
                        int32_t m, void *stream);

/* Single layers, for testing: BF16 tensors are uint16 bit patterns in DEVICE
 * memory, channels-last [batch][N^3][c]; W is DEVICE FP32 [cout][27][cin],
 * bias DEVICE FP32 [cout] or NULL; cin, cout in {8, 16}; any N >= 1.
 * adjoint = 0: out[v][co] = relu?(b[co] + sum W[co][t][ci] in'[v + off_t][ci])
 *              with in' = in * (mask > 0) if mask != NULL (mask shaped like in);
 * adjoint = 1: the backward-data product: `in` has cout channels, out has
 *              cin: out[v][ci] = sum W[co][t][ci] in'[v - off_t][co]
 *              (bias must be NULL).
 * Inputs outside the grid are zero.  Allocates (and frees) device
 * temporaries; returns after the work on `stream` has finished. */
int xamg_conv3d_bf16(const uint16_t *in, const uint16_t *mask, const float *w, const float *bias, uint16_t *out,
                     int32_t batch, int32_t N, int32_t cin, int32_t cout, int32_t relu, int32_t adjoint,
                     void *stream);

/* Weight and bias gradients of one layer (DEVICE FP32 dw[cout][27][cin],
 * db[cout]): dw[co][t][ci] = sum_{b,v} g[v][co] in[v + off_t][ci] and
 * db[co] = sum g[v][co], with g = gout * (act > 0) if act != NULL else gout
 * (gout and act: [batch][N^3][cout], in: [batch][N^3][cin]).  Sums are
 * reduced in a fixed order. */
int xamg_conv3d_bf16_wgrad(const uint16_t *in, const uint16_t *gout, const uint16_t *act, float *dw, float *db,
                           int32_t batch, int32_t N, int32_t cin, int32_t cout, void *stream);

/* ---- measurement ---- */

/* Turns per-launch timing of the sparse row kernels on (1) or off (0).  When
 * on, every launch of a row kernel (the fused SpMM-based steps) is bracketed
 * by CUDA events on the launching stream; the results are accumulated per
 * (level, operator) when the enclosing call finishes.  Off by default. */
int xamg_timing_enable(xamg_hier *h, int32_t enable);

/* Reads and clears nothing: launches and total device milliseconds of the
 * timed row-kernel launches on `level` for operator `which` (0 = A, 1 = P,
 * 2 = R on FP64 blocks; 3, 4, 5 = the same on FP32 blocks) since timing was
 * last enabled, plus the algorithmic flops and bytes
 * of those launches (flops = 2 nnz m_padded; bytes = 12 nnz + 4 (rows+1) +
 * 8 (cols_in + rows) m_padded per product plus the epilogue's block reads and
 * writes).  Output pointers may be NULL. */
int xamg_timing_read(const xamg_hier *h, int32_t level, int32_t which, int64_t *launches,
                     double *total_ms, double *flops, double *bytes);

/* Number of kernel launches the library has issued in this process (all
 * handles, all devices) since it was loaded. */
int64_t xamg_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* XAMG_GPU_H */
