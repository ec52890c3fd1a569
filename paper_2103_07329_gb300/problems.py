"""Seeded synthetic inputs shared by the library, its tests and the benchmark.

This module only *generates problems*: the sparse matrices of the paper's test
systems and the random right-hand sides.  It holds none of the solver's
arithmetic (no setup, smoothing, Krylov or multigrid step), so both the CUDA
path and the CPU oracle can take their inputs from it.

Matrices (paper Sec. 3, "Example case": the 3D Poisson equation on a cube,
7-point stencil):
  * ``poisson7(N)``: A = -Delta_h on an N^3 grid, unit spacing without the h^2
    factor, Dirichlet boundary nodes eliminated (their couplings are simply
    absent), diagonal 6, off-diagonals -1.  The sign makes A symmetric positive
    definite, which CG needs.  Ordering is lexicographic, row index
    i + N j + N^2 k with i fastest.
  * ``poisson27(N)``: the 27-point analogue, diagonal 26, all 26 neighbours -1.

  * ``diffusion7(N, k)``: cell-centred finite volumes for -div(k grad u) with
    cell coefficients k (e.g. lognormal, ``lognormal_cells``), the
    variable-coefficient systems the mixed-precision and batched forms use.
  * ``grf(N, corr_len, sigma, seed)``: Gaussian random fields (log-coefficients
    and smooth right-hand sides of the learned warm start).

Right-hand sides: entries i.i.d. uniform[-1, 1) from numpy's
``default_rng(seed)``, n x m row-major (C order).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """A square sparse matrix in CSR form: int32 row pointers and column
    indices (ascending within each row, diagonal included), float64 values."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _stencil(N: int, offsets, diag: float) -> CSR:
    if N < 1:
        raise ValueError("grid edge N must be >= 1")
    n = N * N * N
    idx = np.arange(n, dtype=np.int64)
    i = idx % N
    j = (idx // N) % N
    k = idx // (N * N)
    cols = np.empty((n, len(offsets)), dtype=np.int32)
    valid = np.empty((n, len(offsets)), dtype=bool)
    vals = np.empty((n, len(offsets)), dtype=np.float64)
    for t, (dk, dj, di) in enumerate(offsets):
        ok = ((i + di >= 0) & (i + di < N) & (j + dj >= 0) & (j + dj < N)
              & (k + dk >= 0) & (k + dk < N))
        cols[:, t] = (idx + di + N * dj + N * N * dk).astype(np.int32)
        valid[:, t] = ok
        vals[:, t] = diag if (dk, dj, di) == (0, 0, 0) else -1.0
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    col = cols[valid]
    val = vals[valid]
    return CSR(n, rowptr.astype(np.int32), np.ascontiguousarray(col, dtype=np.int32),
               np.ascontiguousarray(val, dtype=np.float64))


def poisson7(N: int) -> CSR:
    """7-point -Laplacian on an N^3 grid (Dirichlet nodes eliminated)."""
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    return _stencil(N, offs, 6.0)


def poisson27(N: int) -> CSR:
    """27-point Laplacian on an N^3 grid (Dirichlet nodes eliminated)."""
    offs = [(dk, dj, di) for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
    return _stencil(N, offs, 26.0)


def lognormal_cells(N: int, sigma: float, seed: int) -> np.ndarray:
    """Cell coefficients k = exp(sigma g), g i.i.d. standard normal from
    numpy's default_rng(seed), one per cell in lexicographic order."""
    return np.exp(sigma * np.random.default_rng(seed).standard_normal(N * N * N))


def diffusion7(N: int, kcell: np.ndarray) -> CSR:
    """Cell-centred finite-volume -div(k grad u) on an N^3 grid of unit cells.

    Face transmissibility between cells a and b is the harmonic mean
    2 k_a k_b / (k_a + k_b); a boundary face carries the Dirichlet value at the
    face, half a cell away, so its transmissibility is 2 k_c.  Off-diagonals
    are -T, the diagonal the sum of the cell's six face transmissibilities.
    Rows are lexicographic with i fastest, columns ascending."""
    n = N * N * N
    k = np.asarray(kcell, dtype=np.float64).reshape(-1)
    if k.size != n or np.any(k <= 0) or not np.all(np.isfinite(k)):
        raise ValueError("need N^3 positive finite cell coefficients")
    idx = np.arange(n, dtype=np.int64)
    i = idx % N
    j = (idx // N) % N
    kk = idx // (N * N)
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    cols = np.empty((n, 7), dtype=np.int64)
    valid = np.empty((n, 7), dtype=bool)
    vals = np.zeros((n, 7), dtype=np.float64)
    diag = np.zeros(n, dtype=np.float64)
    for t, (dk, dj, di) in enumerate(offs):
        if (dk, dj, di) == (0, 0, 0):
            continue
        ok = ((i + di >= 0) & (i + di < N) & (j + dj >= 0) & (j + dj < N)
              & (kk + dk >= 0) & (kk + dk < N))
        nb = idx + di + N * dj + N * N * dk
        T = np.where(ok, 2.0 * k * k[np.where(ok, nb, idx)] / (k + k[np.where(ok, nb, idx)]), 2.0 * k)
        diag += T
        cols[:, t] = nb
        valid[:, t] = ok
        vals[:, t] = -T
    cols[:, 3] = idx
    valid[:, 3] = True
    vals[:, 3] = diag
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), np.ascontiguousarray(cols[valid], dtype=np.int32),
               np.ascontiguousarray(vals[valid], dtype=np.float64))


def grf(N: int, corr_len: float, sigma: float, seed: int, count: int = 1, pad: int = 1,
        dtype=np.float64) -> np.ndarray:
    """`count` Gaussian random fields on the N^3 cell grid of the unit cube,
    squared-exponential covariance sigma^2 exp(-r^2 / (2 corr_len^2)).

    White noise (numpy default_rng(seed), drawn on the periodic grid of edge
    pad * N and spacing 1/N) is convolved by FFT with exp(-r^2 / corr_len^2),
    whose self-convolution is the squared-exponential kernel, and scaled by
    the filter's L2 norm so that each point has variance sigma^2; the first
    N^3 points are returned.  pad = 1 gives a periodic field; pad = 2 removes
    the wrap-around (for lags up to N cells the periodic distance on the
    padded grid is the true distance).  Returns count x N^3 (lexicographic, i
    fastest) in `dtype` (float32 halves the work of large batches)."""
    import scipy.fft as sfft
    M = N * pad
    h = 1.0 / N
    d = np.minimum(np.arange(M), M - np.arange(M)) * h          # periodic distance
    r2 = d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2
    g = np.exp(-r2 / corr_len ** 2).astype(dtype)
    G = sfft.rfftn(g, workers=-1)
    scale = sigma / np.sqrt((g.astype(np.float64) ** 2).sum())
    w = np.random.default_rng(seed).standard_normal((count, M, M, M), dtype=dtype)
    f = sfft.irfftn(sfft.rfftn(w, axes=(1, 2, 3), workers=-1) * G, s=(M, M, M), axes=(1, 2, 3),
                    workers=-1)
    f = f[:, :N, :N, :N] * dtype(scale)
    return np.ascontiguousarray(f.reshape(count, -1), dtype=dtype)


# (cin, cout) of the warm-start network's 13 convolutions, in the order of its
# flat parameter vector (per layer W[cout][27][cin], then b[cout]).
NET_LAYERS = [(8, 8), (8, 8), (8, 16), (16, 16), (16, 16), (16, 16), (16, 16), (16, 16), (16, 16),
              (16, 16), (16, 8), (8, 8), (8, 8)]


def net_init(seed: int) -> np.ndarray:
    """He-normal initial weights of the warm-start network (std sqrt(2 / fan_in),
    fan_in = 27 x used input channels; the last, linear layer sqrt(1 / fan_in)),
    zero biases.  The first layer uses 2 of its 8 input channels and the last
    1 of its 8 outputs; the other weights there start (and stay) zero."""
    rng = np.random.default_rng(seed)
    out = []
    last = len(NET_LAYERS) - 1
    for l, (ci, co) in enumerate(NET_LAYERS):
        ci_used = 2 if l == 0 else ci
        std = np.sqrt((1.0 if l == last else 2.0) / (27 * ci_used))
        W = rng.standard_normal((co, 27, ci)) * std
        if l == 0:
            W[:, :, 2:] = 0.0
        if l == last:
            W[1:] = 0.0
        out.append(W.reshape(-1))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def batch_spec(count: int = 64, seed: int = 2, edge_lo: int = 16, edge_hi: int = 96, m_max: int = 32):
    """Sizes of a batch of independent systems: per system s a grid edge
    drawn uniformly from edge_lo..edge_hi and a column count from 1..m_max
    (numpy default_rng(seed)).  Returns a list of (edge, m)."""
    rng = np.random.default_rng(seed)
    edges = rng.integers(edge_lo, edge_hi + 1, size=count)
    ms = rng.integers(1, m_max + 1, size=count)
    return [(int(e), int(m)) for e, m in zip(edges, ms)]


def batch_system(edge: int, m: int, s: int, sigma: float = 0.5):
    """System s of a batch: 7-point finite-volume diffusion on an edge^3 grid
    with i.i.d. lognormal cell coefficients (sigma, seed 100 + s) and an
    n x m block of uniform[-1, 1) right-hand sides (seed 1000 + s)."""
    A = diffusion7(edge, lognormal_cells(edge, sigma, 100 + s))
    return A, rhs_uniform(A.n, m, 1000 + s)


def rhs_uniform(n: int, m: int, seed: int = 0, m_draw: int | None = None) -> np.ndarray:
    """n x m row-major block with entries i.i.d. uniform[-1, 1).

    With ``m_draw`` the generator draws an n x m_draw block and the first m
    columns are returned, so an m-sweep shares its columns across m."""
    md = m if m_draw is None else m_draw
    if m > md:
        raise ValueError("m > m_draw")
    B = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, md))
    return np.ascontiguousarray(B[:, :m])


def csr_from_dense(A: np.ndarray) -> CSR:
    """CSR of a dense square matrix, keeping its nonzeros and its diagonal."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    mask = (A != 0.0) | np.eye(n, dtype=bool)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum(mask.sum(axis=1))
    rows, cols = np.nonzero(mask)
    return CSR(n, rowptr, cols.astype(np.int32), A[rows, cols].astype(np.float64))


def grid_n(N: int) -> int:
    return N * N * N
