"""GPU parity of the reduced-precision preconditioner (paper Sec. 2.3,
"mixed-precision") against the oracle's FP32 / bf16 V-cycle, and of the
FP64 outer solves around it against the FP64 oracle solution.

Tolerances: both sides compute the FP32 V-cycle from identical FP32 / bf16
data; they differ in FP32 rounding (fused multiply-adds, the order of the
Chebyshev coefficient products), so per-column ||g - o|| / ||o|| <= 2e-5.
Solves: true residual <= 1e-8 per column (checked in FP64 by the oracle),
iteration counts within +-1 of the oracle's reduced-precision solve."""
import numpy as np
import pytest

import oracle
from paper_2103_07329_gb300 import binding as B
from paper_2103_07329_gb300 import build as build_mod
from paper_2103_07329_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build_mod.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def colrel(g, o):
    return np.linalg.norm(g - o, axis=0) / np.linalg.norm(o, axis=0)


_cache = {}


def pair(key):
    if key not in _cache:
        if key == "p7_32":
            A = P.poisson7(32)
        elif key == "var_24":
            A = P.diffusion7(24, P.lognormal_cells(24, 1.0, 1))
        else:
            A = P.poisson27(16)
        _cache[key] = (A, B.Hierarchy(A), oracle.Hierarchy(A))
    return _cache[key]


@pytest.mark.parametrize("key", ["p7_32", "var_24", "p27_16"])
@pytest.mark.parametrize("prec", [B.PREC_FP32, B.PREC_BF16])
@pytest.mark.parametrize("m", [1, 4, 32])
def test_reduced_vcycle_parity(key, prec, m):
    A, g, o = pair(key)
    Bm = P.rhs_uniform(A.n, m, 0, m_draw=32)
    X = torch.empty((A.n, m), dtype=torch.float64, device="cuda")
    g.vcycle_precond(prec, dev(Bm), X)
    ref = o.vcycle_prec(prec, Bm)
    assert colrel(X.cpu().numpy(), ref).max() <= 2e-5


@pytest.mark.parametrize("key", ["p7_32", "var_24"])
@pytest.mark.parametrize("prec", [B.PREC_FP32, B.PREC_BF16])
@pytest.mark.parametrize("method", [B.PCG, B.BICGSTAB])
def test_reduced_precision_solve(key, prec, method):
    A, g, o = pair(key)
    Bm = P.rhs_uniform(A.n, 8, 0, m_draw=32)
    X = torch.empty_like(dev(Bm))
    st = g.solve(dev(Bm), X, tol=1e-8, maxit=100, method=method, precond=prec)
    Xg = X.cpu().numpy()
    rr = np.linalg.norm(Bm - oracle.spmm(A, Xg), axis=0) / np.linalg.norm(Bm, axis=0)
    assert st.rc == 0 and np.all(st.status == 0)
    assert np.all(rr <= 1e-8), rr
    ref = (o.pcg if method == B.PCG else o.bicgstab)(Bm, tol=1e-8, prec=prec)
    assert np.all(np.abs(st.iters - ref.iters) <= 1), (st.iters, ref.iters)
    # error against the FP64 oracle solution
    x64 = (o.pcg if method == B.PCG else o.bicgstab)(Bm, tol=1e-8).X
    assert colrel(Xg, x64).max() <= 1e-6


def test_reduced_precision_edge_cases():
    A, g, o = pair("p7_32")
    Bm = P.rhs_uniform(A.n, 3, 4, m_draw=32)
    Bm[:, 1] = 0.0
    X = torch.full((A.n, 3), 5.0, dtype=torch.float64, device="cuda")
    st = g.solve(dev(Bm), X, precond=B.PREC_FP32)
    assert st.iters[1] == 0 and torch.all(X[:, 1] == 0)
    Bm[0, 0] = np.inf
    X = torch.full((A.n, 3), 5.0, dtype=torch.float64, device="cuda")
    with pytest.raises(B.XamgError) as e:
        g.solve(dev(Bm), X, precond=B.PREC_BF16)
    assert e.value.code == B.ERR_NONFINITE and torch.all(X == 5.0)
    with pytest.raises(B.XamgError):
        g.solve(dev(Bm), X, precond=7)


def _long_range(N, *strides):
    """7-point Poisson plus a symmetric coupling of every row to the rows
    `stride` away (diagonally dominant, so still SPD).  Each stride adds two
    column clusters far from the row's own: one stride beyond 65536 needs
    three 16-bit segments per row tile, two such strides five, more than the
    segmented form holds."""
    import scipy.sparse as sp
    A0 = P.poisson7(N)
    M = sp.csr_matrix((A0.val, A0.col, A0.rowptr), shape=(A0.n, A0.n))
    n = A0.n
    for stride in strides:
        E = sp.diags([np.full(n - stride, -0.1), np.full(n - stride, -0.1)], [stride, -stride],
                     shape=(n, n))
        M = M + E + sp.identity(n) * 0.2
    M = M.tocsr()
    M.sort_indices()
    return P.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data)


@pytest.mark.parametrize("which", ["windows", "segments", "fallback"])
def test_bf16_index_compression_paths(which):
    # n = 262144 spans four 65536-column windows: the 7-point rows fit one
    # 16-bit segment per tile, the one-stride long-range rows three; the
    # two-stride rows of the 72^3 grid need five and keep 32-bit indices.  All
    # must match the oracle's bf16 V-cycle.
    A = {"windows": P.poisson7(64), "segments": _long_range(64, 70000),
         "fallback": _long_range(72, 70000, 140000)}[which]
    g, o = B.Hierarchy(A), oracle.Hierarchy(A)
    g.set_index16(True)
    Bm = P.rhs_uniform(A.n, 8, 0, m_draw=32)
    X = torch.empty((A.n, 8), dtype=torch.float64, device="cuda")
    g.vcycle_precond(B.PREC_BF16, dev(Bm), X)
    assert colrel(X.cpu().numpy(), o.vcycle_prec(B.PREC_BF16, Bm)).max() <= 2e-5
    st = g.solve(dev(Bm), X, precond=B.PREC_BF16)
    rr = np.linalg.norm(Bm - oracle.spmm(A, X.cpu().numpy()), axis=0) / np.linalg.norm(Bm, axis=0)
    assert st.rc == 0 and np.all(rr <= 1e-8)


@pytest.mark.parametrize("prec", [B.PREC_FP64, B.PREC_FP32, B.PREC_BF16])
@pytest.mark.parametrize("m", [1, 2, 16, 32])
def test_autotuned_splits_keep_the_results(prec, m):
    # a fresh hierarchy: tuning stores its choices in the hierarchy
    A = P.diffusion7(24, P.lognormal_cells(24, 1.0, 1))
    g = B.Hierarchy(A)
    Bm = P.rhs_uniform(A.n, m, 0, m_draw=32)
    X0 = torch.empty_like(dev(Bm))
    s0 = g.solve(dev(Bm), X0, tol=1e-8, maxit=100, precond=prec)
    z0 = torch.empty_like(X0)
    g.vcycle_precond(prec, dev(Bm), z0)
    tuned, wide = g.autotune(m, prec)
    assert tuned == 3 * (g.levels - 1) and 0 <= wide <= tuned
    X1 = torch.empty_like(X0)
    s1 = g.solve(dev(Bm), X1, tol=1e-8, maxit=100, precond=prec)
    z1 = torch.empty_like(X0)
    g.vcycle_precond(prec, dev(Bm), z1)
    # another split only reorders each row's sum
    assert colrel(z1.cpu().numpy(), z0.cpu().numpy()).max() <= (1e-12 if prec == B.PREC_FP64 else 2e-5)
    assert s1.rc == 0 and np.all(np.abs(s1.iters - s0.iters) <= 1)
    rr = np.linalg.norm(Bm - oracle.spmm(A, X1.cpu().numpy()), axis=0) / np.linalg.norm(Bm, axis=0)
    assert np.all(rr <= 1e-8)
    with pytest.raises(B.XamgError):
        g.autotune(m, 7)


@pytest.mark.parametrize("prec", [B.PREC_FP32, B.PREC_BF16])
@pytest.mark.parametrize("cand", [0, 1, 2, 3, 4, 5, 6])
def test_m1_splits_of_the_reduced_precision_vcycle(prec, cand):
    # every product of the FP32 / bf16 V-cycle at m = 1 forced onto one split:
    # the result moves only by the order of each row's FP32 sums
    A = P.diffusion7(25, P.lognormal_cells(25, 1.0, 1))
    g = B.Hierarchy(A)
    Bm = P.rhs_uniform(A.n, 1, 0, m_draw=32)
    z0 = torch.empty_like(dev(Bm))
    g.vcycle_precond(prec, dev(Bm), z0)
    for l in range(g.levels):
        for which in (0, 1, 2):
            if which == 0 or l + 1 < g.levels:
                g.set_split(1, prec, l, which, cand)
    z1 = torch.empty_like(z0)
    g.vcycle_precond(prec, dev(Bm), z1)
    assert colrel(z1.cpu().numpy(), z0.cpu().numpy()).max() <= 2e-5
    X = torch.empty_like(z0)
    s = g.solve(dev(Bm), X, tol=1e-8, maxit=100, precond=prec)
    rr = np.linalg.norm(Bm - oracle.spmm(A, X.cpu().numpy()), axis=0) / np.linalg.norm(Bm, axis=0)
    assert s.rc == 0 and np.all(rr <= 1e-8)


# ---- products and cycles that must equal the oracle bit for bit ----------
#
# The FP32 row kernels round where the reduced-precision cycle is defined to
# round (one rounding per term of a row sum, in storage order; one per
# elementwise operation), so with the storage-order split on every product
# (tuning candidate 0: a lane group per row, or at m = 1 the stream kernel
# with one lane per row) the GPU and the oracle compute identical bits.  A
# kernel that accumulated in FP64, fused differently or summed in another
# order would fail these tests (the FP32-vs-FP64 gap of the cycle is 1-2e-7,
# and merely fusing the products differently moves it by 1e-7).

def _storage_order(g, m, prec, cand=0):
    # candidate 0: the register narrow split; 2 (FP32 blocks of >= 8
    # columns): the same sums with the operand rows staged through shared
    # memory (operators whose row groups exceed its window fall back to 0);
    # 2 for 2 and 4 columns: the stream kernel with one lane per row
    for l in range(g.levels):
        for which in (0, 1, 2):
            if which == 0 or l + 1 < g.levels:
                g.set_split(m, prec, l, which, cand)


def _fp32_block(rows, m, seed):
    return np.random.default_rng(seed).standard_normal((rows, m)).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("key", ["p7_32", "var_24", "p27_16"])
@pytest.mark.parametrize("prec", [B.PREC_FP32, B.PREC_BF16])
@pytest.mark.parametrize("m,cand", [(1, 0), (4, 0), (32, 0), (8, 2), (16, 2), (32, 2), (2, 2), (4, 2)])
def test_reduced_products_bitwise_in_storage_order(key, prec, m, cand):
    A, _, o = pair(key)
    g = B.Hierarchy(A)
    _storage_order(g, m, prec, cand)
    for l in range(g.levels):
        n = g.level_info(l)[0]
        nc = g.level_info(l + 1)[0] if l + 1 < g.levels else 0
        for which in ((0, 1, 2) if l + 1 < g.levels else (0,)):
            cols, rows = {0: (n, n), 1: (nc, n), 2: (n, nc)}[which]
            X = _fp32_block(cols, m, 100 * l + which)
            Y = torch.empty((rows, m), dtype=torch.float64, device="cuda")
            g.spmm_precond(prec, l, which, dev(X), Y)
            ref = o.spmm_f(l, which, X, bf16=(prec == B.PREC_BF16 and which == 0))
            assert np.array_equal(Y.cpu().numpy(), ref.astype(np.float64)), (l, which)


@pytest.mark.parametrize("key", ["p7_32", "var_24", "p27_16"])
@pytest.mark.parametrize("prec", [B.PREC_FP32, B.PREC_BF16])
@pytest.mark.parametrize("m,cand", [(1, 0), (4, 0), (32, 0), (8, 2), (16, 2), (32, 2), (2, 2), (4, 2)])
def test_reduced_vcycle_bitwise_in_storage_order(key, prec, m, cand):
    A, _, o = pair(key)
    g = B.Hierarchy(A)
    _storage_order(g, m, prec, cand)
    Bm = P.rhs_uniform(A.n, m, 0, m_draw=32)
    X = torch.empty((A.n, m), dtype=torch.float64, device="cuda")
    g.vcycle_precond(prec, dev(Bm), X)
    Xg = X.cpu().numpy()
    ref = o.vcycle_prec(prec, Bm)
    assert np.array_equal(Xg, ref), colrel(Xg, ref).max()
    # and the cycle is genuinely reduced precision: it sits well away from
    # the FP64 cycle (FP32: 1e-7 relative; bf16 values: 1e-3)
    X64 = torch.empty_like(X)
    g.vcycle(dev(Bm), X64)
    gap = colrel(Xg, X64.cpu().numpy()).min()
    assert gap > (3e-8 if prec == B.PREC_FP32 else 1e-4), gap


@pytest.mark.parametrize("key", ["p7_32", "p27_16"])
@pytest.mark.parametrize("prec", [B.PREC_FP32, B.PREC_BF16])
@pytest.mark.parametrize("m", [4, 32])
def test_reduced_products_within_summation_bound_every_split(key, prec, m):
    # the default and the one-row-per-warp splits add a row's terms in another
    # order: each result is within the FP32 summation bound of the oracle's,
    # 2 gamma_k sum |m_ik| |x_k| (k terms, both sides within gamma_k of the
    # exact sum of the same stored values)
    import scipy.sparse as sp
    A, _, o = pair(key)
    g = B.Hierarchy(A)
    u = 2.0 ** -24
    for cand in (-1, 1):
        for l in range(g.levels):
            for which in ((0, 1, 2) if l + 1 < g.levels else (0,)):
                g.set_split(m, prec, l, which, cand)
                rp, ci, v = _ops(o, l)[which]
                rows, cols = len(rp) - 1, (o.level(l + 1).n if which == 1 else o.level(l).n)
                X = _fp32_block(cols, m, 7 * l + which)
                Y = torch.empty((rows, m), dtype=torch.float64, device="cuda")
                g.spmm_precond(prec, l, which, dev(X), Y)
                ref = o.spmm_f(l, which, X, bf16=(prec == B.PREC_BF16 and which == 0)).astype(np.float64)
                Mabs = sp.csr_matrix((np.abs(v) * (1.01 if prec == B.PREC_BF16 else 1.0), ci, rp),
                                     shape=(rows, cols))
                k = int(np.diff(rp).max()) + 1
                bound = 2 * k * u / (1 - k * u) * (Mabs @ np.abs(X))
                assert np.all(np.abs(Y.cpu().numpy() - ref) <= bound + 1e-40), (cand, l, which)


def _ops(o, l):
    lv = o.level(l)
    return {0: lv.A, 1: lv.P if l + 1 < o.nlev else None, 2: lv.R if l + 1 < o.nlev else None}


@pytest.mark.parametrize("kind", ["p7_64", "long_70000"])
@pytest.mark.parametrize("prec", [B.PREC_FP32, B.PREC_BF16])
@pytest.mark.parametrize("m", [2, 4, 32])
def test_index16_products_and_cycle_equal_index32(kind, prec, m):
    # 16-bit column offsets decode exactly: with them on or off every product
    # and the whole cycle give identical bits.  n = 262144 spans four 65536
    # windows; the 7-point tiles take one segment, the long-range ones three
    A = P.poisson7(64) if kind == "p7_64" else _long_range(64, 70000)
    g = B.Hierarchy(A)
    masks = [g.index16_info(l) for l in range(g.levels)]
    assert masks[0] & 1 and masks[0] & 2 and masks[0] & 4, masks
    Bm = P.rhs_uniform(A.n, m, 0, m_draw=32)
    outs = []
    for on in (True, False):
        g.set_index16(on)
        ys = []
        for l in range(g.levels - 1):
            for which in (0, 1, 2):
                lv = g.level_info(l)[0]
                nc = g.level_info(l + 1)[0]
                cols, rows = {0: (lv, lv), 1: (nc, lv), 2: (lv, nc)}[which]
                X = _fp32_block(cols, m, l * 3 + which)
                Y = torch.empty((rows, m), dtype=torch.float64, device="cuda")
                g.spmm_precond(prec, l, which, dev(X), Y)
                ys.append(Y.cpu().numpy())
        Z = torch.empty((A.n, m), dtype=torch.float64, device="cuda")
        g.vcycle_precond(prec, dev(Bm), Z)
        ys.append(Z.cpu().numpy())
        outs.append(ys)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_index16_falls_back_where_rows_do_not_fit():
    # two long-range strides need five segments per tile in the middle rows
    # (n = 373248 > 2 x 140000): level 0's A keeps 32-bit indices, and its
    # products still match the oracle's
    A = _long_range(72, 70000, 140000)
    g, o = B.Hierarchy(A), oracle.Hierarchy(A)
    assert not (g.index16_info(0) & 1)
    _storage_order(g, 8, B.PREC_FP32)
    X = _fp32_block(A.n, 8, 3)
    Y = torch.empty((A.n, 8), dtype=torch.float64, device="cuda")
    g.spmm_precond(B.PREC_FP32, 0, 0, dev(X), Y)
    assert np.array_equal(Y.cpu().numpy(), o.spmm_f(0, 0, X).astype(np.float64))


def test_third_split_candidate_exists_where_documented():
    # candidate 2: the staged narrow split for FP32 blocks of >= 8 columns, the
    # stream kernel for 2 and 4 columns, the pipelined narrow split for FP64
    # blocks of 8 or more columns (which also have 3 and 4, two columns per
    # lane)
    g = B.Hierarchy(P.poisson7(12))
    for m, prec, cand in [(2, B.PREC_FP32, 2), (4, B.PREC_FP32, 2), (8, B.PREC_BF16, 2),
                          (32, B.PREC_FP32, 2), (2, B.PREC_FP64, 2), (4, B.PREC_FP64, 2),
                          (8, B.PREC_FP64, 4), (16, B.PREC_FP64, 4), (32, B.PREC_FP64, 4)]:
        for c in range(2, cand + 1):
            g.set_split(m, prec, 0, 0, c)
        g.set_split(m, prec, 0, 0, -1)
    for m, prec, cand in [(32, B.PREC_FP64, 5), (8, B.PREC_FP64, 5), (32, B.PREC_FP32, 3),
                          (4, B.PREC_FP64, 3)]:
        with pytest.raises(B.XamgError):
            g.set_split(m, prec, 0, 0, cand)
