"""GPU parity: every step of the solve phase, called through the C ABI, against
the CPU oracle on the same seeded inputs.

Tolerances (FP64 on both sides; the products agree up to summation order and
fused multiply-adds):
  * SpMM on integer-valued data: bitwise (every partial sum is exact);
  * SpMM, smoother, coarse solve, V-cycle: per-column ||g - o|| / ||o|| <= 1e-12;
  * solves: true residual <= 1e-8 per column, iteration counts within +-1.
"""
import numpy as np
import pytest

import oracle
from paper_2103_07329_gb300 import binding as B
from paper_2103_07329_gb300 import build as build_mod
from paper_2103_07329_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    build_mod.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def colrel(g, o):
    g = np.asarray(g).reshape(o.shape[0], -1)
    o = o.reshape(o.shape[0], -1)
    num = np.linalg.norm(g - o, axis=0)
    den = np.linalg.norm(o, axis=0)
    return np.where(den > 0, num / np.where(den > 0, den, 1), num)


def csr_of(t, rows):
    rp, ci, v = t
    return P.CSR(rows, rp, ci, v)


class Pair:
    """Library and oracle hierarchies of one matrix."""

    def __init__(self, A, **kw):
        self.A = A
        self.g = B.Hierarchy(A, **kw)
        self.o = oracle.Hierarchy(A, **kw)


_pairs = {}


def pair(name, N, **kw):
    key = (name, N, tuple(sorted(kw.items())))
    if key not in _pairs:
        A = P.poisson7(N) if name == "p7" else P.poisson27(N)
        _pairs[key] = Pair(A, **kw)
    return _pairs[key]


@pytest.fixture(scope="module")
def cfg0():
    return pair("p7", 32)


# ---------------------------------------------------------------- SpMM
@pytest.mark.parametrize("m", [1, 2, 3, 4, 8, 16, 32])
def test_spmm_fine_level_integer_bitwise(cfg0, m):
    A = cfg0.A
    X = np.random.default_rng(m).integers(-1000, 1001, size=(A.n, m)).astype(np.float64)
    Y = torch.empty((A.n, m), dtype=torch.float64, device="cuda")
    cfg0.g.spmm(0, 0, dev(X), Y)
    assert np.array_equal(Y.cpu().numpy(), oracle.spmm(A, X))


@pytest.mark.parametrize("m", [1, 4, 5, 32])
def test_spmm_all_levels_and_operators(cfg0, m):
    rng = np.random.default_rng(10 + m)
    for l in range(cfg0.o.nlev):
        lv = cfg0.o.level(l)
        ops = [(0, csr_of(lv.A, lv.n), lv.n)]
        if lv.P is not None:
            nc = cfg0.o.level(l + 1).n
            ops += [(1, P.CSR(lv.n, *lv.P), nc), (2, P.CSR(nc, *lv.R), lv.n)]
        for which, M, ncols in ops:
            X = rng.uniform(-1, 1, size=(ncols, m))
            Y = torch.empty((M.n, m), dtype=torch.float64, device="cuda")
            cfg0.g.spmm(l, which, dev(X), Y)
            ref = oracle.spmm(M, X, ncols=ncols)
            assert colrel(Y.cpu().numpy(), ref).max() <= RTOL, (l, which)


@pytest.mark.parametrize("N", [5, 17, 33])
def test_spmm_ragged_sizes(N):
    # n not a multiple of any tile: 125, 4913, 35937 rows
    pr = pair("p7", N)
    for m in (1, 2, 32):
        X = np.random.default_rng(N).integers(-50, 51, size=(pr.A.n, m)).astype(np.float64)
        Y = torch.empty((pr.A.n, m), dtype=torch.float64, device="cuda")
        pr.g.spmm(0, 0, dev(X), Y)
        assert np.array_equal(Y.cpu().numpy(), oracle.spmm(pr.A, X))


def test_spmm_27pt_long_rows():
    pr = pair("p27", 20)
    for m in (1, 8):
        X = np.random.default_rng(3).integers(-99, 100, size=(pr.A.n, m)).astype(np.float64)
        Y = torch.empty((pr.A.n, m), dtype=torch.float64, device="cuda")
        pr.g.spmm(0, 0, dev(X), Y)
        assert np.array_equal(Y.cpu().numpy(), oracle.spmm(pr.A, X))


@pytest.mark.parametrize("cand", [0, 1, 2, 3, 4, 5, 6])
def test_spmm_m1_every_split(cand):
    # m = 1 under each row split (stream kernel with the short / long window,
    # 16 lanes per row) on every level and operator: short rows, 27-point
    # rows, the dense Galerkin levels, and a ragged last chunk (33^3 rows)
    for name, N in (("p7", 33), ("p27", 20)):
        pr = pair(name, N)
        rng = np.random.default_rng(cand)
        for l in range(pr.o.nlev):
            lv = pr.o.level(l)
            ops = [(0, csr_of(lv.A, lv.n), lv.n)]
            if lv.P is not None:
                nc = pr.o.level(l + 1).n
                ops += [(1, P.CSR(lv.n, *lv.P), nc), (2, P.CSR(nc, *lv.R), lv.n)]
            for which, M, ncols in ops:
                pr.g.set_split(1, B.PREC_FP64, l, which, cand)
                try:
                    X = rng.integers(-50, 51, size=(ncols, 1)).astype(np.float64)
                    Y = torch.empty((M.n, 1), dtype=torch.float64, device="cuda")
                    pr.g.spmm(l, which, dev(X), Y)
                    ref = oracle.spmm(M, X, ncols=ncols)
                    if l == 0 and which == 0:
                        assert np.array_equal(Y.cpu().numpy(), ref), (name, l, which)
                    else:
                        assert colrel(Y.cpu().numpy(), ref).max() <= RTOL, (name, l, which)
                finally:
                    pr.g.set_split(1, B.PREC_FP64, l, which, -1)


@pytest.mark.parametrize("m", [8, 16, 32])
@pytest.mark.parametrize("cand", [0, 1, 2, 3, 4])
def test_spmm_wide_blocks_every_split(m, cand):
    # FP64 blocks of 8, 16 and 32 columns under every split on every level and
    # operator (32 columns, split 1: four warps share a row; split 2: the
    # pipelined narrow split; 3 and 4: the narrow split and its pipelined
    # form with two columns per lane), the 7-point and 27-point hierarchies
    # with their dense Galerkin levels
    for name, N in (("p7", 33), ("p27", 20)):
        pr = pair(name, N)
        rng = np.random.default_rng(100 + cand)
        for l in range(pr.o.nlev):
            lv = pr.o.level(l)
            ops = [(0, csr_of(lv.A, lv.n), lv.n)]
            if lv.P is not None:
                nc = pr.o.level(l + 1).n
                ops += [(1, P.CSR(lv.n, *lv.P), nc), (2, P.CSR(nc, *lv.R), lv.n)]
            for which, M, ncols in ops:
                pr.g.set_split(m, B.PREC_FP64, l, which, cand)
                try:
                    X = rng.integers(-50, 51, size=(ncols, m)).astype(np.float64)
                    Y = torch.empty((M.n, m), dtype=torch.float64, device="cuda")
                    pr.g.spmm(l, which, dev(X), Y)
                    ref = oracle.spmm(M, X, ncols=ncols)
                    if l == 0 and which == 0:
                        assert np.array_equal(Y.cpu().numpy(), ref), (name, l, which)
                    else:
                        assert colrel(Y.cpu().numpy(), ref).max() <= RTOL, (name, l, which)
                finally:
                    pr.g.set_split(m, B.PREC_FP64, l, which, -1)


@pytest.mark.parametrize("m", [2, 4, 8, 16, 32])
def test_alternative_fp64_splits_are_bitwise_the_narrow_split(m):
    # FP64 candidate 2 -- for 2- and 4-column blocks the stream kernel (one
    # lane per row over the warp's staged entries), for 8 to 32 columns the
    # software-pipelined narrow split -- and for 8 to 32 columns candidates
    # 3 and 4 (two columns per lane) add each column's products in storage
    # order like the narrow split (candidate 0), on every level and operator,
    # so products and the V-cycle agree bit for bit; the solve's fused dot
    # products reduce in another lane and block order, so its iterates agree
    # to rounding
    for name, N in (("p7", 33), ("p27", 20)):
        pr = pair(name, N)
        rng = np.random.default_rng(7)
        outs = []
        for cand in ((0, 2) if m <= 4 else (0, 2, 3, 4)):
            for l in range(pr.o.nlev):
                for which in (0, 1, 2):
                    if which == 0 or l + 1 < pr.o.nlev:
                        pr.g.set_split(m, B.PREC_FP64, l, which, cand)
            ys = []
            for l in range(pr.o.nlev):
                lv = pr.o.level(l)
                ops = [(0, lv.n, lv.n)]
                if lv.P is not None:
                    nc = pr.o.level(l + 1).n
                    ops += [(1, lv.n, nc), (2, nc, lv.n)]
                for which, rows, ncols in ops:
                    X = np.random.default_rng(10 * l + which).standard_normal((ncols, m))
                    Y = torch.empty((rows, m), dtype=torch.float64, device="cuda")
                    pr.g.spmm(l, which, dev(X), Y)
                    ys.append(Y.cpu().numpy())
            Bm = P.rhs_uniform(pr.A.n, m, 0)
            Z = torch.empty((pr.A.n, m), dtype=torch.float64, device="cuda")
            pr.g.vcycle(dev(Bm), Z)
            ys.append(Z.cpu().numpy())
            st = pr.g.solve(dev(Bm), Z, tol=1e-8, maxit=100)
            assert st.rc == 0
            outs.append((ys, Z.cpu().numpy(), st.iters.copy()))
        for l in range(pr.o.nlev):
            for which in (0, 1, 2):
                if which == 0 or l + 1 < pr.o.nlev:
                    pr.g.set_split(m, B.PREC_FP64, l, which, -1)
        ya, xa, ia = outs[0]
        for yb, xb, ib in outs[1:]:
            for a, b in zip(ya, yb):
                assert np.array_equal(a, b), name
            assert np.array_equal(ia, ib) and colrel(xa, xb).max() <= 1e-12


def test_set_split_rejects_bad_arguments(cfg0):
    g = cfg0.g
    L = cfg0.o.nlev
    for args in [(1, B.PREC_FP64, 0, 0, 7), (8, B.PREC_FP64, 0, 0, 5), (2, B.PREC_FP64, 0, 0, 3),
                 (1, 9, 0, 0, 0),
                 (1, B.PREC_FP64, L, 0, 0), (1, B.PREC_FP64, L - 1, 1, 0), (1, B.PREC_FP64, 0, 3, 0),
                 (0, B.PREC_FP64, 0, 0, 0), (33, B.PREC_FP64, 0, 0, 0), (1, B.PREC_FP64, 0, 0, -2)]:
        with pytest.raises(B.XamgError):
            g.set_split(*args)


# ---------------------------------------------------------------- smoother / coarse / V-cycle
@pytest.mark.parametrize("m", [1, 4, 7])
def test_chebyshev_pre_and_post(cfg0, m):
    rng = np.random.default_rng(20 + m)
    for l in range(cfg0.o.nlev - 1):
        n = cfg0.o.level(l).n
        Bm = rng.uniform(-1, 1, size=(n, m))
        X = torch.empty((n, m), dtype=torch.float64, device="cuda")
        R = torch.empty((n, m), dtype=torch.float64, device="cuda")
        cfg0.g.smooth(l, dev(Bm), X, R, x_zero=True)
        xo, ro = cfg0.o.cheb_smooth(l, Bm)
        assert colrel(X.cpu().numpy(), xo).max() <= RTOL
        assert colrel(R.cpu().numpy(), ro).max() <= 1e-11
        X0 = rng.uniform(-1, 1, size=(n, m))
        X = dev(X0)
        cfg0.g.smooth(l, dev(Bm), X, None, x_zero=False)
        xo, _ = cfg0.o.cheb_smooth(l, Bm, X0=X0, want_residual=False)
        assert colrel(X.cpu().numpy(), xo).max() <= RTOL


def test_coarse_solve(cfg0):
    lu, piv = cfg0.o.coarse_lu()
    nc = lu.shape[0]
    Bm = np.random.default_rng(1).uniform(-1, 1, size=(nc, 6))
    X = torch.empty((nc, 6), dtype=torch.float64, device="cuda")
    cfg0.g.coarse_solve(dev(Bm), X)
    ref = oracle.lu_solve(lu, piv, Bm)
    assert colrel(X.cpu().numpy(), ref).max() <= RTOL


@pytest.mark.parametrize("m", [1, 4, 32])
def test_vcycle_parity(cfg0, m):
    Bm = P.rhs_uniform(cfg0.A.n, m, 0)
    X = torch.empty_like(dev(Bm))
    cfg0.g.vcycle(dev(Bm), X)
    assert colrel(X.cpu().numpy(), cfg0.o.vcycle(Bm)).max() <= RTOL


def test_vcycle_parity_27pt():
    pr = pair("p27", 16)
    Bm = P.rhs_uniform(pr.A.n, 3, 0)
    X = torch.empty_like(dev(Bm))
    pr.g.vcycle(dev(Bm), X)
    assert colrel(X.cpu().numpy(), pr.o.vcycle(Bm)).max() <= RTOL


def test_vcycle_single_level_is_exact():
    pr = pair("p7", 4)          # n = 64 <= max_coarse: one level
    assert pr.g.levels == 1
    Bm = P.rhs_uniform(pr.A.n, 2, 0)
    X = torch.empty_like(dev(Bm))
    pr.g.vcycle(dev(Bm), X)
    assert colrel(X.cpu().numpy(), pr.o.vcycle(Bm)).max() <= RTOL


# ---------------------------------------------------------------- solves
def true_relres(A, Bm, X):
    R = Bm - oracle.spmm(A, X)
    return np.linalg.norm(R, axis=0) / np.linalg.norm(Bm, axis=0)


@pytest.mark.parametrize("method", [B.PCG, B.BICGSTAB])
def test_solve_cfg0(cfg0, method):
    Bm = P.rhs_uniform(cfg0.A.n, 4, 0)
    X = torch.empty_like(dev(Bm))
    st = cfg0.g.solve(dev(Bm), X, tol=1e-8, maxit=100, method=method)
    ref = cfg0.o.pcg(Bm) if method == B.PCG else cfg0.o.bicgstab(Bm)
    assert st.rc == 0 and np.all(st.status == 0)
    Xg = X.cpu().numpy()
    rr = true_relres(cfg0.A, Bm, Xg)
    assert np.all(rr <= 1e-8), rr
    assert np.allclose(st.relres, rr, rtol=1e-6, atol=0)
    assert np.all(np.abs(st.iters - ref.iters) <= 1), (st.iters, ref.iters)
    assert colrel(Xg, ref.X).max() <= 1e-6


@pytest.mark.parametrize("method", [B.PCG, B.BICGSTAB])
def test_solve_27pt(method):
    pr = pair("p27", 24)
    Bm = P.rhs_uniform(pr.A.n, 5, 0)
    X = torch.empty_like(dev(Bm))
    st = pr.g.solve(dev(Bm), X, method=method)
    ref = pr.o.pcg(Bm) if method == B.PCG else pr.o.bicgstab(Bm)
    assert np.all(true_relres(pr.A, Bm, X.cpu().numpy()) <= 1e-8)
    assert np.all(np.abs(st.iters - ref.iters) <= 1)


def test_m1_equals_single_column(cfg0):
    Bm = P.rhs_uniform(cfg0.A.n, 4, 0)
    Xb = torch.empty_like(dev(Bm))
    sb = cfg0.g.solve(dev(Bm), Xb)
    for j in range(4):
        X1 = torch.empty((cfg0.A.n, 1), dtype=torch.float64, device="cuda")
        s1 = cfg0.g.solve(dev(Bm[:, j:j + 1]), X1)
        assert s1.iters[0] == sb.iters[j]
        assert colrel(X1.cpu().numpy(), Xb.cpu().numpy()[:, j:j + 1]).max() <= 1e-12


def test_repeatable_bits(cfg0):
    Bm = dev(P.rhs_uniform(cfg0.A.n, 8, 1))
    X1 = torch.empty_like(Bm)
    X2 = torch.empty_like(Bm)
    cfg0.g.solve(Bm, X1, method=B.BICGSTAB)
    cfg0.g.solve(Bm, X2, method=B.BICGSTAB)
    assert torch.equal(X1, X2)


def test_edge_cases(cfg0):
    n = cfg0.A.n
    Bm = P.rhs_uniform(n, 3, 2)
    Bm[:, 1] = 0.0
    X = torch.full((n, 3), 7.0, dtype=torch.float64, device="cuda")
    st = cfg0.g.solve(dev(Bm), X)
    Xg = X.cpu().numpy()
    assert st.iters[1] == 0 and np.all(Xg[:, 1] == 0.0) and st.status[1] == 0
    assert np.all(true_relres(cfg0.A, Bm[:, [0, 2]], Xg[:, [0, 2]]) <= 1e-8)
    # non-finite right-hand side: error, X untouched
    Bm[5, 2] = np.nan
    X = torch.full((n, 3), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(B.XamgError) as e:
        cfg0.g.solve(dev(Bm), X)
    assert e.value.code == B.ERR_NONFINITE
    assert torch.all(X == 7.0)
    # iteration limit
    Bm = P.rhs_uniform(n, 2, 3)
    st = cfg0.g.solve(dev(Bm), torch.empty((n, 2), dtype=torch.float64, device="cuda"),
                      tol=1e-14, maxit=2)
    assert st.rc == B.NOT_CONVERGED and np.all(st.status == 1) and np.all(st.iters == 2)
    ref = cfg0.o.pcg(Bm, tol=1e-14, maxit=2)
    assert np.all(ref.iters == 2)
    # bad arguments
    with pytest.raises(B.XamgError):
        cfg0.g.solve(dev(np.zeros((n, 33))), torch.empty((n, 33), dtype=torch.float64, device="cuda"))


def test_breakdown_on_a_negative_definite_matrix():
    # -A of the 7-point Laplacian: p^T A p < 0 for every p, so the first alpha
    # step flags every column as broken down (the reading of the breakdown
    # rule), X stays at its zero start, and the call returns XAMG_BREAKDOWN,
    # all as in the oracle (its coarsening stalls: one dense level)
    A = P.poisson7(8)
    An = P.CSR(A.n, A.rowptr, A.col, -A.val)
    g = B.Hierarchy(An)
    o = oracle.Hierarchy(An)
    Bm = P.rhs_uniform(A.n, 3, 1)
    X = torch.full((A.n, 3), 7.0, dtype=torch.float64, device="cuda")
    st = g.solve(dev(Bm), X, tol=1e-8, maxit=50)
    ref = o.pcg(Bm, 1e-8, 50)
    assert st.rc == B.BREAKDOWN
    assert np.array_equal(st.status, ref.status) and np.array_equal(st.iters, ref.iters)
    assert np.all(X.cpu().numpy() == 0.0)


def test_host_buffers_match_device(cfg0):
    Bm = P.rhs_uniform(cfg0.A.n, 4, 5)
    Xd = torch.empty_like(dev(Bm))
    sd = cfg0.g.solve(dev(Bm), Xd)
    Xh = np.empty_like(Bm)
    sh = cfg0.g.solve_host(Bm, Xh)
    assert np.array_equal(Xh, Xd.cpu().numpy())
    assert np.array_equal(sh.iters, sd.iters)


@pytest.mark.parametrize("method", [B.PCG, B.BICGSTAB])
def test_pinned_host_buffers_match_device(cfg0, method):
    # page-locked B and X: the solve reads and writes them directly (no
    # staging copies); the kernels are the same, so the bits are too, with
    # and without a starting guess; mixing a pinned and a pageable buffer
    # takes the staged path with the same result
    Bm = P.rhs_uniform(cfg0.A.n, 4, 7)
    Xd = torch.empty_like(dev(Bm))
    sd = cfg0.g.solve(dev(Bm), Xd, method=method)
    Bp = torch.from_numpy(Bm).pin_memory()
    Xp = torch.empty_like(Bp).pin_memory()
    sp = cfg0.g.solve_host(Bp.numpy(), Xp.numpy(), method=method)
    assert np.array_equal(Xp.numpy(), Xd.cpu().numpy()) and np.array_equal(sp.iters, sd.iters)
    X0 = 0.5 * Xd.cpu().numpy()
    Xd0 = dev(X0)
    sd0 = cfg0.g.solve(dev(Bm), Xd0, method=method, x0_given=True)
    Xp.copy_(torch.from_numpy(X0))
    sp0 = cfg0.g.solve_host(Bp.numpy(), Xp.numpy(), method=method, x0_given=True)
    assert np.array_equal(Xp.numpy(), Xd0.cpu().numpy()) and np.array_equal(sp0.iters, sd0.iters)
    Xh = np.empty_like(Bm)
    cfg0.g.solve_host(Bp.numpy(), Xh, method=method)
    assert np.array_equal(Xh, Xd.cpu().numpy())


@pytest.mark.parametrize("prec", [B.PREC_FP64, B.PREC_FP32, B.PREC_BF16])
def test_graph_replay_is_bitwise(prec):
    # the captured steady PCG iteration replays the same kernels with the
    # same arguments: X, iteration counts and residuals equal the uncaptured
    # solve bit for bit (first solve captures, second replays the cache); a
    # second tolerance keys its own graph; a maxit stop and a row-split
    # change (which drops the cache) keep the equality
    A = P.poisson7(20)
    g = B.Hierarchy(A)
    Bm = dev(P.rhs_uniform(A.n, 3, 11))

    def run(tol=1e-8, maxit=100, m=3):
        X = torch.empty_like(Bm[:, :m].contiguous())
        st = g.solve(Bm[:, :m].contiguous(), X, tol=tol, maxit=maxit, precond=prec)
        return X.cpu().numpy(), st

    for kw in ({}, {"tol": 1e-10}, {"maxit": 2}, {"m": 1}):
        g.set_graphs(False)
        x0, s0 = run(**kw)
        g.set_graphs(True)
        for _ in range(2):
            x1, s1 = run(**kw)
            assert np.array_equal(x1, x0), kw
            assert np.array_equal(s1.iters, s0.iters) and np.array_equal(s1.relres, s0.relres), kw
            assert s1.rc == s0.rc
    g.set_split(1, prec, 0, 0, 2)
    x1, s1 = run(m=1)
    g.set_graphs(False)
    x0, s0 = run(m=1)
    assert np.array_equal(x1, x0) and np.array_equal(s1.iters, s0.iters)
    assert s0.rc == 0


def test_caller_workspace(cfg0):
    Bm = dev(P.rhs_uniform(cfg0.A.n, 4, 6))
    nb = cfg0.g.workspace_bytes(4, B.PCG)
    ws = torch.empty(nb // 8 + 64, dtype=torch.float64, device="cuda")
    X1 = torch.empty_like(Bm)
    X2 = torch.empty_like(Bm)
    cfg0.g.solve(Bm, X1)
    cfg0.g.solve(Bm, X2, workspace=ws)
    assert torch.equal(X1, X2)


@pytest.mark.parametrize("m", [1, 3, 32])
def test_coldot(m):
    rng = np.random.default_rng(m)
    U = rng.uniform(-1, 1, size=(10007, m))
    V = rng.uniform(-1, 1, size=(10007, m))
    out = torch.empty(m, dtype=torch.float64, device="cuda")
    B.coldot(dev(U), dev(V), out)
    ref = (U * V).sum(axis=0)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)
    out2 = torch.empty(m, dtype=torch.float64, device="cuda")
    B.coldot(dev(U), dev(V), out2)
    assert torch.equal(out, out2)


@pytest.mark.parametrize("method", [B.PCG, B.BICGSTAB])
@pytest.mark.parametrize("prec", [B.PREC_FP64, B.PREC_FP32])
def test_warm_start_matches_oracle(cfg0, method, prec):
    Bm = P.rhs_uniform(cfg0.A.n, 4, 7)
    Bm[:, 3] = 0.0
    ref = cfg0.o.pcg(Bm, tol=1e-12)
    X0 = ref.X + 1e-4 * np.random.default_rng(2).standard_normal(ref.X.shape)
    X = dev(X0)
    st = cfg0.g.solve(dev(Bm), X, tol=1e-8, method=method, precond=prec, x0_given=True)
    o = (cfg0.o.pcg if method == B.PCG else cfg0.o.bicgstab)(Bm, tol=1e-8, prec=prec, X0=X0)
    Xg = X.cpu().numpy()
    assert st.rc == 0 and np.all(st.status == 0)
    assert np.all(true_relres(cfg0.A, Bm[:, :3], Xg[:, :3]) <= 1e-8)
    assert np.all(Xg[:, 3] == 0.0) and st.iters[3] == 0
    assert np.all(np.abs(st.iters - o.iters) <= 1), (st.iters, o.iters)
    cold = cfg0.g.solve(dev(Bm), torch.empty_like(X), tol=1e-8, method=method, precond=prec)
    assert np.all(st.iters[:3] < cold.iters[:3])
    # the exact solution as guess: nothing to do
    X = dev(ref.X)
    st = cfg0.g.solve(dev(Bm), X, tol=1e-8, method=method, precond=prec, x0_given=True)
    assert np.all(st.iters == 0) and np.all(st.status == 0)
