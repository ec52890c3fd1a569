"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, hand-derived cases, textbook/library routines and invariants.

Each test names the plausible oracle mistakes it would catch.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle
from paper_2103_07329_gb300 import problems as P

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def to_scipy(A):
    return sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))


def lev_scipy(t, rows, cols):
    rp, ci, v = t
    return sp.csr_matrix((v, ci, rp), shape=(rows, cols))


# ---------------------------------------------------------------- generators
@pytest.mark.parametrize("N", [1, 2, 3, 5, 8])
def test_poisson7_closed_forms(N):
    A = P.poisson7(N)
    assert A.n == N ** 3
    assert A.nnz == N ** 3 + 6 * N * N * (N - 1)
    S = to_scipy(A)
    assert (S != S.T).nnz == 0
    # row sum = number of missing (Dirichlet) neighbours
    idx = np.arange(A.n)
    i, j, k = idx % N, (idx // N) % N, idx // (N * N)
    missing = sum((c == 0).astype(int) + (c == N - 1).astype(int) for c in (i, j, k))
    assert np.array_equal(np.asarray(S.sum(axis=1)).ravel(), missing.astype(float))
    for r in range(A.n):
        cols = A.col[A.rowptr[r]:A.rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0)


def test_nnz_at_benchmark_sizes():
    # closed forms at the benchmark grids, without building them
    assert 32 ** 3 + 6 * 32 ** 2 * 31 == 223232
    assert 192 ** 3 + 6 * 192 ** 2 * 191 == 49324032
    assert (3 * 160 - 2) ** 3 == 109215352
    A = P.poisson7(32)
    assert A.nnz == 223232


@pytest.mark.parametrize("N", [2, 3, 6])
def test_poisson27_closed_forms(N):
    A = P.poisson27(N)
    assert A.nnz == (3 * N - 2) ** 3
    S = to_scipy(A)
    assert (S != S.T).nnz == 0
    assert np.all(S.diagonal() == 26.0)


def test_diffusion7_hand_cases():
    # constant k = 1: interior faces T = 1, boundary faces T = 2 (half-cell
    # Dirichlet distance), so the row sum is 2 x (number of boundary faces)
    N = 4
    A = P.diffusion7(N, np.ones(N ** 3))
    S = to_scipy(A)
    assert (S != S.T).nnz == 0
    idx = np.arange(A.n)
    i, j, k = idx % N, (idx // N) % N, idx // (N * N)
    bfaces = sum((c == 0).astype(int) + (c == N - 1).astype(int) for c in (i, j, k))
    assert np.array_equal(np.asarray(S.sum(axis=1)).ravel(), 2.0 * bfaces)
    assert np.array_equal(S.diagonal(), 6.0 + bfaces)
    assert A.nnz == P.poisson7(N).nnz
    # two cells with k = 1 and 3 in a 2x2x2 block: harmonic mean 2*1*3/4 = 1.5
    kc = np.ones(8)
    kc[1] = 3.0
    B = to_scipy(P.diffusion7(2, kc)).toarray()
    assert B[0, 1] == -1.5 and B[1, 0] == -1.5
    # cell 1 has three interior faces (T = 1.5) and three boundary faces (T = 2 k = 6)
    assert B[1, 1] == 3 * 1.5 + 3 * 2 * 3.0


def eigvec7(N, p, q, r):

    g = np.arange(1, N + 1)
    s = lambda a: np.sin(np.pi * a * g / (N + 1))
    v = np.einsum("k,j,i->kji", s(r), s(q), s(p)).reshape(-1)
    lam = sum(2 - 2 * np.cos(np.pi * a / (N + 1)) for a in (p, q, r))
    return v, lam


# ---------------------------------------------------------------- SpMM
def test_spmm_exact_integers_vs_dense():
    # integer data: every partial sum is exact, so the result is bitwise the
    # dense product
    rng = np.random.default_rng(5)
    A = P.poisson27(4)
    Ad = to_scipy(A).toarray()
    for m in (1, 3, 4, 32):
        X = rng.integers(-1000, 1001, size=(A.n, m)).astype(np.float64)
        Y = oracle.spmm(A, X)
        assert np.array_equal(Y, Ad @ X)


def test_spmm_random_matrix_vs_scipy():
    rng = np.random.default_rng(1)
    M = sp.random(300, 300, density=0.03, random_state=2, format="csr") + sp.eye(300)
    M.sort_indices()
    A = P.CSR(300, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data)
    X = rng.standard_normal((300, 7))
    Y = oracle.spmm(A, X)
    ref = M @ X
    assert np.linalg.norm(Y - ref) <= 1e-14 * np.linalg.norm(ref)


def test_spmm_ones_gives_boundary_count():
    A = P.poisson7(6)
    y = oracle.spmm(A, np.ones((A.n, 1)))[:, 0]
    assert np.array_equal(y, np.asarray(to_scipy(A).sum(axis=1)).ravel())
    assert y.min() == 0.0 and y.max() == 3.0


@pytest.mark.parametrize("N,modes", [(8, (1, 1, 1)), (8, (2, 5, 3)), (11, (11, 1, 7))])
def test_spmm_eigenvectors(N, modes):
    A = P.poisson7(N)
    v, lam = eigvec7(N, *modes)
    y = oracle.spmm(A, v[:, None])[:, 0]
    assert np.linalg.norm(y - lam * v) <= 1e-14 * lam * np.linalg.norm(v) * 10


# ---------------------------------------------------------------- generator
def test_splitmix_published_vector():
    vals = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
            if l.startswith("0x")]
    for i, z in enumerate(vals):
        assert oracle.splitmix_uniform(i) == 2.0 * ((z >> 11) * 2.0 ** -53) - 1.0


# ---------------------------------------------------------------- dense LU
@pytest.mark.parametrize("n", [1, 5, 64])
def test_lu_vs_scipy(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + n * np.eye(n) * 0.1
    B = rng.standard_normal((n, 3))
    lu, piv = oracle.lu_factor(A)
    X = oracle.lu_solve(lu, piv, B)
    ref = sla.lu_solve(sla.lu_factor(A), B)
    assert np.allclose(X, ref, rtol=1e-10, atol=1e-12)
    # P A = L U reconstruction
    L = np.tril(lu, -1) + np.eye(n)
    U = np.triu(lu)
    PA = A.copy()
    for k in range(n):
        PA[[k, piv[k]]] = PA[[piv[k], k]]
    assert np.allclose(L @ U, PA, rtol=1e-12, atol=1e-12)


def test_lu_pivots_like_lapack():
    # partial pivoting picks the largest magnitude in the column: LAPACK getrf
    rng = np.random.default_rng(3)
    A = rng.standard_normal((20, 20))
    _, piv = oracle.lu_factor(A)
    _, piv_ref = sla.lu_factor(A)
    assert np.array_equal(piv, piv_ref)


# ---------------------------------------------------------------- setup
def read_gold(name):
    d = {}
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        d[key] = np.array([float(v) for v in vals])
    return d


def lap1d(n):
    M = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    M.sort_indices()
    return P.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(float))


def test_rs_1d_hand_case():
    g = read_gold("rs_1d_n7.txt")
    h = oracle.Hierarchy(lap1d(7), max_coarse=2)
    assert h.nlev == 3
    l0, l1, l2 = h.level(0), h.level(1), h.level(2)
    assert np.array_equal(l0.cf, g["cf0"].astype(int))
    assert np.array_equal(lev_scipy(l0.P, 7, 3).toarray().ravel(), g["P0"])
    assert np.array_equal(lev_scipy(l1.A, 3, 3).toarray().ravel(), g["A1"])
    assert np.array_equal(l1.cf, g["cf1"].astype(int))
    assert np.array_equal(lev_scipy(l1.P, 3, 1).toarray().ravel(), g["P1"])
    assert np.array_equal(lev_scipy(l2.A, 1, 1).toarray().ravel(), g["A2"])
    # R is the transpose of P
    assert np.array_equal(lev_scipy(l0.R, 3, 7).toarray(), lev_scipy(l0.P, 7, 3).toarray().T)


def test_rs_2d_five_point_3x3():
    # 2-D 5-point Laplacian on a 3x3 grid, every coupling strong.  lambda:
    # corners 2, edges 3, centre 4 -> centre (4) is C first; its four edge
    # neighbours become F; each new F raises its undecided influencers, the
    # corners, to 2 + 2 = 4 (two F neighbours each) -> corner 0 is C next,
    # then 2, 6, 8 (ties by index).  Pass 2: edge point 1 has strong F
    # neighbours? none (its neighbours 0, 2, 4 are C).  So C = {0,2,4,6,8}.
    n1 = 3
    T = sp.diags([-np.ones(n1 - 1), 2 * np.ones(n1), -np.ones(n1 - 1)], [-1, 0, 1])
    M = (sp.kron(sp.eye(n1), T) + sp.kron(T, sp.eye(n1))).tocsr()
    M.sort_indices()
    A = P.CSR(9, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(float))
    h = oracle.Hierarchy(A, max_coarse=4)
    l0 = h.level(0)
    assert np.array_equal(l0.cf, np.array([1, 0, 1, 0, 1, 0, 1, 0, 1]))
    # edge point 1 (diag 4, couplings -1 to its C neighbours 0, 2, 4): no weak
    # and no strong F neighbours, so w_ij = -a_ij / a_ii = 1/4 for each of them.
    Pd = lev_scipy(l0.P, 9, 5).toarray()
    assert np.array_equal(Pd[1], np.array([0.25, 0.25, 0.25, 0, 0]))


def level_checks(h, rowsum_zero_rows=True):
    for l in range(h.nlev - 1):
        lv, nx = h.level(l), h.level(l + 1)
        A = lev_scipy(lv.A, lv.n, lv.n)
        Pm = lev_scipy(lv.P, lv.n, nx.n)
        Ac = lev_scipy(nx.A, nx.n, nx.n)
        # Galerkin product against scipy's sparse products (a library routine)
        ref = (Pm.T @ A @ Pm).toarray()
        assert np.abs(Ac.toarray() - ref).max() <= 1e-13 * np.abs(ref).max()
        # symmetric to rounding
        D = Ac.toarray()
        assert np.abs(D - D.T).max() <= 1e-14 * np.abs(D).max()
        # C rows inject, coarse numbering follows fine order
        cf = lv.cf
        cidx = np.cumsum(cf) - 1
        for i in np.nonzero(cf)[0][:50]:
            row = Pm.getrow(i)
            assert row.nnz == 1 and row.indices[0] == cidx[i] and row.data[0] == 1.0
        # interpolation reproduces constants on zero-row-sum F rows
        rs = np.asarray(A.sum(axis=1)).ravel()
        amax = np.abs(A).max(axis=1).toarray().ravel()
        prs = np.asarray(Pm.sum(axis=1)).ravel()
        sel = (cf == 0) & (np.abs(rs) <= 1e-13 * amax)
        if l == 0 and rowsum_zero_rows:
            assert sel.sum() > 0
        assert np.abs(prs[sel] - 1.0).max(initial=0.0) <= 1e-12
        # Chebyshev interval: upper end min(1.1 lambda_hat, Gershgorin), lower 0.3 hi
        lo, hi, lam, gersh = lv.cheb
        assert hi == min(1.1 * lam, gersh) and lo == 0.3 * hi
        # Gershgorin bound of D^-1 A computed independently
        g = (abs(A).multiply(1.0 / np.abs(A.diagonal())[:, None])).sum(axis=1).max()
        assert abs(gersh - g) <= 1e-14 * g


@pytest.mark.parametrize("N", [6, 10, 16])
def test_setup_invariants_poisson7(N):
    h = oracle.Hierarchy(P.poisson7(N))
    assert h.level(h.nlev - 1).n <= 64
    level_checks(h)


def test_setup_invariants_poisson27():
    h = oracle.Hierarchy(P.poisson27(8))
    level_checks(h)


def test_power_iteration_below_lambda_max():
    # fine level of the 7-point operator: D^-1 A = A/6 is symmetric, so the norm
    # ratio is below lambda_max = (6 + 6 cos(pi/(N+1)))/6 and close to it
    N = 20
    h = oracle.Hierarchy(P.poisson7(N))
    lam = h.level(0).cheb[2]
    lmax = 1.0 + np.cos(np.pi / (N + 1))
    assert 0.9 * lmax <= lam <= lmax * (1 + 1e-12)


def test_single_level_when_small():
    # n <= 64: one level, the preconditioner is the exact inverse
    A = P.poisson7(4)
    h = oracle.Hierarchy(A)
    assert h.nlev == 1
    B = P.rhs_uniform(A.n, 3, 0)
    X = h.vcycle(B)
    ref = np.linalg.solve(to_scipy(A).toarray(), B)
    assert np.allclose(X, ref, rtol=1e-12, atol=1e-13)
    r = h.pcg(B)
    assert np.all(r.iters == 1) and np.all(r.status == 0)


# ---------------------------------------------------------------- Chebyshev
def test_chebyshev_error_polynomial_closed_form():
    # error after the smoother from x = 0 on an eigenvector e of D^-1 A with
    # eigenvalue mu: p_2(mu) e with p_2(mu) = T_2((theta-mu)/delta) / T_2(theta/delta)
    N = 12
    A = P.poisson7(N)
    h = oracle.Hierarchy(A)
    lo, hi = h.level(0).cheb[:2]
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T2 = lambda t: 2 * t * t - 1
    for modes in [(1, 1, 1), (3, 7, 2), (12, 12, 12), (6, 6, 6)]:
        e, lam = eigvec7(N, *modes)
        mu = lam / 6.0
        b = lam * e
        x, r = h.cheb_smooth(0, b[:, None])
        p2 = T2((theta - mu) / delta) / T2(theta / delta)
        assert np.linalg.norm((e - x[:, 0]) - p2 * e) <= 1e-13 * np.linalg.norm(e)
        # the returned residual is b - A x
        assert np.linalg.norm(r[:, 0] - (b - lam * x[:, 0])) <= 1e-13 * np.linalg.norm(b)


def test_chebyshev_from_nonzero_start():
    # post-smoothing form: same polynomial acting on the initial error
    N = 10
    A = P.poisson7(N)
    h = oracle.Hierarchy(A)
    lo, hi = h.level(0).cheb[:2]
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    e, lam = eigvec7(N, 2, 3, 4)
    mu = lam / 6.0
    x0 = np.full(A.n, 0.3)
    xs = x0 + e                       # exact solution
    b = oracle.spmm(A, xs[:, None])[:, 0]
    x, _ = h.cheb_smooth(0, b[:, None], X0=x0[:, None], want_residual=False)
    err0 = xs - x0                    # = e
    p2 = (2 * ((theta - mu) / delta) ** 2 - 1) / (2 * (theta / delta) ** 2 - 1)
    assert np.linalg.norm((xs - x[:, 0]) - p2 * err0) <= 1e-12 * np.linalg.norm(e)


# ---------------------------------------------------------------- V-cycle
def test_vcycle_symmetric_positive_definite():
    A = P.poisson7(12)
    h = oracle.Hierarchy(A)
    assert h.nlev >= 3
    rng = np.random.default_rng(0)
    U = rng.standard_normal((A.n, 3))
    V = rng.standard_normal((A.n, 3))
    MU, MV = h.vcycle(U), h.vcycle(V)
    for j in range(3):
        a, b = MU[:, j] @ V[:, j], U[:, j] @ MV[:, j]
        assert abs(a - b) <= 1e-12 * np.linalg.norm(MU[:, j]) * np.linalg.norm(V[:, j])
        assert MU[:, j] @ U[:, j] > 0


def vcycle_rho(h, A, iters=40, seed=0):
    x = np.random.default_rng(seed).standard_normal((A.n, 1))
    lam = 0.0
    for _ in range(iters):
        y = x - h.vcycle(oracle.spmm(A, x))
        lam = np.linalg.norm(y) / np.linalg.norm(x)
        x = y / np.linalg.norm(y)
    return lam


def test_vcycle_convergence_factor_h_independent():
    rhos = []
    for N in (8, 12, 16):
        A = P.poisson7(N)
        h = oracle.Hierarchy(A)
        rhos.append(vcycle_rho(h, A))
    assert max(rhos) < 0.3, rhos
    assert rhos[2] < 1.2 * rhos[0] + 0.02, rhos


def test_vcycle_linear_in_rhs():
    A = P.poisson7(9)
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 2, 1)
    X = h.vcycle(B)
    X2 = h.vcycle(np.ascontiguousarray(B * 4.0))
    assert np.array_equal(X2, 4.0 * X)


# ---------------------------------------------------------------- Krylov
@pytest.mark.parametrize("N", [3, 4, 6, 8])
@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
def test_tiny_systems_vs_dense_solve(N, method):
    A = P.poisson7(N)
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 4, 0)
    r = getattr(h, method)(B, tol=1e-10)
    Ad = to_scipy(A).toarray()
    ref = sla.lu_solve(sla.lu_factor(Ad), B)
    kappa = np.linalg.cond(Ad)
    assert np.all(r.status == 0)
    for j in range(4):
        assert np.linalg.norm(r.X[:, j] - ref[:, j]) <= 1e-10 * kappa * np.linalg.norm(ref[:, j])


@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
def test_eigenvector_rhs_closed_form(method):
    N = 16
    A = P.poisson7(N)
    h = oracle.Hierarchy(A)
    cols, lams = zip(*[eigvec7(N, *md) for md in [(1, 1, 1), (2, 1, 3), (5, 9, 2), (16, 16, 16)]])
    B = np.ascontiguousarray(np.stack(cols, axis=1))
    r = getattr(h, method)(B, tol=1e-8)
    lam = np.array(lams)
    lam_min = 3 * (2 - 2 * np.cos(np.pi / (N + 1)))
    assert np.all(r.status == 0)
    for j in range(B.shape[1]):
        # ||x - x*|| <= ||r|| / lam_min and ||x*|| = ||b|| / lam_j
        xs = B[:, j] / lam[j]
        assert np.linalg.norm(r.X[:, j] - xs) <= 1e-8 * (lam[j] / lam_min) * np.linalg.norm(xs)
        assert r.relres[j] <= 1e-8


@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
def test_multi_rhs_identity_and_invariances(method):
    A = P.poisson7(12)
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 5, 0)
    B[:, 2] = 0.0
    full = getattr(h, method)(B)
    for j in range(5):
        one = getattr(h, method)(np.ascontiguousarray(B[:, j:j + 1]))
        assert np.array_equal(one.X[:, 0], full.X[:, j])
        assert one.iters[0] == full.iters[j]
    # zero column: x = 0 after 0 iterations
    assert full.iters[2] == 0 and np.all(full.X[:, 2] == 0.0) and full.status[2] == 0
    # column permutation
    perm = [3, 0, 4, 2, 1]
    pr = getattr(h, method)(np.ascontiguousarray(B[:, perm]))
    assert np.array_equal(pr.X, full.X[:, perm])
    # scaling one column by a power of two scales its solution exactly
    B2 = B.copy()
    B2[:, 1] *= 2.0 ** 7
    sc = getattr(h, method)(B2)
    assert np.array_equal(sc.X[:, 1], full.X[:, 1] * 2.0 ** 7)
    assert sc.iters[1] == full.iters[1]


def test_true_residual_meets_tolerance_cfg0():
    A = P.poisson7(32)
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 4, 0)
    for method in ("pcg", "bicgstab"):
        r = getattr(h, method)(B, tol=1e-8)
        Ad = to_scipy(A)
        for j in range(4):
            true = np.linalg.norm(B[:, j] - Ad @ r.X[:, j]) / np.linalg.norm(B[:, j])
            assert true <= 1e-8
            assert abs(true - r.relres[j]) <= 1e-3 * true


def test_nonfinite_rhs_rejected():
    A = P.poisson7(5)
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 2, 0)
    B[3, 1] = np.nan
    with pytest.raises(RuntimeError):
        h.pcg(B)


def test_maxit_reports_not_converged():
    A = P.poisson7(12)
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 2, 0)
    r = h.pcg(B, tol=1e-14, maxit=2)
    assert r.rc == 1 and np.all(r.status == 1) and np.all(r.iters == 2)


@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
def test_warm_start(method):
    A = P.poisson7(10)
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 3, 0)
    B[:, 2] = 0.0
    exact = sla.lu_solve(sla.lu_factor(to_scipy(A).toarray()), B)
    # the exact solution as initial guess: no iteration, unchanged up to rounding
    r = getattr(h, method)(B, X0=exact)
    assert np.all(r.iters == 0) and np.all(r.status == 0)
    assert np.allclose(r.X, exact, rtol=0, atol=1e-14)
    # a perturbed guess: fewer iterations than from zero, same tolerance met;
    # the zero column returns x = 0 whatever the guess
    cold = getattr(h, method)(B)
    X0 = exact + 1e-5 * np.random.default_rng(1).standard_normal(exact.shape)
    warm = getattr(h, method)(B, X0=X0)
    assert np.all(warm.relres <= 1e-8) and np.all(warm.status == 0)
    assert np.all(warm.iters[:2] < cold.iters[:2])
    assert np.all(warm.X[:, 2] == 0.0) and warm.iters[2] == 0


def test_grf_covariance():
    # empirical covariance of the periodic fields against the squared-exponential
    # kernel sigma^2 exp(-r^2 / (2 l^2)) at lags along one axis
    N, ell, sigma = 32, 0.1, 1.5
    f = P.grf(N, ell, sigma, seed=3, count=64).reshape(64, N, N, N)
    f = f - f.mean()
    for lag in (0, 1, 2, 3, 5):
        emp = (f * np.roll(f, -lag, axis=3)).mean()
        ref = sigma ** 2 * np.exp(-(lag / N) ** 2 / (2 * ell ** 2))
        assert abs(emp - ref) <= 0.08 * sigma ** 2, (lag, emp, ref)
    # reproducible and seed-dependent
    assert np.array_equal(P.grf(8, 0.2, 1.0, 5), P.grf(8, 0.2, 1.0, 5))
    assert not np.array_equal(P.grf(8, 0.2, 1.0, 5), P.grf(8, 0.2, 1.0, 6))
