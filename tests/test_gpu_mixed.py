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


def _long_range(N, stride):
    """7-point Poisson plus a symmetric coupling of every row to the row
    `stride` away (diagonally dominant, so still SPD): with a stride beyond
    two index windows of 65536 the rows cannot use 16-bit column indices."""
    import scipy.sparse as sp
    A0 = P.poisson7(N)
    M = sp.csr_matrix((A0.val, A0.col, A0.rowptr), shape=(A0.n, A0.n))
    n = A0.n
    E = sp.diags([np.full(n - stride, -0.1), np.full(n - stride, -0.1)], [stride, -stride], shape=(n, n))
    M = (M + E + sp.identity(n) * 0.2).tocsr()
    M.sort_indices()
    return P.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data)


@pytest.mark.parametrize("which", ["windows", "fallback"])
def test_bf16_index_compression_paths(which):
    # n = 262144 spans four windows; the 7-point rows cross window borders but
    # fit two windows (16-bit indices).  The long-range variant does not fit
    # and keeps 32-bit indices.  Both must match the oracle's bf16 V-cycle.
    A = P.poisson7(64) if which == "windows" else _long_range(64, 140000)
    g, o = B.Hierarchy(A), oracle.Hierarchy(A)
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
