"""GPU parity of the BiCGStab variants (paper Sec. 2.1: reordered and
pipelined BiCGStab, merged formulations; XAMG_BICGSTAB_REORDERED /
XAMG_BICGSTAB_PIPELINED) against the oracle's implementations of the same
variants: true residual <= 1e-8 per column (checked by the oracle's FP64
product), iteration counts within +-1 of the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2103_07329_gb300 import binding as B
from paper_2103_07329_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = {B.BICGSTAB_REORDERED: "reordered", B.BICGSTAB_PIPELINED: "pipelined"}
_cache = {}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pair(key):
    if key not in _cache:
        A = P.poisson7(32) if key == "p7_32" else P.diffusion7(24, P.lognormal_cells(24, 1.0, 1))
        _cache[key] = (A, B.Hierarchy(A), oracle.Hierarchy(A))
    return _cache[key]


def true_rel(A, Bm, X):
    return np.linalg.norm(Bm - oracle.spmm(A, X), axis=0) / np.linalg.norm(Bm, axis=0)


@pytest.mark.parametrize("key", ["p7_32", "var_24"])
@pytest.mark.parametrize("method", list(VARIANTS))
@pytest.mark.parametrize("m", [1, 4, 32])
def test_variant_matches_the_oracle(key, method, m):
    A, g, o = pair(key)
    Bm = P.rhs_uniform(A.n, m, 0, m_draw=32)
    X = torch.empty_like(dev(Bm))
    st = g.solve(dev(Bm), X, tol=1e-8, maxit=100, method=method)
    assert st.rc == 0 and np.all(st.status == 0)
    assert np.all(true_rel(A, Bm, X.cpu().numpy()) <= 1e-8)
    ref = o.bicgstab(Bm, tol=1e-8, variant=VARIANTS[method])
    assert np.all(np.abs(st.iters - ref.iters) <= 1), (st.iters, ref.iters)
    # the same method in exact arithmetic as the classical one
    cl = g.solve(dev(Bm), torch.empty_like(X), tol=1e-8, maxit=100, method=B.BICGSTAB)
    assert np.all(np.abs(st.iters - cl.iters) <= 1)


@pytest.mark.parametrize("prec", [B.PREC_FP32, B.PREC_BF16])
def test_reordered_with_reduced_precision(prec):
    A, g, o = pair("var_24")
    Bm = P.rhs_uniform(A.n, 8, 0, m_draw=32)
    X = torch.empty_like(dev(Bm))
    st = g.solve(dev(Bm), X, tol=1e-8, maxit=100, method=B.BICGSTAB_REORDERED, precond=prec)
    assert st.rc == 0 and np.all(true_rel(A, Bm, X.cpu().numpy()) <= 1e-8)
    ref = o.bicgstab(Bm, tol=1e-8, prec=prec, variant="reordered")
    assert np.all(np.abs(st.iters - ref.iters) <= 1), (st.iters, ref.iters)


def test_pipelined_needs_the_fp64_preconditioner():
    A, g, _ = pair("p7_32")
    Bm = P.rhs_uniform(A.n, 2, 0)
    with pytest.raises(B.XamgError) as e:
        g.solve(dev(Bm), torch.empty_like(dev(Bm)), method=B.BICGSTAB_PIPELINED, precond=B.PREC_FP32)
    assert e.value.code == B.ERR_INVALID_ARG
    assert g.workspace_bytes(8, B.BICGSTAB_PIPELINED) > g.workspace_bytes(8, B.BICGSTAB)


@pytest.mark.parametrize("method", list(VARIANTS))
def test_variants_edge_cases(method):
    A, g, _ = pair("var_24")
    Bm = P.rhs_uniform(A.n, 4, 3)
    Bm[:, 1] = 0.0
    X = torch.empty_like(dev(Bm))
    st = g.solve(dev(Bm), X, tol=1e-8, maxit=100, method=method)
    Xh = X.cpu().numpy()
    assert st.rc == 0 and np.all(Xh[:, 1] == 0.0) and st.status[1] == 0
    assert np.all(true_rel(A, Bm[:, [0, 2, 3]], Xh[:, [0, 2, 3]]) <= 1e-8)
    # warm start from the solution: zero iterations
    X2 = X.clone()
    s2 = g.solve(dev(Bm), X2, tol=1e-8, maxit=100, method=method, x0_given=True)
    assert s2.rc == 0 and np.all(s2.iters == 0)
    # maxit 1 leaves the columns unconverged, with the status saying so
    s3 = g.solve(dev(Bm), torch.empty_like(X), tol=1e-14, maxit=1, method=method)
    assert s3.rc == B.NOT_CONVERGED
