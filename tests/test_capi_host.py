"""CPU-side checks of the CUDA library: it loads, exports every entry point the
header declares, rejects bad input without touching a GPU, and its host AMG
setup reproduces the oracle's hierarchy bit for bit."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2103_07329_gb300 import binding as B
from paper_2103_07329_gb300 import build as build_mod
from paper_2103_07329_gb300 import problems as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build_mod.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "xamg_gpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xamg_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    decl = declared_functions()
    assert len(decl) >= 19
    assert sorted(B.EXPORTS) == decl
    L = B.lib()
    for name in decl:
        assert hasattr(L, name), name


def test_strerror_and_defaults():
    assert B.strerror(0) == "success"
    assert "non-finite" in B.strerror(B.ERR_NONFINITE)
    p = B.amg_params()
    assert (p.theta, p.max_coarse, p.cheb_steps, p.power_iters) == (0.25, 64, 2, 20)
    assert p.device_upload == 1


def host_hier(A, **kw):
    return B.Hierarchy(A, device_upload=0, **kw)


def test_invalid_inputs_rejected_on_host():
    A = P.poisson7(4)
    bad = P.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.col[1], bad.col[2] = bad.col[2], bad.col[1]        # unsorted row
    with pytest.raises(B.XamgError) as e:
        host_hier(bad)
    assert e.value.code == B.ERR_INVALID_ARG
    nf = P.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    nf.val[5] = np.inf
    with pytest.raises(B.XamgError) as e:
        host_hier(nf)
    assert e.value.code == B.ERR_NONFINITE
    nd = P.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    nd.val[nd.col == np.repeat(np.arange(A.n), np.diff(A.rowptr))] = 0.0   # zero diagonal
    with pytest.raises(B.XamgError) as e:
        host_hier(nd)
    assert e.value.code == B.ERR_INVALID_ARG


def test_host_only_handle_refuses_device_calls():
    A = P.poisson7(6)
    h = host_hier(A)
    with pytest.raises(B.XamgError) as e:
        h.timing_enable(True)
    assert e.value.code == B.ERR_INVALID_ARG
    rc = B.lib().xamg_solve(h.handle, 1, 1, 1, 1e-8, 10, None, None)
    assert rc == B.ERR_INVALID_ARG
    # the reduced-precision product, the 16-bit index and tail queries need the device copy
    assert B.lib().xamg_level_spmm_precond(h.handle, B.PREC_FP32, 0, 0, 1, 1, 1, None) == B.ERR_INVALID_ARG
    with pytest.raises(B.XamgError) as e:
        h.index16_info(0)
    assert e.value.code == B.ERR_INVALID_ARG
    with pytest.raises(B.XamgError) as e:
        h.tail_info(4)
    assert e.value.code == B.ERR_INVALID_ARG
    # host-side settings are accepted, with their arguments checked
    h.set_index16(True)
    h.set_tail(131072, 0.5, 0)
    h.set_tail(0)
    for bad in [(-1, 2.0, 0), (131072, 0.0, 0), (131072, 61.0, 0), (131072, 2.0, -1)]:
        with pytest.raises(B.XamgError) as e:
            h.set_tail(*bad)
        assert e.value.code == B.ERR_INVALID_ARG


def assert_same_hierarchy(A, **kw):
    ho = oracle.Hierarchy(A, **kw)
    hl = host_hier(A, **kw)
    assert hl.levels == ho.nlev
    for l in range(ho.nlev):
        o = ho.level(l)
        g = hl.level_export(l)
        assert g["n"] == o.n
        for a, b in zip(g["A"], o.A):
            assert np.array_equal(a, b)
        if o.P is not None:
            assert np.array_equal(g["cf"], o.cf)
            for a, b in zip(g["P"], o.P):
                assert np.array_equal(a, b)
            assert np.array_equal(g["cheb"], o.cheb)
    lu_l, piv_l = hl.coarse_export()
    lu_o, piv_o = ho.coarse_lu()
    assert np.array_equal(lu_l, lu_o) and np.array_equal(piv_l, piv_o)


@pytest.mark.parametrize("N", [4, 5, 9, 16, 24])
def test_setup_identical_to_oracle_poisson7(N):
    assert_same_hierarchy(P.poisson7(N))


def test_setup_identical_to_oracle_poisson27():
    assert_same_hierarchy(P.poisson27(10))


def test_setup_identical_to_oracle_32cube_threads():
    A = P.poisson7(32)
    assert_same_hierarchy(A)
    assert_same_hierarchy(A, nthreads=3)


def test_setup_identical_random_spd():
    # a non-stencil SPD matrix with mixed-sign couplings
    import scipy.sparse as sp
    M = sp.random(400, 400, density=0.02, random_state=4, format="csr")
    M = M + M.T
    M.data = -np.abs(M.data)
    M.data[::7] *= -0.3
    M = M + sp.diags(np.abs(M).sum(axis=1).A1 + 1.0)
    M = M.tocsr()
    M.sort_indices()
    A = P.CSR(400, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(float))
    assert_same_hierarchy(A, max_coarse=20)
