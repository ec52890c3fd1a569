"""The fused coarse tail of the V-cycle (one cooperative launch for the
levels below a size threshold, grid barriers between stages; paper Sec. 2.1,
the V-cycle of the MultiGrid preconditioner): bitwise the unfused cycle and
solve, in FP64 and with the reduced-precision preconditioners, with CUDA
graphs on; and the bounded barrier wait, which a test makes run out (fault
injection on the host side: arrivals that never come) and which must end in
XAMG_ERR_TIMEOUT with the device still usable."""
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


_cache = {}


def system(key):
    if key not in _cache:
        if key == "p7_32":
            A = P.poisson7(32)
        elif key == "var_24":
            A = P.diffusion7(24, P.lognormal_cells(24, 1.0, 1))
        else:
            A = P.poisson27(16)
        _cache[key] = A
    return _cache[key]


def cycle(g, prec, Bm):
    X = torch.empty((Bm.shape[0], Bm.shape[1]), dtype=torch.float64, device="cuda")
    if prec == B.PREC_FP64:
        g.vcycle(dev(Bm), X)
    else:
        g.vcycle_precond(prec, dev(Bm), X)
    return X.cpu().numpy()


@pytest.mark.parametrize("key,m", [("p7_32", 4), ("p7_32", 32), ("var_24", 8), ("p27_16", 16), ("p27_16", 2)])
@pytest.mark.parametrize("prec", [B.PREC_FP64, B.PREC_FP32, B.PREC_BF16])
def test_fused_tail_cycle_is_bitwise_the_unfused_one(key, m, prec):
    A = system(key)
    g = B.Hierarchy(A)
    assert g.tail_info(m) == -1          # off by default
    g.set_tail(131072)
    first = g.tail_info(m)
    assert 0 <= first <= g.levels - 2
    Bm = P.rhs_uniform(A.n, m, 0, m_draw=32)
    fused = cycle(g, prec, Bm)
    g.set_tail(0)
    assert g.tail_info(m) == -1
    plain = cycle(g, prec, Bm)
    assert np.array_equal(fused, plain)
    if prec == B.PREC_FP64:
        ref = oracle.Hierarchy(A).vcycle(Bm)
        rel = np.linalg.norm(fused - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert rel.max() <= 1e-12


def test_tail_covers_the_whole_cycle_of_a_small_system():
    # 7-point 32^3 with four right-hand sides: every level's block holds at
    # most 131072 elements, so the cycle from level 0 is one launch
    g = B.Hierarchy(system("p7_32"))
    g.set_tail(131072)
    assert g.tail_info(4) == 0
    assert g.tail_info(1) == -1          # m = 1 keeps the stream kernels
    g.set_tail(4096)
    assert g.tail_info(4) > 0            # a lower threshold starts deeper


@pytest.mark.parametrize("prec", [B.PREC_FP64, B.PREC_FP32])
@pytest.mark.parametrize("method", [B.PCG, B.BICGSTAB])
def test_fused_tail_solve_is_bitwise_the_unfused_one(prec, method):
    # graphs on (the default): the steady PCG iteration captures the
    # cooperative launch; a second solve replays it
    A = system("var_24")
    Bm = P.rhs_uniform(A.n, 8, 0, m_draw=32)
    out = []
    for elems in (131072, 0):
        g = B.Hierarchy(A)
        g.set_tail(elems)
        X = torch.empty_like(dev(Bm))
        for _ in range(2):
            st = g.solve(dev(Bm), X, tol=1e-8, maxit=100, method=method, precond=prec)
        assert st.rc == 0 and np.all(st.status == 0)
        out.append((X.cpu().numpy(), st.iters.copy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    rr = np.linalg.norm(Bm - oracle.spmm(A, out[0][0]), axis=0) / np.linalg.norm(Bm, axis=0)
    assert np.all(rr <= 1e-8)


def test_tail_barrier_wait_runs_out_and_the_device_stays_usable():
    A = system("p7_32")
    g = B.Hierarchy(A)
    g.set_tail(131072)
    Bm = P.rhs_uniform(A.n, 4, 0, m_draw=32)
    ref = cycle(g, B.PREC_FP64, Bm)
    # every barrier now expects one arrival that never comes: each wait ends
    # after 20 ms with the error recorded, and the kernel returns
    g.set_tail(131072, 0.02, 1)
    X = torch.empty((A.n, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(B.XamgError) as e:
        g.vcycle(dev(Bm), X)
    assert e.value.code == B.ERR_TIMEOUT
    with pytest.raises(B.XamgError) as e:
        g.solve(dev(Bm), X, tol=1e-8, maxit=3)
    assert e.value.code == B.ERR_TIMEOUT
    # back to normal waits: the same hierarchy and context give the same bits
    g.set_tail(131072, 2.0, 0)
    assert np.array_equal(cycle(g, B.PREC_FP64, Bm), ref)
    st = g.solve(dev(Bm), X, tol=1e-8, maxit=100)
    assert st.rc == 0 and np.all(st.status == 0)
    with pytest.raises(B.XamgError):
        g.set_tail(-1)
    with pytest.raises(B.XamgError):
        g.set_tail(131072, 0.0)
