"""Pins of the oracle's reduced-precision preconditioner (paper Sec. 2.3,
"mixed-precision"): the bf16 rounding against torch's conversion, FP32 and
bf16 row products against the textbook summation error bound, the FP32
V-cycle against the FP64 one, and flexible PCG / BiCGStab against dense
solves."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle
from paper_2103_07329_gb300 import problems as P

torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


def to_scipy(A):
    return sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    vals = np.concatenate([
        rng.standard_normal(2000).astype(np.float32),
        (rng.standard_normal(500) * 1e-30).astype(np.float32),        # tiny
        (rng.standard_normal(500) * 1e30).astype(np.float32),         # huge
        np.array([0.0, -0.0, 1.0, -1.0, 3.3895314e38, 1e-45, 1.17549435e-38], np.float32),
    ])
    # exact halfway cases between consecutive bf16 values: ties go to even
    base = (rng.integers(0, 2 ** 15, 500, dtype=np.uint32) << 16) | 0x8000
    vals = np.concatenate([vals, base.view(np.float32)])
    vals = vals[np.isfinite(vals)]
    ref = torch.from_numpy(vals).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = np.array([oracle.bf16_bits(float(v)) for v in vals], dtype=np.uint16)
    assert np.array_equal(got, ref)


def fine_hier(N=12):
    A = P.poisson7(N)
    return A, oracle.Hierarchy(A)


def test_fp32_products_within_summation_bound():
    A, h = fine_hier(12)
    rng = np.random.default_rng(1)
    for l in range(2):
        lv = h.level(l)
        for which, (rp, ci, v), ncols in [(0, lv.A, lv.n), (1, lv.P, h.level(l + 1).n),
                                          (2, lv.R, lv.n)]:
            rows = len(rp) - 1
            X = rng.standard_normal((ncols, 3)).astype(np.float32)
            Y = h.spmm_f(l, which, X)
            M = sp.csr_matrix((v.astype(np.float32).astype(np.float64), ci, rp), shape=(rows, ncols))
            exact = M @ X.astype(np.float64)
            absd = abs(M) @ np.abs(X.astype(np.float64))
            k = np.diff(rp).max()
            gamma = k * U32 / (1 - k * U32)
            assert np.all(np.abs(Y - exact) <= gamma * absd + 1e-45)


def test_bf16_values_and_products():
    A, h = fine_hier(10)
    lv = h.level(1)                     # a Galerkin level: non-integer values
    rp, ci, v = lv.A
    n = lv.n
    rng = np.random.default_rng(2)
    X = rng.standard_normal((n, 2)).astype(np.float32)
    Y = h.spmm_f(1, 0, X, bf16=True)
    Ad = sp.csr_matrix((v, ci, rp), shape=(n, n))
    exact = Ad @ X.astype(np.float64)
    absd = abs(Ad) @ np.abs(X.astype(np.float64))
    # each stored value is within half a bf16 ulp (2^-9 relative) of fl32(a_ij),
    # plus the FP32 summation and the scale product
    k = np.diff(rp).max()
    bound = (2.0 ** -8 + (k + 2) * U32) * absd
    assert np.all(np.abs(Y - exact) <= bound)
    # and bf16 is genuinely coarser than FP32 on these values
    Y32 = h.spmm_f(1, 0, X)
    assert np.abs(Y - exact).max() > 10 * np.abs(Y32 - exact).max()


@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (2, 5e-2)])
def test_reduced_vcycle_close_to_fp64(prec, tol):
    A, h = fine_hier(16)
    B = P.rhs_uniform(A.n, 3, 0)
    X64 = h.vcycle(B)
    X = h.vcycle_prec(prec, B)
    rel = np.linalg.norm(X - X64, axis=0) / np.linalg.norm(X64, axis=0)
    assert np.all(rel <= tol) and np.all(rel > 0)
    # prec 0 is the FP64 cycle itself
    assert np.array_equal(h.vcycle_prec(0, B), X64)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
@pytest.mark.parametrize("N", [5, 8])
def test_reduced_precision_solves_vs_dense(prec, method, N):
    A = P.poisson7(N)
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 3, 0)
    r = getattr(h, method)(B, tol=1e-10, prec=prec)
    Ad = to_scipy(A).toarray()
    ref = sla.lu_solve(sla.lu_factor(Ad), B)
    kappa = np.linalg.cond(Ad)
    assert np.all(r.status == 0)
    for j in range(3):
        assert np.linalg.norm(r.X[:, j] - ref[:, j]) <= 1e-10 * kappa * np.linalg.norm(ref[:, j])


def test_flexible_pcg_iterations_and_accuracy():
    A = P.diffusion7(16, P.lognormal_cells(16, 1.0, 1))
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 4, 0)
    r64 = h.pcg(B, tol=1e-8)
    for prec in (1, 2):
        r = h.pcg(B, tol=1e-8, prec=prec)
        assert np.all(r.status == 0) and np.all(r.relres <= 1e-8)
        assert np.all(r.iters <= r64.iters + (1 if prec == 1 else 3))


def _rn32(q):
    """Nearest FP32 value of the rational q, ties to even (normal range)."""
    from fractions import Fraction
    if q == 0:
        return 0.0
    sgn = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    elif Fraction(2) ** (e + 1) <= a:
        e += 1
    assert -126 <= e <= 127
    m = a / Fraction(2) ** (e - 23)              # in [2^23, 2^24)
    f = m.numerator // m.denominator
    rem = m - f
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return sgn * float(Fraction(f) * Fraction(2) ** (e - 23))


def test_fp32_accumulation_is_one_rounding_per_term_in_storage_order():
    # reading R9: each term of a row product is added with one rounding (a
    # fused multiply-add), in the row's storage order.  Brute force with exact
    # rational arithmetic and an independent round-to-nearest-even, on the
    # non-integer values of a Galerkin level and of P and R
    from fractions import Fraction
    A, h = fine_hier(8)
    rng = np.random.default_rng(5)
    separate_differs = False
    for l, which in [(1, 0), (0, 1), (0, 2)]:
        lv = h.level(l)
        rp, ci, v = lv.A if which == 0 else (lv.P if which == 1 else lv.R)
        ncols = h.level(l + 1).n if which == 1 else lv.n
        X = rng.standard_normal((ncols, 2)).astype(np.float32)
        Y = h.spmm_f(l, which, X)
        v32 = v.astype(np.float32)
        for i in range(0, len(rp) - 1, 7):
            for j in range(2):
                y = Fraction(0)
                ys = np.float32(0)
                for p in range(rp[i], rp[i + 1]):
                    term = Fraction(float(v32[p])) * Fraction(float(X[ci[p], j]))
                    y = Fraction(_rn32(term + y))
                    ys = np.float32(ys + np.float32(v32[p] * X[ci[p], j]))
                assert Y[i, j] == np.float32(float(y)), (l, which, i, j)
                separate_differs |= bool(ys != Y[i, j])
    # the check can tell a fused chain from a multiply-then-add chain
    assert separate_differs
