"""Pins of the oracle's BiCGStab variants (paper Sec. 2.1: reordered and
pipelined BiCGStab, merged formulations).  Both are exact rearrangements of
the classical right-preconditioned BiCGStab: in FP64 with the (linear) FP64
V-cycle their iterates must equal the classical method's, iteration by
iteration, to rounding; the classical method itself is pinned against dense
solves and closed forms in test_oracle.py."""
import numpy as np
import pytest

import oracle
from paper_2103_07329_gb300 import problems as P


@pytest.fixture(scope="module")
def var():
    A = P.diffusion7(14, P.lognormal_cells(14, 1.5, 3))
    return A, oracle.Hierarchy(A)


def colrel(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


@pytest.mark.parametrize("variant", ["reordered", "pipelined"])
def test_iterates_equal_the_classical_ones(var, variant):
    A, h = var
    B = P.rhs_uniform(A.n, 3, 0)
    for k in (1, 2, 3):
        c = h.bicgstab(B, tol=1e-15, maxit=k)
        v = h.bicgstab(B, tol=1e-15, maxit=k, variant=variant)
        assert colrel(v.X, c.X).max() <= 1e-12, (k, colrel(v.X, c.X))
        assert np.allclose(v.relres, c.relres, rtol=1e-6)


@pytest.mark.parametrize("variant", ["reordered", "pipelined"])
def test_variants_converge_like_the_classical_method(var, variant):
    A, h = var
    B = P.rhs_uniform(A.n, 4, 1)
    B[:, 2] = 0.0                                   # a zero column returns x = 0
    c = h.bicgstab(B, tol=1e-8)
    v = h.bicgstab(B, tol=1e-8, variant=variant)
    assert v.rc == 0 and np.all(v.status == 0)
    rr = np.linalg.norm(B - oracle.spmm(A, v.X), axis=0) / np.maximum(np.linalg.norm(B, axis=0), 1e-300)
    assert np.all(rr[[0, 1, 3]] <= 1e-8) and np.all(v.X[:, 2] == 0.0)
    assert np.all(np.abs(v.iters - c.iters) <= 1)
    # warm start from the solution: nothing left to do
    w = h.bicgstab(B, tol=1e-8, variant=variant, X0=v.X.copy())
    assert np.all(w.iters == 0) and w.rc == 0


def test_reordered_with_the_reduced_precision_preconditioner(var):
    A, h = var
    B = P.rhs_uniform(A.n, 2, 2)
    for prec in (1, 2):
        c = h.bicgstab(B, tol=1e-8, prec=prec)
        v = h.bicgstab(B, tol=1e-8, prec=prec, variant="reordered")
        assert v.rc == 0 and np.all(np.abs(v.iters - c.iters) <= 1)


def test_dense_case():
    # a tiny grid with one level: the V-cycle is the exact solve, so BiCGStab
    # finishes in one iteration and matches the dense LU solution
    A = P.poisson7(3)
    h = oracle.Hierarchy(A)
    B = P.rhs_uniform(A.n, 2, 4)
    dense = np.zeros((A.n, A.n))
    for i in range(A.n):
        dense[i, A.col[A.rowptr[i]:A.rowptr[i + 1]]] = A.val[A.rowptr[i]:A.rowptr[i + 1]]
    Xd = np.linalg.solve(dense, B)
    for variant in ("reordered", "pipelined"):
        v = h.bicgstab(B, tol=1e-10, variant=variant)
        assert np.all(v.iters == 1) and colrel(v.X, Xd).max() <= 1e-12
