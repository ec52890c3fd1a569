"""GPU parity of the batched solve (csrc/batch*.cu through xamg_batch_*):
every system of a batch gets what its own single-system solve with the FP32
preconditioner gets, and what the oracle's FP32-preconditioned flexible PCG
gets.

Tolerances: the batched stages run the single-system row code on the same
data, and the FP64 dot products differ only in the order of the per-block
partial sums (the grid may differ), so each column's iteration count equals
the single solve's within 1 and the solutions agree to 1e-9 relative (both
are within 1e-8 of the exact one).  Against the oracle: iteration counts
within +-1, true residual <= 1e-8 per column (checked in FP64 by the
oracle's product)."""
import numpy as np
import pytest

import oracle
from paper_2103_07329_gb300 import binding as B
from paper_2103_07329_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPEC = [(8, 1), (12, 3), (16, 8), (10, 16), (14, 32), (9, 5), (20, 2)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def colrel(g, o):
    return np.linalg.norm(g - o, axis=0) / np.linalg.norm(o, axis=0)


@pytest.fixture(scope="module")
def systems():
    out = []
    for s, (edge, m) in enumerate(SPEC):
        A, Bm = P.batch_system(edge, m, s)
        out.append((A, Bm, B.Hierarchy(A)))
    return out


def solve_batch(systems, **kw):
    batch = B.Batch([h for _, _, h in systems], [Bm.shape[1] for _, Bm, _ in systems], **kw)
    Bd = [dev(Bm) for _, Bm, _ in systems]
    Xs = [torch.full_like(b, np.nan) for b in Bd]
    st = batch.solve(Bd, Xs, tol=1e-8, maxit=100)
    return batch, [x.cpu().numpy() for x in Xs], st


def test_batch_matches_single_solves(systems):
    batch, Xs, st = solve_batch(systems)
    info = batch.info()
    assert info["ops_tuned"] > 0 and info["launches_per_iteration"] > 0
    for (A, Bm, h), X, s in zip(systems, Xs, st):
        assert s.rc == 0 and np.all(s.status == 0)
        rr = np.linalg.norm(Bm - oracle.spmm(A, X), axis=0) / np.linalg.norm(Bm, axis=0)
        assert np.all(rr <= 1e-8), rr
        X1 = torch.empty_like(dev(Bm))
        s1 = h.solve(dev(Bm), X1, tol=1e-8, maxit=100, precond=B.PREC_FP32)
        assert np.all(np.abs(s.iters - s1.iters) <= 1), (s.iters, s1.iters)
        assert colrel(X, X1.cpu().numpy()).max() <= 1e-9


def test_batch_matches_the_oracle(systems):
    _, Xs, st = solve_batch(systems[:3])
    for (A, Bm, _), X, s in zip(systems[:3], Xs, st):
        o = oracle.Hierarchy(A)
        ref = o.pcg(Bm, tol=1e-8, prec=B.PREC_FP32)
        assert np.all(np.abs(s.iters - ref.iters) <= 1), (s.iters, ref.iters)
        x64 = o.pcg(Bm, tol=1e-8).X
        assert colrel(X, x64).max() <= 1e-6


def test_graph_and_autotune_options(systems):
    _, Xg, sg = solve_batch(systems, autotune=False, use_graph=True)
    _, Xn, sn = solve_batch(systems, autotune=False, use_graph=False)
    _, Xt, st = solve_batch(systems, autotune=True, use_graph=True)
    for a, b, c, s1, s2, s3 in zip(Xg, Xn, Xt, sg, sn, st):
        # the graph replays the same launches: bitwise equal
        assert np.array_equal(a, b) and np.array_equal(s1.iters, s2.iters)
        # another row split sums each row's products in another order
        assert np.all(np.abs(s1.iters - s3.iters) <= 1)
        assert colrel(c, a).max() <= 1e-9


def test_repeated_solves_and_zero_columns(systems):
    sub = systems[1:4]
    batch = B.Batch([h for _, _, h in sub], [Bm.shape[1] for _, Bm, _ in sub])
    Bs = [Bm.copy() for _, Bm, _ in sub]
    Bs[0][:, 1] = 0.0            # a zero column
    Bs[1][:] = 0.0               # a zero system
    Bd = [dev(b) for b in Bs]
    X1 = [torch.empty_like(b) for b in Bd]
    X2 = [torch.empty_like(b) for b in Bd]
    s1 = batch.solve(Bd, X1)
    s2 = batch.solve(Bd, X2)
    for a, b, p, q in zip(X1, X2, s1, s2):
        assert torch.equal(a, b) and np.array_equal(p.iters, q.iters)
    assert float(X1[0][:, 1].abs().max()) == 0.0 and s1[0].status[1] == 0
    assert float(X1[1].abs().max()) == 0.0 and np.all(s1[1].status == 0)
    A, Bm, _ = sub[2]
    rr = np.linalg.norm(Bm - oracle.spmm(A, X1[2].cpu().numpy()), axis=0) / np.linalg.norm(Bm, axis=0)
    assert np.all(rr <= 1e-8)


def test_invalid_batches(systems):
    one_level = B.Hierarchy(P.poisson7(3))
    with pytest.raises(B.XamgError) as e:
        B.Batch([systems[0][2], one_level], [1, 1])
    assert e.value.code == B.ERR_INVALID_ARG
    with pytest.raises(B.XamgError):
        B.Batch([systems[0][2]], [33])


def test_batch_at_the_workload_sizes_matches_the_oracle():
    # systems of the benchmark's size range side by side: an 80^3 system with
    # 32 right-hand sides (512 000 unknowns, many blocks per system in every
    # fine-level stage), a 64^3 one with 7 and a 16^3 one with 4
    spec = [(80, 32), (16, 4), (64, 7)]
    sys_ = []
    for s, (edge, m) in enumerate(spec):
        A, Bm = P.batch_system(edge, m, 40 + s)
        sys_.append((A, Bm, B.Hierarchy(A)))
    _, Xs, st = solve_batch(sys_)
    for (A, Bm, h), X, s in zip(sys_, Xs, st):
        assert s.rc == 0 and np.all(s.status == 0)
        rr = np.linalg.norm(Bm - oracle.spmm(A, X), axis=0) / np.linalg.norm(Bm, axis=0)
        assert np.all(rr <= 1e-8), rr
        ref = oracle.Hierarchy(A).pcg(Bm, tol=1e-8, prec=B.PREC_FP32)
        assert np.all(np.abs(s.iters - ref.iters) <= 1), (s.iters, ref.iters)
        X1 = torch.empty_like(dev(Bm))
        s1 = h.solve(dev(Bm), X1, tol=1e-8, maxit=100, precond=B.PREC_FP32)
        assert np.all(np.abs(s.iters - s1.iters) <= 1)
        assert colrel(X, X1.cpu().numpy()).max() <= 1e-9
