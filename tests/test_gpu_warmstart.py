"""What the trained warm-start network gains over the solve from X0 = 0, on a
held-out 64^3 diffusion system (log k Gaussian random field, 32 smooth
right-hand sides), with the parameters trained on the GPU by
``python -m paper_2103_07329_gb300.warmstart train`` and stored in the
package.  The plain solve to 1e-8 is the measure of the initial guess: every form must
reach the tolerance; the network's X0 must be much closer to the solution in
the energy norm (the norm PCG reduces) than X0 = 0 or an untrained network's
output, and must not cost iterations."""
import numpy as np
import pytest
import torch

from paper_2103_07329_gb300 import binding as B
from paper_2103_07329_gb300 import problems as P
from paper_2103_07329_gb300 import warmstart as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def system():
    s = next(W.build_systems(W.GRID, [W.TEST_SEED + 3], [W.TEST_RHS_SEED + 3], W.M, workers=1))
    yield s
    s.hier.close()


def anorm_rel_error(h, X, Xs, Bd):
    E = X - Xs
    AE = torch.empty_like(E)
    h.spmm(0, 0, E, AE)
    torch.cuda.synchronize()
    return (torch.sqrt((E * AE).sum(0) / (Xs * Bd).sum(0))).cpu().numpy()


def test_trained_network_improves_the_initial_guess(system):
    params, c, info = W.load()
    assert info["N"] == W.GRID and info["pairs"] == 4096
    h = system.hier
    Bd = torch.as_tensor(system.B, device="cuda")
    logk = torch.as_tensor(system.logk, dtype=torch.float32, device="cuda")
    Xs = torch.zeros_like(Bd)
    st0 = h.solve(Bd, Xs, tol=1e-8, maxit=200)
    assert st0.rc == 0 and st0.relres.max() <= 1e-8
    net = B.Net(W.GRID, W.M)
    errs = {}
    for name, p in (("trained", params), ("untrained", P.net_init(0))):
        net.set_params(p)
        X0 = torch.empty_like(Bd)
        net.predict_x0(Bd, logk, X0, 1.0 / c)
        errs[name] = anorm_rel_error(h, X0, Xs, Bd)
        X = X0.clone()
        st = h.solve(Bd, X, tol=1e-8, maxit=200, x0_given=True)
        assert st.rc == 0 and st.relres.max() <= 1e-8          # the plain solve's accuracy
        if name == "trained":
            assert st.iters.max() <= st0.iters.max()             # no iterations lost
    # X0 = 0 has relative A-norm error 1; the trained network's is far below it
    assert errs["trained"].max() < 0.3, errs["trained"]
    assert errs["untrained"].min() > 0.9, errs["untrained"]
