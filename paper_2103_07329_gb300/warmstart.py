"""Learned initial guess for the solve: data, training and evaluation.

The workload is steady diffusion -div(k grad u) = f on a 64^3 grid of unit
cells (``problems.diffusion7``) with log k a Gaussian random field
(squared-exponential covariance, correlation length 0.1 of the domain,
sigma = 1) and smooth right-hand sides from a Gaussian random field
(correlation length 0.2), 32 right-hand sides per coefficient field.  Fields
are synthesised on the padded periodic grid (``problems.grf``, pad = 2).

* Training pairs: field f (seed 10000 + f) and its 32 right-hand sides (one
  batch, seed 110000 + f); labels X solve A X = B to 1e-8 with this library's
  FP64 AMG-PCG.  Network input per column j: (B_j / s_j, log k) with s_j the
  column's root mean square; target X_j / s_j times a global constant c that
  gives the targets unit mean square.
* Held-out pairs: fields 20000 + f, right-hand sides 120000 + f.
* Training: Adam on the mean squared error, then (fine-tuning) on the
  relative energy-norm error ||X0_j - X_j||_A^2 / ||X_j||_A^2
  (||X_j||_A^2 = X_j^T B_j from the label solve), the norm in which PCG's
  error decreases.  The energy norm alone is badly conditioned (its Hessian
  in the output is A): started from scratch it settles at X0 = 0, so it only
  refines a network whose smooth part the mean squared error has fitted.
  Mini-batches of 32 samples come from a seeded permutation each epoch; each
  phase decays its step size by a cosine.
* Use: ``Net.predict_x0(B, log k, X0, 1 / c)``, optionally one Chebyshev
  smoothing of X0 on the finest level (``Hierarchy.smooth(0, B, X0,
  x_zero=False)``: it removes the high-frequency part of the network's
  error, which dominates the initial residual), then ``Hierarchy.solve(...,
  x0_given=True)``.  The plain solve from X0 = 0 is the fallback and the
  measure of accuracy (all forms run to 1e-8).

Run ``python -m paper_2103_07329_gb300.warmstart train --out PATH`` to train
and store the parameters, ``... eval --params PATH`` to compare held-out
iterations and right-hand sides per second with and without X0.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import time

import numpy as np

from . import binding as B
from . import problems as P

GRID = 64
M = 32
FIELD_CORR, RHS_CORR, SIGMA = 0.1, 0.2, 1.0
TRAIN_SEED, TRAIN_RHS_SEED = 10000, 110000
TEST_SEED, TEST_RHS_SEED = 20000, 120000
PARAMS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "warmstart_net64.npz")


def coefficient_field(N: int, seed: int) -> np.ndarray:
    """log k on the N^3 cells (lexicographic, x fastest)."""
    return P.grf(N, FIELD_CORR, SIGMA, seed, pad=2)[0]


def rhs_block(N: int, seed: int, m: int) -> np.ndarray:
    """n x m row-major block of m smooth right-hand sides."""
    f = P.grf(N, RHS_CORR, SIGMA, seed, count=m, pad=2, dtype=np.float32)
    return np.ascontiguousarray(f.T, dtype=np.float64)


class System:
    """One coefficient field: its matrix's hierarchy (on the device) and data."""

    def __init__(self, N: int, field_seed: int, rhs_seed: int, m: int, nthreads: int = 0):
        self.N = N
        self.logk = coefficient_field(N, field_seed)
        self.hier = B.Hierarchy(P.diffusion7(N, np.exp(self.logk)), nthreads=nthreads)
        self.B = rhs_block(N, rhs_seed, m)


def build_systems(N: int, seeds, rhs_seeds, m: int, workers: int = 4):
    """Systems for the given seeds, in order, set up by `workers` host threads
    at once (the library's setup runs outside the interpreter lock); at most
    2 x workers systems are alive at a time."""
    nthreads = max(1, (os.cpu_count() or 4) // workers)
    jobs = list(zip(seeds, rhs_seeds))
    with cf.ThreadPoolExecutor(workers) as ex:
        window = [ex.submit(System, N, s, r, m, nthreads) for s, r in jobs[:2 * workers]]
        nxt = len(window)
        while window:
            sysf = window.pop(0).result()
            if nxt < len(jobs):
                window.append(ex.submit(System, N, *jobs[nxt], m, nthreads))
                nxt += 1
            yield sysf


def _col_rms(Bm: np.ndarray) -> np.ndarray:
    return np.sqrt((Bm * Bm).mean(axis=0))


def make_pairs(N: int, nfields: int, seed0: int, rhs_seed0: int, m: int = M, tol: float = 1e-8,
               log=print):
    """Inputs [nfields m, N^3, 2], unscaled targets X_j / s_j [nfields m, N^3]
    (float32 CUDA tensors) and the targets' energies X_j^T B_j / s_j^2
    (float64 CUDA [nfields m]) from solves of the library."""
    import torch
    n = N ** 3
    inp = torch.empty((nfields * m, n, 2), dtype=torch.float32, device="cuda")
    tgt = torch.empty((nfields * m, n), dtype=torch.float32, device="cuda")
    energy = torch.empty(nfields * m, dtype=torch.float64, device="cuda")
    t0 = time.time()
    iters = []
    seeds = [seed0 + f for f in range(nfields)]
    rseeds = [rhs_seed0 + f for f in range(nfields)]
    for f, sysf in enumerate(build_systems(N, seeds, rseeds, m)):
        Bd = torch.as_tensor(sysf.B, device="cuda")
        X = torch.zeros_like(Bd)
        st = sysf.hier.solve(Bd, X, tol=tol, maxit=200)
        if st.rc != 0 or np.any(st.relres > tol):
            raise RuntimeError(f"label solve of field {seeds[f]} did not converge")
        iters.append(int(st.iters.max()))
        s = torch.as_tensor(_col_rms(sysf.B), device="cuda")
        sl = slice(f * m, (f + 1) * m)
        inp[sl, :, 0] = (Bd / s).T.float()
        inp[sl, :, 1] = torch.as_tensor(sysf.logk, dtype=torch.float32, device="cuda")[None, :]
        tgt[sl] = (X / s).T.float()
        energy[sl] = (X * Bd).sum(dim=0) / (s * s)
        sysf.hier.close()
        if log and (f + 1) % 16 == 0:
            log(f"  pairs: {f + 1}/{nfields} fields, {time.time() - t0:.1f} s")
    return inp, tgt, energy, iters


def train(N: int = GRID, nfields: int = 128, epochs: int = 30, batch: int = 32, lr: float = 2e-3,
          seed: int = 0, loss: str = "mse", finetune_epochs: int = 0, finetune_lr: float = 5e-4,
          log=print):
    """Trains the network on solver-generated pairs; returns (params, c, info)."""
    import torch
    t0 = time.time()
    inp, tgt, energy, iters = make_pairs(N, nfields, TRAIN_SEED, TRAIN_RHS_SEED, log=log)
    t_data = time.time() - t0
    c = float(1.0 / torch.sqrt((tgt.double() ** 2).mean()))
    tgt.mul_(c)
    # relative energy error: weight 1 / ||t_b||_A^2 with t = c X / s
    weight = (1.0 / (c * c * energy)).float()
    S = inp.shape[0]
    net = B.Net(N, batch)
    net.set_params(P.net_init(seed))
    rng = np.random.default_rng(seed)
    phases = [(B.LOSS_ENERGY if loss == "energy" else B.LOSS_MSE, epochs, lr)]
    if finetune_epochs:
        phases.append((B.LOSS_ENERGY, finetune_epochs, finetune_lr))
    hist = []
    t1 = time.time()
    for ph, (kind, ne, plr) in enumerate(phases):
        if ph:
            net.set_params(net.get_params())  # fresh Adam moments for the new loss
        steps = ne * (S // batch)
        k = 0
        w = weight if kind == B.LOSS_ENERGY else None
        for ep in range(ne):
            perm = rng.permutation(S).astype(np.int32)
            el = []
            for b0 in range(0, S - batch + 1, batch):
                idx = torch.as_tensor(perm[b0:b0 + batch], device="cuda")
                step_lr = 0.5 * plr * (1.0 + np.cos(np.pi * k / steps))
                el.append(net.train_step(inp, tgt, idx, lr=float(step_lr), loss=kind, weight=w))
                k += 1
            hist.append(float(np.mean(el)))
            if log and ((ep + 1) % 10 == 0 or ep == 0):
                name = "energy" if kind == B.LOSS_ENERGY else "mse"
                log(f"  {name} epoch {ep + 1}/{ne}: loss {hist[-1]:.5f} ({time.time() - t1:.1f} s)")
    torch.cuda.synchronize()
    t_train = time.time() - t1
    info = dict(N=N, fields=nfields, pairs=S, epochs=epochs, batch=batch, lr=lr, seed=seed, loss=loss,
                finetune_epochs=finetune_epochs, finetune_lr=finetune_lr, loss_history=hist,
                data_seconds=t_data, train_seconds=t_train, label_iters_max=int(max(iters)))
    return net.get_params(), c, info


def save(path: str, params: np.ndarray, c: float, info: dict):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez(path, params=params.astype(np.float32), c=np.float64(c), info=json.dumps(info))


def load(path: str = PARAMS_FILE):
    z = np.load(path, allow_pickle=False)
    return z["params"], float(z["c"]), json.loads(str(z["info"]))


def _timed(fn, reps: int = 3):
    """Median device time (ms) of fn() on the current stream, after one warm-up."""
    import torch
    fn()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), r


def evaluate(params: np.ndarray, c: float, N: int = GRID, nfields: int = 8, m: int = M,
             tol: float = 1e-8, precond: int = B.PREC_FP64, reps: int = 3, sweeps: int = 1, log=print):
    """Held-out comparison of the solve from X0 = 0 and from the network's X0.

    Per field: iterations (max over columns), device time of the solve (and of
    the prediction plus the solve), true relative residuals.  Returns a dict
    with the per-field records and the totals in right-hand sides per second."""
    import torch
    net = B.Net(N, m)
    net.set_params(params)
    recs = []
    seeds = [TEST_SEED + f for f in range(nfields)]
    rseeds = [TEST_RHS_SEED + f for f in range(nfields)]
    for sysf in build_systems(N, seeds, rseeds, m):
        Bd = torch.as_tensor(sysf.B, device="cuda")
        logk = torch.as_tensor(sysf.logk, dtype=torch.float32, device="cuda")
        X = torch.empty_like(Bd)

        def plain():
            X.zero_()
            return sysf.hier.solve(Bd, X, tol=tol, maxit=200, precond=precond)

        def warm(smooth=False):
            net.predict_x0(Bd, logk, X, 1.0 / c)
            for _ in range(sweeps if smooth else 0):
                sysf.hier.smooth(0, Bd, X, x_zero=False)
            return sysf.hier.solve(Bd, X, tol=tol, maxit=200, precond=precond, x0_given=True)

        t_plain, st_p = _timed(plain, reps)
        t_warm, st_w = _timed(warm, reps)
        t_warms, st_s = _timed(lambda: warm(True), reps)
        t_pred, _ = _timed(lambda: net.predict_x0(Bd, logk, X, 1.0 / c), reps)
        # quality of X0 (and of X0 after the smoothing) against the converged
        # solution X*: relative L2 and A-norm errors and the initial relative
        # residual (max over columns)
        plain()
        Xs = X.clone()

        def quality(smooth):
            net.predict_x0(Bd, logk, X, 1.0 / c)
            for _ in range(sweeps if smooth else 0):
                sysf.hier.smooth(0, Bd, X, x_zero=False)
            E, AE, AX = X - Xs, torch.empty_like(X), torch.empty_like(X)
            sysf.hier.spmm(0, 0, E, AE)
            sysf.hier.spmm(0, 0, X, AX)
            torch.cuda.synchronize()
            return (float(torch.linalg.norm(E) / torch.linalg.norm(Xs)),
                    float(torch.sqrt((E * AE).sum(0) / (Xs * Bd).sum(0)).max()),
                    float((torch.linalg.norm(Bd - AX, dim=0) / torch.linalg.norm(Bd, dim=0)).max()))

        e0, ea, r0 = quality(False)
        _, eas, r0s = quality(True)
        rec = dict(iters_plain=int(st_p.iters.max()), iters_warm=int(st_w.iters.max()),
                   iters_warm_smooth=int(st_s.iters.max()), x0_l2_error=e0, x0_anorm_error=ea,
                   x0_relres=r0, x0s_anorm_error=eas, x0s_relres=r0s,
                   mean_iters_plain=float(st_p.iters.mean()), mean_iters_warm=float(st_w.iters.mean()),
                   mean_iters_warm_smooth=float(st_s.iters.mean()),
                   ms_plain=t_plain, ms_warm=t_warm, ms_warm_smooth=t_warms, ms_predict=t_pred,
                   relres_max_plain=float(st_p.relres.max()), relres_max_warm=float(st_w.relres.max()),
                   relres_max_warm_smooth=float(st_s.relres.max()),
                   rc_plain=st_p.rc, rc_warm=st_w.rc, rc_warm_smooth=st_s.rc)
        recs.append(rec)
        sysf.hier.close()
        if log:
            log(f"  field: iters {rec['iters_plain']} -> {rec['iters_warm']} / {rec['iters_warm_smooth']} "
                f"(smoothed), ms {t_plain:.2f} -> {t_warm:.2f} / {t_warms:.2f} (predict {t_pred:.2f}); "
                f"X0 L2 error {e0:.3f}, A-norm {ea:.3f} / {eas:.3f}, residual {r0:.3f} / {r0s:.3f}")
    tp = sum(r["ms_plain"] for r in recs)
    tw = sum(r["ms_warm"] for r in recs)
    ts = sum(r["ms_warm_smooth"] for r in recs)
    return dict(fields=nfields, m=m, tol=tol, sweeps=sweeps, records=recs,
                rhs_per_s_plain=nfields * m / (tp * 1e-3), rhs_per_s_warm=nfields * m / (tw * 1e-3),
                rhs_per_s_warm_smooth=nfields * m / (ts * 1e-3), speedup=tp / tw, speedup_smooth=tp / ts)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", default=PARAMS_FILE)
    t.add_argument("--grid", type=int, default=GRID)
    t.add_argument("--fields", type=int, default=128)
    t.add_argument("--epochs", type=int, default=30)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--loss", choices=["energy", "mse"], default="mse")
    t.add_argument("--eval-fields", type=int, default=8)
    t.add_argument("--finetune-epochs", type=int, default=0)
    t.add_argument("--finetune-lr", type=float, default=5e-4)
    t.add_argument("--sweeps", type=int, default=1)
    e = sub.add_parser("eval")
    e.add_argument("--params", default=PARAMS_FILE)
    e.add_argument("--fields", type=int, default=8)
    e.add_argument("--sweeps", type=int, default=1)
    a = ap.parse_args(argv)
    if a.cmd == "train":
        params, c, info = train(a.grid, a.fields, a.epochs, lr=a.lr, loss=a.loss,
                                finetune_epochs=a.finetune_epochs, finetune_lr=a.finetune_lr)
        save(a.out, params, c, info)
        print(json.dumps({k: v for k, v in info.items() if k != "loss_history"}))
        if a.eval_fields:
            r = evaluate(params, c, a.grid, a.eval_fields, sweeps=a.sweeps)
            print(json.dumps({k: v for k, v in r.items() if k != "records"}))
    else:
        params, c, info = load(a.params)
        r = evaluate(params, c, info["N"], a.fields, sweeps=a.sweeps)
        print(json.dumps(r))


if __name__ == "__main__":
    main()
