#!/usr/bin/env python3
"""Throughput benchmark: right-hand sides solved per second to 1e-8 relative
residual by the GPU solve phase (plain FP64 PCG preconditioned by one V(1,1)
Chebyshev-2 cycle of classical Ruge-Stueben AMG).

Default workload: 3-D 7-point Poisson on a 192^3 grid (n = 7,077,888,
nnz = 49,324,032), m = 32 right-hand sides uniform[-1, 1) from seed 0, PCG to
||b_j - A x_j|| <= 1e-8 ||b_j||.  One step = one complete ``xamg_solve`` of the
m-column block with the inputs resident in HBM (each block, 1.8 GB, is larger
than the 129 MB L2).  The AMG setup is done once before timing.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank solves its own block of m right-hand sides (seed =
rank) on its own GPU with no collective on the data path (weak scaling); the
ranks meet only at the barriers around the timed region and for the max-time /
sum-count reductions.

``--impl reference`` times the plain FP64 CPU oracle (oracle/) on the same
matrix, one column per step, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS solved/s to 1e-8 residual, plain FP64 vs mixed/batched/warm; SpMM %HBM"
UNIT = "RHS/s"
# FP64 FMA peak derived from the part's unit counts and clock: 152 SMs x 2 FP64
# FMA lanes per SM per clock x 2 flop x 2.07 GHz (1.259 TFLOP/s; ncu reports
# the same two DFMA per SM per clock as the FP64 pipe's sustained peak).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


METHODS = {"pcg": 0, "bicgstab": 1, "bicgstab_reordered": 2, "bicgstab_pipelined": 3}


def oracle_threads() -> int:
    """Threads the oracle's OpenMP loops use: OMP_NUM_THREADS if set, else
    every host core."""
    try:
        return max(1, int(os.environ["OMP_NUM_THREADS"]))
    except (KeyError, ValueError):
        return os.cpu_count()


def oracle_solve(h, a, Bm):
    """The oracle's solve of the benchmark's method."""
    if a.method == "pcg":
        return h.pcg(Bm, a.tol, a.maxit)
    variant = {"bicgstab": "classical", "bicgstab_reordered": "reordered",
               "bicgstab_pipelined": "pipelined"}[a.method]
    return h.bicgstab(Bm, a.tol, a.maxit, variant=variant)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--matrix", default="poisson7", choices=["poisson7", "poisson27", "diffusion7"])
    ap.add_argument("--sigma", type=float, default=1.0, help="diffusion7: lognormal sigma of k")
    ap.add_argument("--kseed", type=int, default=1, help="diffusion7: seed of the cell coefficients")
    ap.add_argument("--grid", type=int, default=None)
    ap.add_argument("--m", type=int, default=32)
    ap.add_argument("--method", default="pcg",
                    choices=["pcg", "bicgstab", "bicgstab_reordered", "bicgstab_pipelined"])
    ap.add_argument("--sweep-ms", default="1,2,4,8,16,32", help="--sweep: comma-separated m values")
    ap.add_argument("--sweep-methods", default="pcg,bicgstab",
                    help="--sweep: comma-separated methods (also bicgstab_reordered, bicgstab_pipelined)")
    ap.add_argument("--fp32-split", type=int, default=-1,
                    help="--sweep: force this split candidate on every FP32-block product "
                         "(-1: the default rule)")
    ap.add_argument("--fp64-split", type=int, default=-1,
                    help="--sweep: force this split candidate on every FP64 product of the "
                         "levels averaging at most --split-max-row entries per row")
    ap.add_argument("--split-max-row", type=float, default=1e9,
                    help="--sweep: the forced splits apply to levels with at most this many "
                         "entries per row on average")
    ap.add_argument("--index16", action="store_true",
                    help="--sweep: 16-bit column indices in the reduced-precision products")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=100)
    ap.add_argument("--cpu-cols", type=int, default=8,
                    help="cpu_baseline: columns of the oracle's sample (one multi-column solve)")
    ap.add_argument("--ref-cols", type=int, default=1,
                    help="--impl reference: columns the oracle solves per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the reduced-precision and warm forms")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned-initial-guess form")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the variable-coefficient precision workload")
    ap.add_argument("--precision-grid", type=int, default=192,
                    help="grid edge of the variable-coefficient precision workload")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched form")
    ap.add_argument("--batch-count", type=int, default=64, help="systems of the batched form")
    ap.add_argument("--batch-only", action="store_true",
                    help="measurement mode: only the batched form, as one JSON line")
    ap.add_argument("--batch-no-seq", action="store_true",
                    help="with --batch-only: skip the one-system-at-a-time solves (profiling)")
    ap.add_argument("--sweep", action="store_true",
                    help="measurement mode: m in 1..32, PCG and BiCGStab, FP64/FP32/bf16 "
                         "preconditioner, one JSON line each (not the benchmark line)")
    ap.add_argument("--split-table", action="store_true",
                    help="measurement mode: every row split of every level's product y = M x "
                         "on --m columns (--precond), microseconds per product, one JSON line per "
                         "operator")
    ap.add_argument("--tail-table", action="store_true",
                    help="measurement mode: small solves (7-point 32^3 and 64^3, m = 4 and 32; "
                         "variable-coefficient 64^3, m = 32) with the fused coarse tail on and off, "
                         "FP64 and FP32 preconditioners, one JSON line each")
    ap.add_argument("--spmm-only", action="store_true",
                    help="profiling mode: four products y = A x of level --level on --m columns "
                         "with the default row split, nothing else (the case for kernel captures)")
    ap.add_argument("--level", type=int, default=0, help="--spmm-only: the level")
    ap.add_argument("--precond", default="fp64", choices=["fp64", "fp32", "bf16"],
                    help="--spmm-only, --split-table: FP64 blocks, or FP32 blocks with FP32 / bf16 "
                         "values of A")
    a = ap.parse_args()
    if a.grid is None:
        a.grid = 160 if a.matrix == "poisson27" else 192
    return a


def make_matrix(a):
    from paper_2103_07329_gb300 import problems as P
    if a.matrix == "diffusion7":
        return P.diffusion7(a.grid, P.lognormal_cells(a.grid, a.sigma, a.kseed))
    return P.poisson7(a.grid) if a.matrix == "poisson7" else P.poisson27(a.grid)


def workload_name(a, A):
    if a.matrix == "diffusion7":
        kind = (f"3-D 7-point variable-coefficient diffusion (cell k lognormal sigma={a.sigma:g}, "
                f"seed {a.kseed})")
    else:
        kind = "3-D 7-point Poisson" if a.matrix == "poisson7" else "3-D 27-point Poisson"
    return (f"{kind} {a.grid}^3 (n={A.n}, nnz={A.nnz}), m={a.m} RHS uniform[-1,1) "
            f"seed 0, {a.method.upper()} + classical RS AMG V(1,1) Chebyshev-2, tol {a.tol:g}, FP64")


class Clocks:
    """nvidia-smi sampler for the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 power=float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        load = [r for r in rows if r["power"] > 250.0] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load),
                "sm_max_mhz": max(r["smax"] for r in rows), "samples": len(load),
                "reasons": sorted(reasons)}


def measured_hbm():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ("paper_2103_07329_gb300/csrc/kernels.cuh", "paper_2103_07329_gb300/csrc/rows_inst.cuh")
TRAFFIC_FILE = "profiles/traffic_k_rows_poisson7_96_m32.txt"


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def kernel_traffic(a, algorithmic_bytes_per_launch):
    """DRAM bytes (read + write) per row-kernel launch of the FP64 solve,
    scaled from the committed ncu capture of the same solve on the 96^3 grid
    (the 192^3 solve holds too much device memory for a capture) by the
    algorithmic bytes per launch: traffic = captured DRAM bytes x (this run's
    algorithmic bytes / the captured run's).  None when the capture is
    missing, the workload is not the 7-point m = 32 PCG solve, or the kernel
    sources changed since the capture."""
    if (a.matrix, a.m, a.method) != ("poisson7", 32, "pcg"):
        return None
    try:
        kv = {}
        for line in open(os.path.join(ROOT, TRAFFIC_FILE)):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != kernel_source_hash():
            return None
        ratio = float(kv["dram_bytes_per_launch"]) / float(kv["algorithmic_bytes_per_launch"])
        return round(ratio * algorithmic_bytes_per_launch)
    except Exception:
        return None


def cpu_baseline(a, A, seconds_note=True):
    """The oracle, as it stands, on a bounded sample: `cpu_cols` columns of the
    same workload solved to tol; returns (RHS/s, info)."""
    import oracle
    from paper_2103_07329_gb300 import problems as P
    t0 = time.perf_counter()
    h = oracle.Hierarchy(A)
    t_setup = time.perf_counter() - t0
    Bm = P.rhs_uniform(A.n, a.cpu_cols, 0, m_draw=max(a.m, a.cpu_cols))
    t0 = time.perf_counter()
    r = oracle_solve(h, a, Bm)
    t = time.perf_counter() - t0
    ok = int(np.sum((r.status == 0) & (r.relres <= a.tol)))
    return ok / t, dict(t_solve=t, t_setup=t_setup, iters=r.iters.tolist(), h=h)


def batch_form(a, seq=True):
    """The batched form: `batch_count` independent 7-point diffusion systems
    (grid edge uniform in 16..96, m uniform in 1..32, lognormal sigma 0.5
    coefficients; problems.batch_spec / batch_system) solved to a.tol, timed
    over a.steps rounds after one warm-up: one system after another with the
    plain FP64 solve and with the FP32 preconditioner, and all systems at once
    (xamg_batch_solve: one launch per stage for all systems, CUDA graph,
    autotuned row splits).  RHS/s count the columns that reached the
    tolerance."""
    import concurrent.futures as cf

    import torch

    from paper_2103_07329_gb300 import binding as B
    from paper_2103_07329_gb300 import problems as P
    spec = P.batch_spec(a.batch_count)
    t0 = time.perf_counter()
    nth = max(1, (os.cpu_count() or 4) // 4)

    def mk(s):
        e, m = spec[s]
        A, Bm = P.batch_system(e, m, s)
        return A, Bm, B.Hierarchy(A, nthreads=nth)

    with cf.ThreadPoolExecutor(4) as ex:
        systems = list(ex.map(mk, range(len(spec))))
    t_setup = time.perf_counter() - t0
    hs = [h for _, _, h in systems]
    ms = [Bm.shape[1] for _, Bm, _ in systems]
    Bd = [torch.from_numpy(Bm).cuda() for _, Bm, _ in systems]
    Xs = [torch.empty_like(b) for b in Bd]
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        solved = 0
        e0.record(stream)
        for _ in range(a.steps):
            solved += fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), solved

    def seq_fn(prec):
        def f():
            ok = 0
            for h, b, x in zip(hs, Bd, Xs):
                st = h.solve(b, x, a.tol, a.maxit, precond=prec)
                ok += int(np.sum((st.status == 0) & (st.relres <= a.tol)))
            return ok
        return f

    out = {"workload": (f"{len(spec)} independent 3-D 7-point diffusion systems, grid edge uniform "
                        f"16..96 and m uniform 1..32 (seed 2), cell k lognormal sigma 0.5 (seed 100+s), "
                        f"B uniform[-1,1) (seed 1000+s), tol {a.tol:g}"),
           "systems": len(spec), "rhs": int(sum(ms)), "unknowns": int(sum(e ** 3 for e, _ in spec)),
           "setup_s": round(t_setup, 2), "max_levels": max(h.levels for h in hs)}
    if seq:
        ms64, ok64 = timed(seq_fn(B.PREC_FP64))
        ms32, ok32 = timed(seq_fn(B.PREC_FP32))
        out["rhs_per_s_plain_fp64_one_by_one"] = ok64 / (ms64 * 1e-3)
        out["rhs_per_s_fp32_one_by_one"] = ok32 / (ms32 * 1e-3)
    t0 = time.perf_counter()
    batch = B.Batch(hs, ms)
    out["create_s"] = round(time.perf_counter() - t0, 3)
    last = []

    def bf():
        st = batch.solve(Bd, Xs, a.tol, a.maxit)
        last[:] = st
        return sum(int(np.sum((s.status == 0) & (s.relres <= a.tol))) for s in st)

    l0 = B.kernel_launches()
    msb, okb = timed(bf)
    out["gpu_launches_per_solve"] = (B.kernel_launches() - l0) // (a.steps + 1)
    out["value"] = okb / (msb * 1e-3)
    out["ms_per_step"] = msb / a.steps
    if seq:
        out["speedup_vs_plain_fp64"] = out["value"] / out["rhs_per_s_plain_fp64_one_by_one"]
        out["speedup_vs_fp32_one_by_one"] = out["value"] / out["rhs_per_s_fp32_one_by_one"]
    out["iterations_max"] = max(s.iterations for s in last)
    out["max_relres"] = max(float(s.relres.max()) for s in last)
    out.update(batch.info())
    batch.close()
    for h in hs:
        h.close()
    return out


def run_batch_only(a):
    import torch

    from paper_2103_07329_gb300 import build as build_mod
    build_mod.build()
    torch.cuda.set_device(0)
    r = batch_form(a, seq=not a.batch_no_seq)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": 1, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": r["workload"], "form": "batched"}, "batched": r}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(a):
    from paper_2103_07329_gb300 import multirank as MR

    if MR.rank_env()[0] != 0:
        return 0
    import oracle
    from paper_2103_07329_gb300 import problems as P
    oracle.build()
    A = make_matrix(a)
    h = oracle.Hierarchy(A)
    Bm = P.rhs_uniform(A.n, a.ref_cols, 0, m_draw=max(a.m, a.ref_cols))

    def solve(Bm, tol, maxit):
        return oracle_solve(h, a, Bm)
    for _ in range(a.warmup):
        solve(Bm, a.tol, a.maxit)
    times, solved = [], 0
    for _ in range(a.steps):
        t0 = time.perf_counter()
        r = solve(Bm, a.tol, a.maxit)
        times.append(time.perf_counter() - t0)
        solved += int(np.sum((r.status == 0) & (r.relres <= a.tol)))
    total = sum(times)
    value = solved / total
    cores = oracle_threads()
    sample = (f"{a.ref_cols} of the {a.m} columns per step (a per-column rate: the oracle's "
              f"multi-column solve runs at about the same rate per column), full matrix, oracle "
              f"setup untimed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a, A), "matrix": a.matrix, "grid": a.grid, "n": A.n,
                       "nnz": A.nnz, "m": a.m, "method": a.method, "tol": a.tol},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iters": r.iters.tolist()}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(a):
    import torch

    from paper_2103_07329_gb300 import binding as B
    from paper_2103_07329_gb300 import build as build_mod
    from paper_2103_07329_gb300 import problems as P

    from paper_2103_07329_gb300 import multirank as MR

    rank, world, local = MR.rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build_mod.build()
    A = make_matrix(a)
    t0 = time.perf_counter()
    h = B.Hierarchy(A)
    t_setup = time.perf_counter() - t0
    method = METHODS[a.method]
    Bm = P.rhs_uniform(A.n, a.m, MR.rhs_seed(rank), m_draw=max(a.m, 32))
    Bd = torch.from_numpy(Bm).cuda()
    X = torch.empty_like(Bd)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def solves(hh, Bb, Xb, steps, prec=B.PREC_FP64, meth=method):
        """`steps` complete solves on the current stream, bracketed by CUDA
        events; returns (ms, columns that reached tol, last stats)."""
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ok, st = 0, None
        for _ in range(steps):
            st = hh.solve(Bb, Xb, a.tol, a.maxit, meth, precond=prec)
            ok += int(np.sum((st.status == 0) & (st.relres <= a.tol)))
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), ok, st

    def row_timing(hh, base):
        """Totals and per-level A-product figures of the row kernel launches
        recorded since timing was enabled (base 0: FP64 blocks, 3: FP32)."""
        tot = dict(launches=0, ms=0.0, flops=0.0, bytes=0.0)
        levels = []
        for l in range(hh.levels):
            for which in (0, 1, 2):
                if which and l + 1 == hh.levels:
                    continue
                r = hh.timing_read(l, base + which)
                for k in tot:
                    tot[k] += r[k]
                if which == 0 and r["launches"]:
                    levels.append(dict(level=l, launches=r["launches"], ms=round(r["ms"], 3),
                                       tflops=round(r["flops"] / r["ms"] / 1e9, 4),
                                       gbs=round(r["bytes"] / r["ms"] / 1e6, 1)))
        return tot, levels

    for _ in range(a.warmup):
        h.solve(Bd, X, a.tol, a.maxit, method)
    # timed region: K complete solves on the product path (CUDA graphs of the
    # steady iteration, no per-launch events)
    clocks = Clocks(local)
    barrier()
    clocks.start()
    l0 = B.kernel_launches()
    ms, solved, st = solves(h, Bd, X, a.steps)
    barrier()
    launches = B.kernel_launches() - l0
    ck = clocks.stop()
    stats = [st]
    value, t_max, solved_all = MR.job_throughput(ms / 1e3, solved, dist, "cuda")

    # roofline of the dominant kernel, the fused sparse row kernel (A, P, R of
    # all levels): a separate instrumented pass of the same K solves, every
    # row launch bracketed by CUDA events on the solve's stream
    h.timing_enable(True)
    barrier()
    ms_i, solved_i, _ = solves(h, Bd, X, a.steps)
    tot, per_level = row_timing(h, 0)
    h.timing_enable(False)
    achieved_tf = tot["flops"] / tot["ms"] / 1e9 if tot["ms"] > 0 else 0.0
    achieved_gbs = tot["bytes"] / tot["ms"] / 1e6 if tot["ms"] > 0 else 0.0
    hbm, hbm_kind = measured_hbm()
    traffic = kernel_traffic(a, tot["bytes"] / max(1, tot["launches"]))
    roofline = {"bound": "alu", "achieved": round(achieved_tf, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(achieved_tf / FP64_PEAK_TFLOPS, 4),
                "traffic": traffic,
                "traffic_unit": ("bytes per launch (DRAM read + write, ncu on the 96^3 solve, scaled "
                                 "by algorithmic bytes per launch)"),
                "algorithmic_bytes_per_launch": round(tot["bytes"] / max(1, tot["launches"])),
                "kernel": "k_rows<NV=32> fused SpMM row kernel, all levels (A, P, R)",
                "launches": tot["launches"], "avg_launch_ms": round(tot["ms"] / max(1, tot["launches"]), 4),
                "peak_kind": "derived FP64 FMA peak (152 SM x 2 DFMA/clk x 2.07 GHz)",
                "hbm": {"achieved_gbs": round(achieved_gbs, 1), "peak_gbs": hbm,
                        "frac": round(achieved_gbs / hbm, 4), "peak_kind": hbm_kind},
                "share_of_step": round(tot["ms"] / ms_i, 4),
                "pass": "instrumented pass of the same solves (per-launch CUDA events, no graphs)",
                "instrumented_value": round(solved_i / (ms_i / 1e3), 3)}

    def precision_forms(hh, Bb, Xb, value64, X64, index16=False):
        """The FP32 and bf16 preconditioners inside the FP64 outer loop on the
        same system: RHS/s (product path), the FP32 row kernel's algorithmic
        GB/s from an instrumented pass, and per column the relative error
        ||X_form - X_fp64|| / ||X_fp64|| against the FP64 GPU solution.  With
        index16 also both forms with 16-bit column indices."""
        out = {}
        x64 = X64.cpu().numpy()
        variants = [("fp32", B.PREC_FP32, False), ("bf16", B.PREC_BF16, False)]
        if index16:
            variants += [("fp32_index16", B.PREC_FP32, True), ("bf16_index16", B.PREC_BF16, True)]
        for name, prec, i16 in variants:
            hh.set_index16(i16)
            hh.solve(Bb, Xb, a.tol, a.maxit, method, precond=prec)
            barrier()
            fms, fok, fst = solves(hh, Bb, Xb, a.steps, prec)
            fv, ft, _ = MR.job_throughput(fms / 1e3, fok, dist, "cuda")
            xf = Xb.cpu().numpy()
            err = np.linalg.norm(xf - x64, axis=0) / np.linalg.norm(x64, axis=0)
            hh.timing_enable(True)
            barrier()
            ims, _, _ = solves(hh, Bb, Xb, a.steps, prec)
            f32, flev = row_timing(hh, 3)
            hh.timing_enable(False)
            gbs = f32["bytes"] / f32["ms"] / 1e6 if f32["ms"] > 0 else 0.0
            lv0 = [x for x in flev if x["level"] == 0]
            out["mixed_" + name] = {
                "value": fv, "speedup_vs_fp64": fv / value64, "ms_per_step": 1e3 * ft / a.steps,
                "iters": fst.iters.tolist(), "max_relres": float(fst.relres.max()),
                "error_vs_fp64_per_column": [float(f"{e:.3e}") for e in err],
                "precond_row_kernel": {"bound": "hbm", "achieved_gbs": round(gbs, 1), "peak_gbs": hbm,
                                       "frac": round(gbs / hbm, 4), "launches": f32["launches"],
                                       "share_of_step": round(f32["ms"] / ims, 4),
                                       "level0_frac": round(lv0[0]["gbs"] / hbm, 4) if lv0 else None,
                                       "pass": "instrumented pass of the same solves"},
                "roofline_levels": flev}
        hh.set_index16(False)
        return out

    def precision_workload():
        """The precision workload: 3-D 7-point variable-coefficient diffusion
        on precision_grid^3 cells with lognormal (sigma 1, seed 1) cell
        coefficients and m = 16, plain FP64 against the FP32 and bf16
        preconditioners (outer FP64 flexible PCG, same tolerance)."""
        g = a.precision_grid
        Av = P.diffusion7(g, P.lognormal_cells(g, 1.0, 1))
        t0 = time.perf_counter()
        hv = B.Hierarchy(Av)
        t_set = time.perf_counter() - t0
        Bv = P.rhs_uniform(Av.n, 16, MR.rhs_seed(rank), m_draw=32)
        Bvd = torch.from_numpy(Bv).cuda()
        Xv = torch.empty_like(Bvd)
        hv.solve(Bvd, Xv, a.tol, a.maxit, method)
        barrier()
        vms, vok, vst = solves(hv, Bvd, Xv, a.steps)
        v64, vt, _ = MR.job_throughput(vms / 1e3, vok, dist, "cuda")
        out = {"workload": (f"3-D 7-point variable-coefficient diffusion {g}^3 (n={Av.n}, nnz={Av.nnz}), "
                            f"cell k lognormal sigma=1 seed 1, m=16 RHS uniform[-1,1) seed 0, "
                            f"{a.method.upper()} + classical RS AMG V(1,1) Chebyshev-2, tol {a.tol:g}"),
               "levels": hv.levels, "op_complexity": round(hv.op_complexity, 4), "setup_s": round(t_set, 2),
               "fp64": {"value": v64, "ms_per_step": 1e3 * vt / a.steps, "iters": vst.iters.tolist(),
                        "max_relres": float(vst.relres.max())}}
        out.update(precision_forms(hv, Bvd, Xv, v64, Xv.clone(), index16=True))
        hv.close()
        del Bvd, Xv
        return out

    def spmm_form():
        """The fine-level sparse product alone, y = A x on the benchmark's
        blocks (m columns), FP64 blocks and FP32 blocks (FP32 and bf16 values of
        A): algorithmic GB/s of the row kernel by CUDA events over 20 products
        after 3 warm-ups, against the measured HBM copy peak."""
        out = {}
        Yd = torch.empty_like(Bd)
        for name, prec in (("fp64", B.PREC_FP64), ("fp32", B.PREC_FP32), ("bf16", B.PREC_BF16)):
            def prod():
                if prec == B.PREC_FP64:
                    h.spmm(0, 0, Bd, Yd)
                else:
                    h.spmm_precond(prec, 0, 0, Bd, Yd)
            for _ in range(3):
                prod()
            h.timing_enable(True)
            for _ in range(20):
                prod()
            r = h.timing_read(0, 0 if prec == B.PREC_FP64 else 3)
            h.timing_enable(False)
            gbs = r["bytes"] / r["ms"] / 1e6
            out[name] = {"launches": r["launches"], "us_per_product": round(1e3 * r["ms"] / r["launches"], 1),
                         "achieved_gbs": round(gbs, 1), "peak_gbs": hbm, "frac_of_hbm": round(gbs / hbm, 4),
                         "tflops": round(r["flops"] / r["ms"] / 1e9, 4),
                         "algorithmic_bytes_per_product": round(r["bytes"] / r["launches"])}
        del Yd
        return out

    def parity_case_form():
        """The small parity workload: 7-point Poisson 32^3, m = 4 (seed 0), PCG
        to tol, plain FP64 and with the FP32 preconditioner; RHS/s over
        max(steps, 20) solves after 3 warm-ups (CUDA graphs on)."""
        As = P.poisson7(32)
        hs = B.Hierarchy(As)
        Bs = torch.from_numpy(P.rhs_uniform(As.n, 4, 0)).cuda()
        Xs = torch.empty_like(Bs)
        out = {"workload": (f"3-D 7-point Poisson 32^3 (n={As.n}, nnz={As.nnz}), m=4 RHS uniform[-1,1) "
                            f"seed 0, PCG + classical RS AMG V(1,1) Chebyshev-2, tol {a.tol:g}")}
        for name, prec in (("fp64", B.PREC_FP64), ("fp32", B.PREC_FP32)):
            for _ in range(3):
                hs.solve(Bs, Xs, a.tol, a.maxit, method, precond=prec)
            pms, pok, pst = solves(hs, Bs, Xs, max(a.steps, 20), prec)
            out[name] = {"value": pok / (pms / 1e3), "ms_per_solve": pms / max(a.steps, 20),
                         "iters": pst.iters.tolist(), "max_relres": float(pst.relres.max())}
        hs.close()
        return out

    forms = None
    if not a.no_forms:
        forms = {"spmm_level0": spmm_form(), "parity_case_32": parity_case_form()}
        X64 = X.clone()
        forms.update(precision_forms(h, Bd, X, value, X64))
        del X64
        if not a.no_precision:
            forms["precision_var%d" % a.precision_grid] = precision_workload()

    # learned initial guess: held-out 64^3 GRF-coefficient diffusion systems,
    # 32 smooth right-hand sides each, solved from X0 = 0 and from the trained
    # network's X0 (prediction time included), all to the same tolerance
    if not a.no_forms and not a.no_warm:
        from paper_2103_07329_gb300 import warmstart as W
        params, c, info = W.load()
        r = W.evaluate(params, c, info["N"], nfields=2, tol=a.tol, sweeps=3, log=None)
        recs = r["records"]
        forms["warm_start_64"] = {
            "workload": (f"3-D 7-point diffusion {info['N']}^3, log k Gaussian random field "
                         f"(corr. 0.1, sigma 1), 32 smooth GRF right-hand sides (corr. 0.2), held-out "
                         f"fields {W.TEST_SEED}..{W.TEST_SEED + 1}, PCG + AMG FP64, tol {a.tol:g}"),
            "rhs_per_s_plain": r["rhs_per_s_plain"], "rhs_per_s_warm": r["rhs_per_s_warm"],
            "rhs_per_s_warm_smoothed": r["rhs_per_s_warm_smooth"],
            "speedup_vs_plain": r["speedup"], "speedup_smoothed_vs_plain": r["speedup_smooth"],
            "iters_plain": [x["iters_plain"] for x in recs], "iters_warm": [x["iters_warm"] for x in recs],
            "iters_warm_smoothed": [x["iters_warm_smooth"] for x in recs],
            "mean_iters_per_column_plain": [round(x["mean_iters_plain"], 3) for x in recs],
            "mean_iters_per_column_warm": [round(x["mean_iters_warm"], 3) for x in recs],
            "x0_anorm_error": [round(x["x0_anorm_error"], 4) for x in recs],
            "x0_relres": [round(x["x0_relres"], 4) for x in recs],
            "ms_predict": [round(x["ms_predict"], 3) for x in recs],
            "max_relres": max(max(x["relres_max_warm"], x["relres_max_warm_smooth"]) for x in recs),
            "training": {k: info[k] for k in ("fields", "pairs", "epochs", "finetune_epochs", "train_seconds")}}

    if not a.no_forms and not a.no_batch:
        forms["batched_64"] = batch_form(a)

    # end to end through the host-buffer entry point: H2D of B and D2H of X inside
    e2e = None
    if not a.no_e2e:
        Bh = torch.from_numpy(Bm).pin_memory()
        Xh = torch.empty_like(Bh).pin_memory()
        Bh_np, Xh_np = Bh.numpy(), Xh.numpy()
        h.solve_host(Bh_np, Xh_np, a.tol, a.maxit, method)
        barrier()
        t0 = time.perf_counter()
        s2 = 0
        for _ in range(a.steps):
            st = h.solve_host(Bh_np, Xh_np, a.tol, a.maxit, method)
            s2 += int(np.sum((st.status == 0) & (st.relres <= a.tol)))
        barrier()
        e2e_value, _, _ = MR.job_throughput(time.perf_counter() - t0, s2, dist, "cuda")
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(Bm.nbytes),
               "d2h_bytes_per_step": int(Bm.nbytes)}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        del Bd, X
        v, info = cpu_baseline(a, A)
        cpu = {"value": v, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
               "sample": f"the first {a.cpu_cols} of the {a.m} columns of the same workload, "
                         f"one {a.cpu_cols}-column oracle solve to {a.tol:g} (oracle setup "
                         f"{info['t_setup']:.1f} s untimed, solve {info['t_solve']:.1f} s, "
                         f"iterations {info['iters']}); OpenMP over the SpMM row loops, the "
                         f"rest single-threaded"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": 1e3 * t_max / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(a, A), "matrix": a.matrix, "grid": a.grid,
                           "n": A.n, "nnz": A.nnz, "m": a.m, "method": a.method, "tol": a.tol,
                           "form": "plain FP64", "levels": h.levels,
                           "op_complexity": round(h.op_complexity, 4),
                           "l2": "inputs larger than L2 (each n x m block is "
                                 f"{Bm.nbytes / 1e9:.2f} GB vs 129 MB L2)",
                           "parallelism": f"{world} independent RHS blocks (one per GPU)",
                           "setup_s": round(t_setup, 2)},
                "iters": stats[-1].iters.tolist(), "vcycles_per_step": stats[-1].vcycles,
                "max_relres": float(stats[-1].relres.max()),
                "roofline": roofline, "roofline_levels": per_level,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": ck, "gpu_launches": int(launches),
                "forms": forms}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_sweep(a):
    """One JSON line per (m, method, preconditioner precision) on the chosen
    matrix: RHS/s over `steps` solves after one warm-up, iterations, and the
    row kernel's achieved FP64 TFLOP/s or FP32 GB/s per level."""
    import torch

    from paper_2103_07329_gb300 import binding as B
    from paper_2103_07329_gb300 import build as build_mod
    from paper_2103_07329_gb300 import problems as P

    build_mod.build()
    A = make_matrix(a)
    t0 = time.perf_counter()
    h = B.Hierarchy(A)
    setup = time.perf_counter() - t0
    if a.index16:
        h.set_index16(True)
    hbm = measured_hbm()[0]
    for m in [int(v) for v in a.sweep_ms.split(",")]:
        Bm = P.rhs_uniform(A.n, m, 0, m_draw=32)
        Bd = torch.from_numpy(Bm).cuda()
        X = torch.empty_like(Bd)
        for method_name in a.sweep_methods.split(","):
            method = METHODS[method_name]
            for form, prec in (("fp64", B.PREC_FP64), ("mixed_fp32", B.PREC_FP32),
                               ("mixed_bf16", B.PREC_BF16)):
                if method == B.BICGSTAB_PIPELINED and prec != B.PREC_FP64:
                    continue  # its recurrences need a linear preconditioner
                force = a.fp64_split if prec == B.PREC_FP64 else a.fp32_split
                if force >= 0:
                    for l in range(h.levels):
                        n_l, nnz_l, _ = h.level_info(l)
                        if nnz_l / max(n_l, 1) > a.split_max_row:
                            continue
                        for which in (0, 1, 2):
                            if which == 0 or l + 1 < h.levels:
                                try:
                                    h.set_split(m, prec, l, which, force)
                                except B.XamgError:
                                    pass
                h.solve(Bd, X, a.tol, a.maxit, method, precond=prec)
                h.timing_enable(True)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                solved = 0
                for _ in range(a.steps):
                    st = h.solve(Bd, X, a.tol, a.maxit, method, precond=prec)
                    solved += int(np.sum((st.status == 0) & (st.relres <= a.tol)))
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / a.steps
                base = 0 if prec == B.PREC_FP64 else 3
                levels = []
                for l in range(h.levels - 1):
                    r = h.timing_read(l, base)
                    if r["launches"]:
                        levels.append({"level": l, "ms_per_launch": round(r["ms"] / r["launches"], 4),
                                       "tflops": round(r["flops"] / r["ms"] / 1e9, 3),
                                       "gbs": round(r["bytes"] / r["ms"] / 1e6, 1)})
                h.timing_enable(False)
                print(json.dumps({"matrix": a.matrix, "grid": a.grid, "n": A.n, "m": m,
                                  "index16": a.index16, "fp32_split": a.fp32_split, "fp64_split": a.fp64_split,
                                  "split_max_row": a.split_max_row,
                                  "method": method_name, "form": form,
                                  "rhs_per_s": round(solved / (ms * a.steps / 1e3), 2),
                                  "ms_per_solve": round(ms, 3), "iters": int(st.iters.max()),
                                  "max_relres": float(st.relres.max()), "setup_s": round(setup, 1),
                                  "hbm_peak_gbs": hbm, "levels": levels}), flush=True)
    return 0


SPLIT_NAMES = {1: ["stream1x256", "lanes16", "stream1x1024", "stream4x1024", "stream32x1024",
                    "stream1x512", "stream2x512"],
               0: ["narrow", "row_per_warp"]}


def split_names(m, prec_fp64):
    """Names of the row-split candidates of xamg_set_split for m columns."""
    if m == 1:
        return SPLIT_NAMES[1]
    mp = 1 << (m - 1).bit_length()
    if mp in (2, 4):
        return SPLIT_NAMES[0] + ["stream_lane_per_row"]
    if not prec_fp64 and mp >= 8:
        return SPLIT_NAMES[0] + ["staged"]
    if prec_fp64 and mp >= 8:
        return SPLIT_NAMES[0] + ["pipelined", "narrow_2col", "pipelined_2col"]
    return SPLIT_NAMES[0]


def run_split_table(a):
    """Microseconds per product y = M x of every level and operator under
    every row split (xamg_set_split), 20 timed products after 3 warm-ups: FP64
    blocks, or with --precond fp32 / bf16 the preconditioner's FP32 blocks."""
    import torch

    from paper_2103_07329_gb300 import binding as B
    from paper_2103_07329_gb300 import build as build_mod

    build_mod.build()
    A = make_matrix(a)
    h = B.Hierarchy(A)
    L = h.levels
    info = [h.level_info(l) for l in range(L)]
    prec = {"fp64": B.PREC_FP64, "fp32": B.PREC_FP32, "bf16": B.PREC_BF16}[a.precond]
    names = split_names(a.m, prec == B.PREC_FP64)

    def product(l, which, X, Y):
        if prec == B.PREC_FP64:
            h.spmm(l, which, X, Y)
        else:
            h.spmm_precond(prec, l, which, X, Y)

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for l in range(L):
        for which in (0, 1, 2):
            if which > 0 and l + 1 >= L:
                continue
            n_out = info[l][0] if which in (0, 1) else info[l + 1][0]
            n_src = info[l][0] if which in (0, 2) else info[l + 1][0]
            X = torch.rand(n_src, a.m, dtype=torch.float64, device="cuda")
            Y = torch.empty(n_out, a.m, dtype=torch.float64, device="cuda")
            us = {}
            for c, name in enumerate(names):
                h.set_split(a.m, prec, l, which, c)
                for _ in range(3):
                    product(l, which, X, Y)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(20):
                    product(l, which, X, Y)
                e1.record()
                torch.cuda.synchronize()
                us[name] = round(e0.elapsed_time(e1) / 20 * 1e3, 1)
            h.set_split(a.m, prec, l, which, -1)
            nnz = info[l][1] if which == 0 else info[l][2]
            print(json.dumps({"matrix": a.matrix, "grid": a.grid, "m": a.m, "precond": a.precond, "level": l,
                              "op": "APR"[which], "rows": n_out, "nnz": nnz,
                              "avg_row": round(nnz / max(n_out, 1), 1), "us": us}), flush=True)
    return 0


def run_spmm_only(a):
    """Four products y = A_l x with the default split, for kernel captures
    (FP32 blocks for --precond fp32 / bf16: the preconditioner's product)."""
    import torch

    from paper_2103_07329_gb300 import binding as B
    from paper_2103_07329_gb300 import build as build_mod

    build_mod.build()
    A = make_matrix(a)
    h = B.Hierarchy(A)
    if a.index16:
        h.set_index16(True)
    n, nnz, _ = h.level_info(a.level)
    X = torch.rand(n, a.m, dtype=torch.float64, device="cuda")
    Y = torch.empty(n, a.m, dtype=torch.float64, device="cuda")
    prec = {"fp64": B.PREC_FP64, "fp32": B.PREC_FP32, "bf16": B.PREC_BF16}[a.precond]
    for _ in range(4):
        if prec == B.PREC_FP64:
            h.spmm(a.level, 0, X, Y)
        else:
            h.spmm_precond(prec, a.level, 0, X, Y)
    torch.cuda.synchronize()
    print(json.dumps({"matrix": a.matrix, "grid": a.grid, "level": a.level, "n": n, "nnz": nnz, "m": a.m,
                      "precond": a.precond, "index16": a.index16, "products": 4}))
    return 0


def run_tail_table(a):
    """Milliseconds per PCG solve (tol 1e-8) of small systems with the fused
    coarse tail (xamg_set_tail, 131072 elements) and without it, CUDA graphs
    on, after five warm-up solves; CUDA events around max(steps, 20) solves."""
    import torch

    from paper_2103_07329_gb300 import binding as B
    from paper_2103_07329_gb300 import build as build_mod
    from paper_2103_07329_gb300 import problems as P

    build_mod.build()
    cases = [("poisson7", 32, 4), ("poisson7", 32, 32), ("poisson7", 64, 4), ("poisson7", 64, 32),
             ("diffusion7", 64, 32)]
    steps = max(a.steps, 20)
    for kind, grid, m in cases:
        A = P.poisson7(grid) if kind == "poisson7" else P.diffusion7(grid, P.lognormal_cells(grid, 1.0, 1))
        Bm = P.rhs_uniform(A.n, m, 0, m_draw=32)
        Bd = torch.from_numpy(Bm).cuda()
        X = torch.empty_like(Bd)
        for prec in (B.PREC_FP64, B.PREC_FP32):
            for elems in (131072, 0):
                h = B.Hierarchy(A)
                h.set_tail(elems)
                for _ in range(5):
                    st = h.solve(Bd, X, a.tol, a.maxit, precond=prec)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                l0 = B.kernel_launches()
                e0.record()
                for _ in range(steps):
                    st = h.solve(Bd, X, a.tol, a.maxit, precond=prec)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                print(json.dumps({"matrix": kind, "grid": grid, "m": m, "precond": "fp64" if prec == 0 else "fp32",
                                  "tail_first_level": h.tail_info(m), "ms_per_solve": round(ms, 4),
                                  "rhs_per_s": round(m / ms * 1e3, 1), "iters": int(st.iters.max()),
                                  "launches_per_solve": (B.kernel_launches() - l0) // steps}), flush=True)
                h.close()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.sweep:
        return run_sweep(a)
    if a.split_table:
        return run_split_table(a)
    if a.spmm_only:
        return run_spmm_only(a)
    if a.tail_table:
        return run_tail_table(a)
    if a.batch_only:
        return run_batch_only(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
