"""Host-side behaviour of bench.py (no GPU): the reference arm's JSON line
(the CPU oracle on a tiny grid) and the oracle thread count it reports."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--grid", "8",
                          "--m", "2", "--ref-cols", "2", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_reference({"OMP_NUM_THREADS": "2"})
    assert d["impl"] == "reference"
    assert d["unit"] == "RHS/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert d["config"]["grid"] == 8 and d["config"]["m"] == 2
    # both sampled columns converged in the oracle's solve
    assert len(d["iters"]) == 2 and all(0 < i <= 100 for i in d["iters"])
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_oracle_threads_follows_the_environment(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("OMP_NUM_THREADS", "3")
    assert bench.oracle_threads() == 3
    monkeypatch.delenv("OMP_NUM_THREADS")
    assert bench.oracle_threads() == os.cpu_count()


def test_split_table_names_match_the_candidate_counts():
    # --split-table times one product per xamg_set_split candidate; the
    # counts documented there: 7 at m = 1, 3 for 2 or 4 columns (the stream
    # kernel) and for FP32 blocks of 8 or more (the staged split), 5 for FP64
    # blocks of 8 or more (pipelined, and both with two columns per lane)
    sys.path.insert(0, ROOT)
    import bench
    assert len(bench.split_names(1, True)) == 7
    for m in (2, 3, 4):
        assert len(bench.split_names(m, True)) == 3 and len(bench.split_names(m, False)) == 3
    for m in (5, 8, 16, 17, 32):
        assert len(bench.split_names(m, False)) == 3
        assert len(bench.split_names(m, True)) == 5
    assert len(set(bench.split_names(32, True))) == 5
