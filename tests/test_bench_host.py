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
