"""The benchmark's JSON contract on the CPU: the reference arm (the oracle timed on the host
cores) prints one line with every key the contract names, for a small grid."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--nx", "16", "--steps", "1", "--warmup", "3", *extra],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    r = _line()
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "cpu_baseline"):
        assert k in r, k
    assert r["impl"] == "reference" and r["value"] > 0 and r["steps"] == 1 and r["warmup"] == 3
    assert r["higher_is_better"] is True and r["scaling"] == "weak" and r["vs_baseline"] is None
    assert r["config"]["grid"] == [16, 16, 16] and "16x16x16" in r["config"]["workload"]
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"]
    assert "16^3 grid" in cb["sample"] and "full Lambda iteration" in cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_follows_the_scheme():
    r = _line("--scheme", "face")
    assert "face-hitting" in r["config"]["workload"] and "face-hitting" in r["cpu_baseline"]["sample"]


def test_one_thread_oracle_iteration():
    """The single-thread figure of the CPU baseline: one oracle iteration in a process whose
    OpenMP runtime has one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-iteration", "12"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, check=True, env=env)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["cores"] == 1 and r["value"] > 0 and "12^3 grid" in r["sample"]
