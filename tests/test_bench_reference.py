"""bench.py's reference arm (the float64 oracle on the host cores) on a small
workload: one JSON line with the contract's keys, the oracle's time scaled by
its recorded iteration count, and an e2e entry that copies nothing; a workload
without a recorded count prints an "unavailable" line instead."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(workload):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload, "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_reference("16x16x16x32")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["steps"] == 1
    assert d["config"]["workload"] == "wilson_eo_16x16x16x32"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # value = the per-iteration time times the oracle's recorded iteration count for this workload
    n_iter = d["value"] / (d["ms_per_step"] / 1e3)
    assert abs(n_iter - round(n_iter)) < 1e-6 and round(n_iter) > 100


def test_reference_arm_without_a_recorded_count():
    d = run_reference("8x8x8x8")
    assert d["impl"] == "reference" and "unavailable" in d
