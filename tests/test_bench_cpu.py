"""bench.py's host-only parts: the reference arm (the FP64 oracle timed on the host cores)
prints one JSON line with the keys the benchmark contract asks for, the oracle timing helper
advances exactly what it reports, and the warm-up floor is enforced before any GPU work."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench

    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["config"]["workload"] == bench.workload().name
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_oracle_timing_helper_counts_what_it_runs():
    import bench
    from paper_2403_06706_gb300 import synth

    wl = synth.c1_plain_fp64()
    nodes = synth.wind_grid(wl.wind, dtype=np.float64)
    n, k, el = bench._oracle_run(wl, nodes, 64, 2, n_steps=10)
    assert (n, k) == (64, 10) and el > 0
    n, k, el = bench._oracle_run(wl, nodes, 32, 1, seconds=0.05, pilot_steps=5)
    assert n == 32 and k >= 5 and el > 0


@pytest.mark.parametrize("impl", ["ours", "reference"])
def test_warmup_below_three_is_refused(impl):
    r = subprocess.run([sys.executable, "bench.py", "--impl", impl, "--warmup", "2"], cwd=ROOT,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "--warmup must be >= 3" in r.stderr
