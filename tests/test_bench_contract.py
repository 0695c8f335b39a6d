"""The benchmark's reference arm on the host: one JSON line with the native arm's metric, unit and
direction, the oracle's timing as cpu_baseline and an end-to-end record without transfers."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = run_bench("--impl", "reference", "--steps", "2", "--warmup", "0", "--reference-sizes", "160,240")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"].startswith("Fisher-BT iters/s and Cholesky TFLOP/s")
    assert d["unit"] == "iters/s" and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 0
    assert d["config"]["workload"] == "n65536" and d["config"]["n"] == 65536
    # the timed steps' own duration, and the fitted time per iteration at the full size
    assert 0 < d["ms_per_step"] < 60_000
    assert d["extrapolated_s_per_iteration"] == pytest.approx(1.0 / d["value"])
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "n=160" in cb["sample"] and "n=240" in cb["sample"] and "a n^2 + b n^3" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_oracle_extrapolation_recovers_a_cubic_plus_quadratic_law():
    sys.path.insert(0, ROOT)
    import bench
    a, b = 3e-7, 2e-10
    times = {m: [a * m ** 2 + b * m ** 3] for m in (1024, 2048, 4096)}
    t, a2, b2 = bench.oracle_extrapolation(times, 65536)
    assert a2 == pytest.approx(a, rel=1e-9) and b2 == pytest.approx(b, rel=1e-9)
    assert t == pytest.approx(a * 65536 ** 2 + b * 65536 ** 3, rel=1e-9)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], cwd=ROOT,
                       capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_other_precisions_are_refused_for_the_single_field_line():
    r = run_bench("--precision", "mixed")
    assert r.returncode != 0 and "--compare-mixed" in r.stderr
