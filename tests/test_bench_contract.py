"""The benchmark's reference arm on the CPU: `bench.py --impl reference` times the FP64 oracle's
whole job on the workload (one job per step, as many steps as fit its time budget) and prints one
JSON line with the keys the benchmark contract fixes (impl, metric, value, unit, the steps and
warm-up it actually ran, a cpu_baseline that describes the run and an e2e object without
host-device traffic); a rank other than 0 of a multi-process launch prints nothing and exits 0.
"""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.pop("LOCAL_RANK", None)
    if extra_env:
        env.update(extra_env)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run(None, "--workload", "disk512", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "s" and d["higher_is_better"] is False
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1000.0 * d["value"]) < 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "whole job" in cb["sample"]
    assert set(cb["phases_s"]) == {"compress", "factor", "solve"}
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("disk512")


def test_reference_arm_stops_at_its_time_budget_and_reports_the_steps_run():
    r = _run(None, "--workload", "disk512", "--steps", "50", "--warmup", "5", "--ref-budget-s", "0.01")
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["steps"] == 1 and d["warmup"] == 0 and d["steps_requested"] == 50


def test_reference_arm_other_ranks_stay_silent():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--workload", "disk512")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
