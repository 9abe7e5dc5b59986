"""The benchmark's reference arm (the CPU oracle) keeps the JSON-line
contract: one line on rank 0 with the arm's metric, unit, direction and
workload name, a cpu_baseline describing the run and an e2e object without
host-device traffic; the other ranks print nothing and exit 0 (no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def reference_line(cores):
    p = run(["--impl", "reference", "--config", "cloth_sphere", "--steps", "2", "--warmup", "1",
             "--ref-budget", "3", "--ref-cores", str(cores)])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "steps/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1000.0 / d["value"]) < 1e-6 * d["ms_per_step"]
    assert d["config"]["workload"] == "cloth32_sphere3_fp64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == cores and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    return d


def test_reference_line_contract():
    reference_line(1)


def test_reference_line_on_several_cores():
    # two single-threaded oracles side by side: their steps per second add up
    import pytest
    if (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1) < 4:
        pytest.skip("fewer than four host cores")
    d1, d2 = reference_line(1), reference_line(2)
    assert d2["value"] > 1.2 * d1["value"]


def test_reference_other_ranks_are_silent():
    p = run(["--impl", "reference", "--config", "cloth_sphere", "--steps", "1", "--warmup", "0"],
            {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0 and p.stdout.strip() == ""
