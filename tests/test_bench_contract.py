"""The benchmark's JSON line: the reference arm (the CPU oracle, runnable
here) prints the contract's keys, other ranks stay silent, and the stored
bench lines under profiles/ carry every key the contract asks for with
self-consistent values."""
import glob
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REJECTED_REASONS = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}


def _bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    r = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, env=e, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def _common(d):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["data"] == "synthetic" and isinstance(d["config"]["workload"], str)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["unit"] == d["unit"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] >= 0 and e["d2h_bytes_per_step"] >= 0


def test_reference_arm_line():
    lines = _bench("--impl", "reference", "--config", "1", "--steps", "1", "--warmup", "1")
    d = json.loads(lines[-1])
    _common(d)
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["config_id"] == 1


def test_reference_arm_other_ranks_print_nothing():
    lines = _bench("--impl", "reference", "--config", "1", "--steps", "1", "--warmup", "1",
                   env={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert lines == []


STORED = sorted(glob.glob(os.path.join(ROOT, "profiles", "bench_config*.json")))


@pytest.mark.parametrize("path", STORED, ids=[os.path.basename(p) for p in STORED])
def test_stored_bench_lines_keep_the_contract(path):
    d = json.loads(open(path).read().strip().splitlines()[-1])
    _common(d)
    assert d["steps"] >= 1 and d["warmup"] >= 3
    n = d["config"]["n_points_per_gpu"] * d["n_gpus"]
    assert abs(d["value"] - n / (d["ms_per_step"] / 1e3)) <= 1e-3 * d["value"]
    r = d["roofline"]
    assert r["bound"] in ("hbm", "tensor", "alu") and r["unit"] in ("GB/s", "TFLOP/s")
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert r["traffic"] is None or r["traffic"] > 0
    assert d["gpu_launches"] > 0
    c = d["clocks"]
    assert c["sm_mhz"] > 0 and c["sm_max_mhz"] > 0 and not (set(c["reasons"]) & REJECTED_REASONS)
    assert d["cpu_baseline"]["cores"] > 1
    e = d["e2e"]
    assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
