"""The benchmark's one-line JSON contract: the reference arm (the oracle on
the host cores) on CPU, the headline line on a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

BASE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _run(args, timeout):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                         timeout=timeout, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--steps", "2", "--warmup", "3"], timeout=600)
    for k in BASE_KEYS:
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["unit"] == "moves/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


@pytest.mark.gpu
def test_headline_line():
    d = _run(["--steps", "5", "--warmup", "3", "--no-batched", "--no-cpu", "--no-smart", "--no-energy"], timeout=900)
    for k in BASE_KEYS + ("roofline", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["unit"] == "moves/s" and d["value"] > 0 and d["steps"] == 5 and d["warmup"] == 3
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and 0 < r["frac"] < 1.5
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    iss = d["issue_roofline"]  # null when the committed ncu summary is of another kernel source
    if iss is not None:
        assert iss["bound"] == "alu" and 0 < iss["frac"] < 1.05
        assert abs(iss["floor_ms"] / r["move_ms"] - iss["frac"]) < 1e-9
    assert d["gpu_launches"] >= d["steps"]  # at least the move kernel of every timed step
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["clocks"]["sm_mhz"] > 0 and isinstance(d["clocks"]["reasons"], list)
    assert "l2" in d["config"] and d["dtype"] == "f32" and d["data"] == "synthetic"
    st = d["step_ms_stats"]
    assert 0 < st["min"] <= st["median"] <= st["max"] and st["min"] <= d["ms_per_step"] <= st["max"]
    c2 = d["config2"]  # the second full-size melt, timed in the same run
    assert c2["n_beads"] == 1048576 * 64 and c2["n_cells"] == 256 ** 3 and c2["steps"] == 5
    assert abs(c2["frac"] - c2["achieved_gbs"] / r["peak"]) < 1e-9 and 0 < c2["frac"] < 1.5
    assert c2["value"] > 0 and c2["move_ms"] <= c2["ms_per_step"] * 1.05


@pytest.mark.gpu
def test_partitioned_line_at_one_rank():
    # the chain-partition mode at N = 1: the whole system as one partition,
    # the exchange a no-op; its line keeps the contract's keys
    d = _run(["--partition", "--partition-workload", "melt_131072x32", "--steps", "5", "--warmup", "3"],
             timeout=900)
    for k in BASE_KEYS + ("roofline", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["scaling"] == "strong" and d["n_gpus"] == 1 and d["value"] > 0
    assert d["config"]["n_beads"] == 131072 * 32 and d["gpu_launches"] == 5
    r = d["roofline"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9 and 0 < r["frac"] < 1.5
