"""bench.py's step and buffer-set arithmetic (CPU), and the driver's exact
command on a GPU (the JSON line it prints)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("steps,sets", [(20, 32), (1, 32), (32, 32), (33, 32), (2048, 32), (20, 1), (7, 3)])
def test_timing_plan_times_exactly_k_steps(steps, sets):
    import bench
    full, tail, secondary = bench.timing_plan(steps, sets)
    assert full * sets + tail == steps
    assert 0 <= tail < sets
    assert secondary >= 1


def test_timing_plan_rejects_empty():
    import bench
    with pytest.raises(ValueError):
        bench.timing_plan(0, 32)


@pytest.mark.gpu
@pytest.mark.slow
def test_bench_driver_command_prints_a_full_line():
    """`bench.py --gpus 1 --steps 20 --warmup 5` (fewer steps than buffer
    sets), with the slow sections left out: one JSON line carrying the
    roofline, the CPU baseline, the end-to-end rate and the clocks."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "1", "--steps", "20", "--warmup", "5",
           "--no-warm", "--no-rect", "--no-batched"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["steps"] == 20 and d["warmup"] == 5 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert abs(d["value"] * d["ms_per_step"] / 1000.0 - 1.0) < 1e-9
    assert d["dtype"] == "f64" and "10,000-bus" in d["config"]["workload"]
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and 0 < rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert rf["kernel_us"] * 1e-3 <= d["ms_per_step"] * 1.5
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["host_cores"] >= 1 and cb["value"] > 0
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] >= 20
    assert d["clocks"]["samples"] >= 1


@pytest.mark.parametrize("kernel", ["fused", "branch", "bus"])
def test_stored_counters_and_their_commands(kernel):
    """The per-launch counters bench.py reads from the committed ncu
    summaries parse, and each names the whole ncu command that took them
    (clocks left alone, a bench.py run of committed files)."""
    import bench
    assert bench.profile_value(kernel, "dram_bytes_per_launch") > 0
    assert bench.profile_value(kernel, "fp64_flops_per_launch") > 0
    src = bench.profile_source(kernel)
    cmd = src["ncu_command"]
    assert cmd.startswith("ncu ") and "--clock-control none" in cmd
    assert "python bench.py" in cmd and "\\" not in cmd
