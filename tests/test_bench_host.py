"""Host-side pieces of bench.py on the CPU: the clock sampler's summary of nvidia-smi lines (median
SM clock under load, the throttle reasons seen), the roofline object's arithmetic and choice of
roof, and the whole-job throughput over ranks."""
import math

import pytest

import bench
import torch


def sampler(lines):
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.lines = list(lines)
    return s


def test_clock_summary_median_max_and_reasons():
    lines = [
        "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
        "1995, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
        "2040, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 10.0, Not Active, Not Active, Not Active, Not Active",   # unreadable: skipped
        "2070, 2070",                                                           # short: skipped
    ]
    s = sampler(lines).summary()
    assert s["sm_mhz"] == 2040 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    s = sampler(lines + ["1500, 2070, 800.0, Active, Not Active, Active, Not Active"]).summary()
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert sampler([]).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}


def test_roofline_takes_the_roof_with_the_larger_fraction():
    # native FP64: 1e6 cells in 1 ms at 375 flops and 80 B per cell -> 0.375 TFLOP/s, 80 GB/s
    r = bench.roofline("fp64", 1e6, [1.0, 1.0], 375.0, 6681.8, "measured", None)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(0.375) and r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS, abs=0.01)
    assert r["frac"] == pytest.approx(0.375 / bench.FP64_PEAK_TFLOPS, abs=1e-4)
    assert r["hbm_frac"] == pytest.approx(80.0 / 6681.8, abs=1e-4)
    assert r["algorithmic_bytes_per_launch"] == 80e6 and r["traffic"] is None
    # FP32 with few flops per cell: the HBM roof binds
    r = bench.roofline("fp32", 1e6, [0.5], 10.0, 6681.8, "measured", 1.23e8)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(80.0) and r["frac"] == pytest.approx(80.0 / 6681.8, abs=1e-4)
    assert r["traffic"] == 1.23e8
    # double-float: the method's 375 flops per cell against the FP32 peak (0.1875 TFLOP/s, 0.0023)
    # lose to HBM (40 GB/s, 0.006); the emulating FP32 operations are reported beside it
    r = bench.roofline("df64", 1e6, [2.0], 375.0, 6681.8, "measured", None)
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(40.0) and r["unit"] == "GB/s"
    assert r["alu_frac"] == pytest.approx(0.1875 / bench.FP32_PEAK_TFLOPS, abs=1e-4)
    assert r["algorithmic_flops_per_launch"] == 375e6
    tfl = 1e6 * bench.ALG_DF_FLOPS_PER_CELL["turb_minmod"] / 2e-3 / 1e12
    assert r["emulated_fp32_tflops"] == pytest.approx(tfl, abs=1e-3)
    assert r["emulated_fp32_frac"] == pytest.approx(tfl / bench.FP32_PEAK_TFLOPS, abs=1e-4)


def test_job_value_counts_every_rank_over_the_slowest():
    assert bench.job_value(1e6, 10, 1, 100.0) == pytest.approx(100.0)      # 1e7 updates in 0.1 s
    assert bench.job_value(1e6, 10, 4, 200.0) == pytest.approx(200.0)      # 4e7 updates in 0.2 s
    assert math.isclose(bench.job_time_ms(12.5, 1, "cpu"), 12.5)


def test_e2e_summary_median_and_mean_of_the_step_times():
    # 1e6 cells; steps of 10 ms with one 100 ms stall: the median step gives 100 Mcell/s, the mean 50
    e = bench.e2e_summary([10.0, 10.0, 100.0] + [10.0] * 9, 1e6)
    assert e["steps"] == 12 and e["ms_per_step_median"] == 10.0 and e["ms_per_step_max"] == 100.0
    assert e["value"] == pytest.approx(100.0) and e["mean_value"] == pytest.approx(1e6 / 17.5 / 1e3)
    e = bench.e2e_summary([4.0, 2.0, 6.0, 8.0], 1e6)      # even count: the mean of the two middle steps
    assert e["ms_per_step_median"] == 5.0 and e["value"] == pytest.approx(200.0)


def _run_bench(args, env_extra):
    import json
    import os
    import subprocess
    import sys
    env = dict(os.environ, OMP_NUM_THREADS="2", **env_extra)
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py")] + args,
                       capture_output=True, text=True, env=env, timeout=600)
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    return r.returncode, lines


def test_reference_arm_line():
    """The reference arm (the CPU oracle on a bounded sample) prints one line with the contract's
    keys; its cores are the oracle's OpenMP threads."""
    rc, lines = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {})
    assert rc == 0 and len(lines) == 1
    line = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1 and line["n_gpus"] == 1
    assert line["higher_is_better"] is True and line["vs_baseline"] is None and "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    rc, lines = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--gpus", "2"],
                           {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert rc == 0 and lines == []


def test_oracle_leg_errors_and_attachment():
    """The CPU oracle leg computes the oracle's outputs for recorded samples (sampled cells' 5^3
    neighbourhoods, whole ghosted boxes) and attaches the normwise error per field to the headline and
    to nested forms; a GPU output off by a relative 1e-9 reads as ~1e-9."""
    import numpy as np
    import oracle
    import workloads
    U = workloads.turbulent_state(12, seed=2, mach=5.0, sedov=True).numpy()
    dx = 1.0 / 12
    cfg = oracle.config()
    dt = oracle.cfl_periodic(U, dx, cfg)
    full = oracle.step_periodic(U, dx, dt, cfg)
    cells = bench.sample_cells((12, 12, 12), 30, seed=1)
    t = torch.as_tensor(U)
    nbs = bench.neighbourhoods(t, cells, 2)
    got = full[:, cells[:, 0], cells[:, 1], cells[:, 2]].T * (1 + 1e-9)
    bench.CHECKS.clear()
    bench.CHECKS.append({"path": ("headline",), "scheme": "plm", "inputs": nbs, "got": got, "dx": dx,
                         "dt": [dt] * len(cells), "limiter": "minmod", "what": "cells"})
    Ug = oracle.fill_ghosts_periodic(U)
    bench.record_boxes(("batched", "octs"), "plm", [(Ug, full + 1e-7 * np.abs(full).max(axis=(1, 2, 3), keepdims=True), dx, dt)], "minmod", "box")
    line = {"forms": {"batched": {"octs": {}}, "other": {}}}
    bench.cpu_oracle_leg(line, 0.2)
    e = line["err_vs_oracle"]
    assert 0.5e-9 <= e["max"] <= 2e-9 and len(e["per_field"]) == 5
    assert line["forms"]["batched"]["octs"]["err_vs_oracle"]["max"] == pytest.approx(1e-7, rel=1e-3)
    assert "err_vs_oracle" not in line["forms"]["other"]
    assert line["cpu_baseline"]["kind"] == "oracle"
    bench.CHECKS.clear()
