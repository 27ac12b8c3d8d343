"""The algorithmic flop counts per cell that bench.py divides by for its roofline, recomputed with
the oracle's op-counting scalar type on a 64^3 sample of each benchmark workload."""
import importlib.util
import os

import pytest

import oracle
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench_module():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.mark.parametrize("key,limiter,kw", [
    ("turb_minmod", "minmod", dict(seed=2, mach=5.0, sigma_rho=1.0, p_over_rho=1e-4, sedov=True)),
    ("turb_mc", "mc", dict(seed=2, mach=5.0, sigma_rho=1.0, p_over_rho=1e-4, sedov=True)),
    ("mach10_mc", "mc", dict(seed=5, mach=10.0, sigma_rho=1.5, p_over_rho=1e-5, sedov=False)),
])
def test_flop_constants(key, limiter, kw):
    b = bench_module()
    U = workloads.turbulent_state(64, **kw).numpy()
    cfg = oracle.config(limiter=limiter)
    dt = oracle.cfl_periodic(U, 1 / 64, cfg)
    c = oracle.count_ops(U, 1 / 64, dt, cfg)
    assert c["per_cell"] == pytest.approx(b.ALG_FLOPS_PER_CELL[key], rel=0.01)


def test_double_float_flop_constant():
    b = bench_module()
    U = workloads.turbulent_state(64, seed=2, mach=5.0, sigma_rho=1.0, p_over_rho=1e-4, sedov=True).numpy()
    cfg = oracle.config()
    c = oracle.count_ops(U, 1 / 64, oracle.cfl_periodic(U, 1 / 64, cfg), cfg)
    df = sum(b.DF_COST[k] * v for k, v in c["by_kind"].items())
    assert df == pytest.approx(b.ALG_DF_FLOPS_PER_CELL["turb_minmod"], rel=0.01)


@pytest.mark.parametrize("precision,bytes_per_cell", [("df64", 80), ("fp64", 80), ("fp32", 40), ("mixed", 80)])
def test_step_profiles_were_taken_on_the_current_step_kernel(precision, bytes_per_cell):
    """The committed ncu summaries of the step kernel carry the hash of the kernel's sources they were
    taken on; the bench reports their DRAM traffic only while that hash matches, so a change to the
    step kernel without a new capture shows here (and as a null roofline.traffic)."""
    b = bench_module()
    traffic, src = b.profile_traffic("step_uniform_512_%s.txt" % precision)
    assert src.endswith("step_uniform_512_%s.txt" % precision), src
    # the DRAM bytes of one 512^3 launch stay within a few percent of the algorithmic bytes per cell
    assert traffic == pytest.approx(512 ** 3 * bytes_per_cell, rel=0.05)


def test_launch_list_and_other_step_profiles_carry_the_current_hash():
    b = bench_module()
    for name in ("launches_bench_512_df64.txt", "step_batched_mixed_512patches.txt", "step_ppm_256_df64.txt"):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert "kernel_source_hash = %s" % b.kernel_source_hash() in text, name
