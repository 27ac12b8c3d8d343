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


def test_headline_profile_was_taken_on_the_current_step_kernel():
    """The committed ncu summary of the headline step kernel carries the hash of the kernel's sources
    it was taken on; the bench reports its DRAM traffic only while that hash matches, so a change to
    the step kernel without a new capture shows here (and as a null roofline.traffic)."""
    b = bench_module()
    traffic, src = b.profile_traffic("step_uniform_512_df64.txt")
    assert src.endswith("step_uniform_512_df64.txt"), src
    # the DRAM bytes of one 512^3 launch stay within a few percent of the algorithmic 80 B per cell
    assert traffic == pytest.approx(512 ** 3 * 80, rel=0.05)
