"""Conditioning of the discrete step, measured on the oracle alone: the output change under a
1-ulp relative perturbation of the input.  This is what bounds any two correct implementations'
agreement (they round differently), and why the FP64 parity tests run the unlimited scheme on
smooth data only."""
import numpy as np
import pytest

import oracle
import workloads


def sensitivity(U, dx, limiter):
    cfg = oracle.config(limiter=limiter)
    dt = oracle.cfl_periodic(U, dx, cfg)
    o = oracle.step_periodic(U, dx, dt, cfg)
    Up = U * (1 + np.random.default_rng(0).choice([-1, 1], U.shape) * 2.2e-16)
    op = oracle.step_periodic(Up, dx, dt, cfg)
    return max(np.abs(op[f] - o[f]).max() / np.abs(o[f]).max() for f in range(5))


@pytest.mark.parametrize("limiter", ["minmod", "mc"])
def test_tvd_limiters_are_well_conditioned_on_white_noise(limiter):
    U = workloads.white_velocity_state((9, 13, 20), seed=1).numpy()
    assert sensitivity(U, 1 / 20, limiter) < 1e-14


def test_unlimited_scheme_is_ill_conditioned_on_rough_data_only():
    U = workloads.white_velocity_state((9, 13, 20), seed=1).numpy()
    assert sensitivity(U, 1 / 20, "none") > 1e-13
    B = workloads.turbulent_state((9, 13, 20), seed=2, mach=5.0, sedov=True).numpy()
    assert sensitivity(B, 1 / 20, "none") > 1e-13  # the point blast next to cold gas
    T = workloads.turbulent_state((9, 13, 20), seed=2, mach=5.0, sedov=False).numpy()
    assert sensitivity(T, 1 / 20, "none") < 1e-14
    W, _ = workloads.sound_wave((9, 13, 20), amp=0.1, kvec=(1, 1, 1), phase=0.3)
    assert sensitivity(W.numpy(), 1 / 20, "none") < 1e-14


@pytest.mark.parametrize("limiter", ["minmod", "mc"])
def test_tvd_limiters_are_well_conditioned_across_the_blast(limiter):
    B = workloads.turbulent_state((9, 13, 20), seed=2, mach=5.0, sedov=True).numpy()
    assert sensitivity(B, 1 / 20, limiter) < 1e-14
