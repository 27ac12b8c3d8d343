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


def adjoint_sensitivity(U, dx, limiter):
    cfg = oracle.config(limiter=limiter)
    dt = 0.8 * oracle.cfl_periodic(U, dx, cfg)
    lam = np.random.default_rng(7).standard_normal(U.shape)
    a = oracle.step_periodic_adjoint(U, lam, dx, dt, cfg, block=6)
    Up = U * (1 + np.random.default_rng(0).choice([-1, 1], U.shape) * 2.2e-16)
    b = oracle.step_periodic_adjoint(Up, lam, dx, dt, cfg, block=6)
    return max(np.abs(a[f] - b[f]).max() / np.abs(a[f]).max() for f in range(5))


def test_adjoint_is_undefined_on_limiter_kinks_only():
    """With a uniform pressure every recovered pressure difference is rounding noise, so MinMod sits
    on its a*b = 0 kink and the derivative jumps by percents under a 1-ulp input change; with a
    non-uniform pressure it is defined and stable."""
    shape = (12, 10, 9)
    flat = workloads.white_velocity_state(shape, seed=1).numpy()
    assert adjoint_sensitivity(flat, 1 / 9, "minmod") > 1e-3
    jit = workloads.white_velocity_state(shape, seed=1, p_jitter=0.2).numpy()
    assert adjoint_sensitivity(jit, 1 / 9, "minmod") < 1e-13
    turb = workloads.turbulent_state(shape, seed=2, mach=5.0, sedov=True).numpy()
    assert adjoint_sensitivity(turb, 1 / 9, "minmod") < 1e-13
