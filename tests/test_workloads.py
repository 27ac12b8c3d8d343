"""The seeded synthetic inputs have the distributions and structure their recipe states: lognormal
density of mean 1, k^-4 velocities at the requested 3D rms Mach number with P/rho uniform, the
Sedov cell's energy, the patch-set mix (4096 patches, half cubes and half 2:1 boxes, edges
{8..48}, levels 0..5, 199 M interior cells at a ghost ratio of 1.31), oct origins on even cells,
the magnetised gas's plasma beta and Mach number; the same seed gives the same input."""
import math

import numpy as np
import pytest
import torch

import workloads

G = workloads.GAMMA


def primitives(U):
    rho = U[0]
    v = U[1:4] / rho
    p = (G - 1.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho)
    return rho, v, p


def test_turbulent_state_recipe():
    n, mach, por = 64, 5.0, 1e-4
    U = workloads.turbulent_state(n, seed=2, mach=mach, p_over_rho=por, sedov=False).numpy()
    rho, v, p = primitives(U)
    # lognormal density: log rho ~ N(-sigma^2/2, sigma^2) with sigma = 1, mean 1
    lr = np.log(rho)
    assert abs(lr.std() - 1.0) < 0.01 and abs(lr.mean() + 0.5) < 0.01 and abs(rho.mean() - 1.0) < 0.02
    # cold gas at uniform P/rho, velocities at 3D rms Mach 5 of c_s = sqrt(gamma P/rho)
    np.testing.assert_allclose(p / rho, por, rtol=1e-9)
    cs = math.sqrt(G * por)
    assert math.sqrt((v ** 2).sum(axis=0).mean()) / cs == pytest.approx(mach, rel=1e-12)
    # each component has zero mean and a k^-4 power spectrum (shell-averaged mode power, k = 2..16)
    k = np.fft.fftfreq(n) * n
    K = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    kb = np.arange(2, 17)
    for c in range(3):
        assert abs(v[c].mean()) < 1e-12 * np.abs(v[c]).max()
        P = np.abs(np.fft.fftn(v[c])) ** 2
        assert P[0, 0, 0] < 1e-20 * P.sum()
        pk = [P[(K >= a - 0.5) & (K < a + 0.5)].mean() for a in kb]
        slope = np.polyfit(np.log(kb), np.log(pk), 1)[0]
        assert -4.3 < slope < -3.7, slope
    # the Sedov cell: energy E = 1 added to cell (n/2, n/2, n/2), i.e. 1/dx^3 to its energy density
    S = workloads.turbulent_state(n, seed=2, mach=mach, p_over_rho=por, sedov=True).numpy()
    diff = S - U
    assert np.count_nonzero(diff) == 1
    assert diff[4, n // 2, n // 2, n // 2] == pytest.approx(float(n) ** 3, rel=1e-12)


def test_white_velocity_state_recipe():
    U = workloads.white_velocity_state(32, seed=1, sigma_rho=0.5, p0=1.0, vel_frac=0.3).numpy()
    rho, v, p = primitives(U)
    np.testing.assert_allclose(p, 1.0, rtol=1e-12)
    cs = math.sqrt(G * 1.0)
    for c in range(3):
        m = (U[1 + c] / rho)
        assert abs(m.std() / cs - 0.3) < 0.01
    assert abs(np.log(rho).std() - 0.5) < 0.01


def test_patch_set_mix():
    ps = workloads.patch_set()
    assert len(ps) == 4096
    cubes = [p for p in ps if p["nx"] == p["ny"] == p["nz"]]
    boxes = [p for p in ps if not (p["nx"] == p["ny"] == p["nz"])]
    assert len(cubes) == len(boxes) == 2048
    for p in boxes:
        d = sorted((p["nx"], p["ny"], p["nz"]))
        assert d[0] == d[1] and d[2] == 2 * d[0]
    assert {min(p["nx"], p["ny"], p["nz"]) for p in ps} == set(workloads.PATCH_EDGES)
    assert {p["level"] for p in ps} == set(range(6))
    assert all(p["dx"] == 2.0 ** (-p["level"]) / 64 for p in ps)
    long_axes = [int(np.argmax([p["nx"], p["ny"], p["nz"]])) for p in boxes]
    assert min(np.bincount(long_axes, minlength=3)) > 600        # the long axis spread over x, y, z
    cells = sum(p["nx"] * p["ny"] * p["nz"] for p in ps)
    ghosted = sum((p["nx"] + 4) * (p["ny"] + 4) * (p["nz"] + 4) for p in ps)
    assert cells == pytest.approx(199e6, rel=0.005) and ghosted / cells == pytest.approx(1.31, abs=0.005)


def test_oct_origins_and_gathered_stencils():
    o = workloads.oct_origins(1000, (16, 12, 20), seed=3)
    assert o.shape == (1000, 3) and np.all(o % 2 == 0)
    assert np.all(o[:, 0] < 20) and np.all(o[:, 1] < 12) and np.all(o[:, 2] < 16)
    U = workloads.white_velocity_state((16, 12, 20), seed=4)
    g = workloads.gather_octs(U, o[:5])
    for i, (x, y, z) in enumerate(o[:5]):
        want = workloads.ghosted_from_periodic(U, (int(x), int(y), int(z)), (2, 2, 2))
        assert torch.equal(g[:, i], want)


def test_mhd_state_recipe():
    beta, mach = 0.5, 2.0
    U = workloads.mhd_state((24, 20, 28), seed=63, beta=beta, mach=mach, psi_amp=0.05).numpy()
    rho = U[0]
    v = U[1:4] / rho
    B = U[5:8]
    p = (G - 1.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho - 0.5 * (B ** 2).sum(axis=0))
    assert rho.min() > 0 and p.min() > 0 and abs(rho.mean() - 1.0) < 0.05
    assert 2.0 * p.mean() / (B ** 2).sum(axis=0).mean() == pytest.approx(beta, rel=0.1)
    cs = math.sqrt(G * p.mean() / rho.mean())
    assert math.sqrt((v ** 2).sum(axis=0).mean()) / cs == pytest.approx(mach, rel=0.1)
    assert math.sqrt((U[8] ** 2).mean()) == pytest.approx(0.05, rel=1e-12)   # psi of rms psi_amp


def test_same_seed_same_input():
    a = workloads.turbulent_state(16, seed=7)
    assert torch.equal(a, workloads.turbulent_state(16, seed=7))
    assert not torch.equal(a, workloads.turbulent_state(16, seed=8))
    assert workloads.patch_set(seed=3) == workloads.patch_set(seed=3)
