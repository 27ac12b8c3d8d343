"""Pins of the PPM oracle (oracle/ppm.py): its pipeline with PLM edges reproduces the pinned PLM
oracle; its interface values are exact for cubic profiles; its edges satisfy the monotonicity
properties of Colella & Woodward's constraints; it conserves, keeps uniform flow, and converges on
a smooth sound wave faster than PLM/MinMod."""
import math

import numpy as np
import pytest

import oracle
from oracle import ppm
import workloads


def normwise(g, o):
    return max(np.abs(g[f] - o[f]).max() / np.abs(o[f]).max() for f in range(5))


@pytest.mark.parametrize("limiter", ["minmod", "none"])
def test_edge_form_with_plm_edges_is_the_plm_step(limiter):
    shape = (12, 10, 14)
    if limiter == "none":
        U, _ = workloads.sound_wave(shape, amp=0.1, kvec=(1, 1, 1), phase=0.3)
    else:
        U = workloads.turbulent_state(shape, seed=31, mach=2.0, sedov=False)
    U = U.numpy()
    dx = 1.0 / 14
    cfg = oracle.config(limiter=limiter)
    dt = 0.6 * oracle.cfl_periodic(U, dx, cfg)
    a = ppm.step_periodic(U, dx, dt, cfg, edges=ppm.plm_edges, limiter=limiter)
    b = oracle.step_periodic(U, dx, dt, cfg)
    assert normwise(a, b) <= 1e-14


def cubic_averages(coef, n, h):
    """Cell averages over [i h, (i+1) h] of sum_k coef[k] x^k, from the antiderivative."""
    x = np.arange(n + 1) * h
    P = sum(c * x ** (k + 1) / (k + 1) for k, c in enumerate(coef))
    return (P[1:] - P[:-1]) / h


def test_interfaces_exact_for_cubics():
    n, h = 24, 1.0 / 24
    coefs = [(1.0, 0.3, 0.1, 0.05), (2.0, -0.4, 0.2, -0.1), (0.5, 0.2, -0.1, 0.03), (1.0, 1.0, 0.5, 0.2),
             (3.0, -0.5, 0.05, 0.01)]
    q = np.stack([cubic_averages(c, n, h) for c in coefs])[:, None, None, :]
    qi = ppm.interfaces(q, axis=3)[:, 0, 0, :]
    x = (np.arange(n) + 1) * h
    for f, c in enumerate(coefs):
        exact = sum(ck * x ** k for k, ck in enumerate(c))
        # interfaces whose 4-cell stencil does not wrap
        np.testing.assert_allclose(qi[f, 1:n - 2], exact[1:n - 2], rtol=0, atol=1e-14)
    # no constraint acts on these monotone, gently curved profiles: the edges are the interfaces
    qL, qR = ppm.ppm_edges(q, axis=3)
    np.testing.assert_array_equal(qR[:, 0, 0, 2:n - 3], ppm.interfaces(q, 3)[:, 0, 0, 2:n - 3])


def test_edge_properties_on_rough_data():
    rng = np.random.default_rng(32)
    q = rng.standard_normal((5, 3, 4, 200)) + np.linspace(0, 3, 200)
    qi = ppm.interfaces(q, axis=3)
    lo = np.minimum(q, np.roll(q, -1, 3))
    hi = np.maximum(q, np.roll(q, -1, 3))
    assert np.all(qi >= lo - 1e-12) and np.all(qi <= hi + 1e-12)  # between its two cells
    qL, qR = ppm.ppm_edges(q, axis=3)
    flat = (qL == q) & (qR == q)
    D = qR - qL
    Q6 = 6.0 * (q - 0.5 * (qL + qR))
    # a parabola that is not flat has no extremum inside its cell: |Q6| <= |D|
    assert np.all(flat | (np.abs(Q6) <= np.abs(D) * (1 + 1e-12) + 1e-14))
    # local extrema are flattened
    ext = (np.roll(q, -1, 3) - q) * (q - np.roll(q, 1, 3)) <= 0
    assert np.all(flat[ext])
    # each edge stays between its cell's value and the neighbour's across it: the constraints move
    # the edge on the side of the parabola's extremum towards the cell value, never past it
    qp, qm = np.roll(q, -1, 3), np.roll(q, 1, 3)
    assert np.all((qR >= np.minimum(q, qp) - 1e-12) & (qR <= np.maximum(q, qp) + 1e-12))
    assert np.all((qL >= np.minimum(q, qm) - 1e-12) & (qL <= np.maximum(q, qm) + 1e-12))
    # the parabola's mean is the cell value: qL + D/2 + Q6/6 == q
    np.testing.assert_allclose(qL + 0.5 * D + Q6 / 6.0, q, rtol=0, atol=1e-12)


def test_uniform_flow_unchanged_and_conservation():
    cfg = oracle.config()
    shape = (6, 8, 10)
    rho = np.full(shape, 1.3)
    q = np.stack([rho, np.full(shape, 0.4), np.full(shape, -0.2), np.full(shape, 0.1), np.full(shape, 0.7)])
    U = oracle.prim_to_cons(q, cfg)
    dt = oracle.cfl_periodic(U, 0.1, cfg)
    np.testing.assert_allclose(ppm.step_periodic(U, 0.1, dt, cfg), U, rtol=1e-15, atol=0)
    V = workloads.turbulent_state((12, 10, 14), seed=33, mach=5.0, sedov=True).numpy()
    dt = oracle.cfl_periodic(V, 1.0 / 14, cfg)
    W = V.copy()
    for _ in range(5):
        W = ppm.step_periodic(W, 1.0 / 14, dt, cfg)
    tot0, tot = V.sum(axis=(1, 2, 3)), W.sum(axis=(1, 2, 3))
    scale = np.abs(V).sum(axis=(1, 2, 3))
    assert np.all(np.abs(tot - tot0) / scale <= 1e-13)


def test_sound_wave_converges_faster_than_plm_minmod():
    cfg = oracle.config()
    errs, errs_plm = [], []
    ns = (16, 32, 64)
    for n in ns:
        U0, period = workloads.sound_wave((4, n, n), amp=1e-5, kvec=(1, 1, 0), phase=0.3)
        U0 = U0.numpy()
        dx = 1.0 / n
        for stepper, out in ((ppm.step_periodic, errs), (oracle.step_periodic, errs_plm)):
            U, t = U0.copy(), 0.0
            while t < period - 1e-14:
                dt = min(oracle.cfl_periodic(U, dx, cfg), period - t)
                U = stepper(U, dx, dt, cfg)
                t += dt
            out.append(np.abs(U[0] - U0[0]).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert orders[-1] >= 1.8, (errs, orders)
    assert errs[-1] < 0.5 * errs_plm[-1], (errs, errs_plm)


def test_ghosted_patch_step_is_the_periodic_step_of_its_cells():
    """A patch cut from a periodic box with exact ghosts (three layers) steps to the box's own step
    on its cells, including patches that wrap around the box."""
    shape = (14, 12, 16)
    U = workloads.turbulent_state(shape, seed=34, mach=3.0, sedov=True)
    dx = 1.0 / 16
    cfg = oracle.config()
    Un = U.numpy()
    dt = oracle.cfl_periodic(Un, dx, cfg)
    full = ppm.step_periodic(Un, dx, dt, cfg)
    for origin, dims in (((0, 0, 0), (5, 4, 3)), ((13, 10, 11), (6, 5, 7)), ((2, 3, 4), (1, 1, 1))):
        Ug = workloads.ghosted_from_periodic(U, origin, dims, ghost=3).numpy()
        got = ppm.step_patch(Ug, dx, dt, cfg)
        ix = np.arange(origin[0], origin[0] + dims[0]) % shape[2]
        iy = np.arange(origin[1], origin[1] + dims[1]) % shape[1]
        iz = np.arange(origin[2], origin[2] + dims[2]) % shape[0]
        want = full[:, iz][:, :, iy][:, :, :, ix]
        assert np.abs(got - want).max() <= 1e-15 * np.abs(full).max(), origin


def test_sod_converges_to_the_exact_solution_below_plm():
    """Sod's shock tube at gamma 1.4 (zero-gradient ends): the L1 density error against the exact
    Riemann solution falls at first order (discontinuities) and stays below PLM/MinMod's."""
    from oracle import riemann_exact
    cfg = oracle.config(gamma=1.4)
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)

    def l1(n, stepper, g):
        U = workloads.riemann_1d(n, left, right, axis=0, ntrans=4, gamma=1.4).numpy()
        dx, t = 1.0 / n, 0.0
        while t < 0.2 - 1e-15:
            Ug = np.pad(U, ((0, 0), (g, g), (g, g), (g, g)), mode="edge")
            dt = min(oracle.cfl_periodic(U, dx, cfg), 0.2 - t)
            U = stepper(Ug, dx, dt, cfg)
            t += dt
        xc = (np.arange(n) + 0.5) / n
        return np.abs(U[0, 1, 1, :] - riemann_exact.sample(left, right, 1.4, (xc - 0.5) / 0.2)[0]).mean()

    e = [l1(n, ppm.step_patch, 3) for n in (64, 128, 256)]
    plm = [l1(n, oracle.step_patch, 2) for n in (64, 128, 256)]
    assert e[0] > e[1] > e[2] and e[0] / e[2] > 2.5, e
    assert e[2] < 0.003, e
    assert all(a < b for a, b in zip(e, plm)), (e, plm)


def test_axis_permutation():
    """Swapping x and y (with the velocities) commutes with the PPM step bit for bit (the axis sums
    are pairwise commutative); swapping x and z agrees to round-off (the summation order changes)."""
    cfg = oracle.config()
    U = workloads.turbulent_state((10, 12, 14), seed=35, mach=2.0, sedov=False).numpy()
    dx = 1.0 / 14
    dt = 0.5 * oracle.cfl_periodic(U, dx, cfg)
    V = ppm.step_periodic(U, dx, dt, cfg)
    Us = np.transpose(U, (0, 1, 3, 2))[[0, 2, 1, 3, 4]]
    Vs = ppm.step_periodic(Us, dx, dt, cfg)
    np.testing.assert_array_equal(np.transpose(Vs, (0, 1, 3, 2))[[0, 2, 1, 3, 4]], V)
    Uz = np.transpose(U, (0, 3, 2, 1))[[0, 3, 2, 1, 4]]
    Vz = ppm.step_periodic(Uz, dx, dt, cfg)
    back = np.transpose(Vz, (0, 3, 2, 1))[[0, 3, 2, 1, 4]]
    assert normwise(back, V) <= 1e-14


def test_mirror_symmetry():
    """Reflecting x -> -x (cells reversed, m_x negated) commutes with the PPM step up to the
    rounding of the HLLC S* numerator: the parabola, its constraints and the face states are
    mirror-symmetric, so an edge rule that favours one side fails here."""
    cfg = oracle.config()
    U = workloads.white_velocity_state((8, 10, 12), seed=33, p_jitter=0.3).numpy()

    def mirror(V):
        W = V[..., ::-1].copy()
        W[1] = -W[1]
        return W

    dx = 1.0 / 12
    dt = 0.4 * oracle.cfl_periodic(U, dx, cfg)
    A = ppm.step_periodic(mirror(U), dx, dt, cfg)
    B = mirror(ppm.step_periodic(U, dx, dt, cfg))
    for f in range(5):
        assert np.abs(A[f] - B[f]).max() <= 1e-14 * np.abs(B[f]).max(), f
