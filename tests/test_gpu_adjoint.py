"""GPU adjoint parity: hydro_adjoint_step against the oracle's reverse-mode tape, element by
element; adjoint vs central differences of the GPU forward (dot-product form); the checkpointed
autograd gradient of the 64^3 / 40-step loss against central differences and, on a small case,
against the oracle's chained adjoint."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from hydro_testlib import check_clean, ctx, dev, dts, normwise

import paper_1412_0934_gb300 as hy
from paper_1412_0934_gb300 import autograd as hag

pytestmark = pytest.mark.gpu


def gpu_adjoint(c, U, lam, dx, dt):
    a = dev(U, c.dtype)
    l = dev(lam, c.dtype)
    o = torch.empty_like(a)
    hy.hydro_adjoint_step(c, hy.patch(a, 0, dx), dts(dt), hy.patch(l, 0, dx), hy.patch(o, 0, dx))
    torch.cuda.synchronize()
    return o.double().cpu().numpy()


def inputs(limiter, shape):
    """Inputs whose derivative is defined: no limiter argument pair on its kink up to rounding.
    (A uniform pressure makes every recovered pressure difference rounding noise, which puts MinMod
    exactly on its a*b = 0 kink; there the oracle's own adjoint jumps by percents under a 1-ulp
    input change -- test_oracle_conditioning.py.)  Unlimited slopes: smooth data only."""
    if limiter == "none":
        w, _ = workloads.sound_wave(shape, amp=0.1, kvec=(1, 1, 1), phase=0.3)
        w2, _ = workloads.sound_wave(shape, amp=0.05, kvec=(2, 1, 0), phase=1.1)
        return [w.numpy(), w2.numpy()]
    return [workloads.turbulent_state(shape, seed=2, mach=5.0, sedov=True).numpy(),
            workloads.white_velocity_state(shape, seed=1, p_jitter=0.2).numpy()]


# FP64 adjoints: native double, and the same reverse sweep in double-float arithmetic.
F64 = ["fp64", "df64"]


@pytest.mark.parametrize("precision", F64)
@pytest.mark.parametrize("limiter", ["minmod", "mc", "none"])
@pytest.mark.parametrize("shape", [(12, 10, 9), (18, 20, 17)])
def test_fp64_adjoint_matches_oracle_tape(limiter, shape, precision):
    c = ctx(precision, limiter)
    dx = 1.0 / shape[2]
    cfg = oracle.config(limiter=limiter)
    for U in inputs(limiter, shape):
        dt = 0.8 * oracle.cfl_periodic(U, dx, cfg)
        lam = np.random.default_rng(7).standard_normal(U.shape)
        o = oracle.step_periodic_adjoint(U, lam, dx, dt, cfg, block=6)
        g = gpu_adjoint(c, U, lam, dx, dt)
        assert normwise(g, o).max() <= 1e-12, normwise(g, o)
    check_clean(c)


@pytest.mark.parametrize("limiter", ["minmod", "mc"])
def test_fp32_adjoint_matches_oracle_tape(limiter):
    shape = (16, 16, 16)
    c = ctx("fp32", limiter)
    dx = 1.0 / 16
    cfg = oracle.config(limiter=limiter)
    U = workloads.turbulent_state(shape, seed=2, mach=2.0, sedov=False).numpy()
    U32 = U.astype(np.float32).astype(np.float64)
    dt = 0.8 * oracle.cfl_periodic(U32, dx, cfg)
    lam = np.random.default_rng(8).standard_normal(U.shape)
    o = oracle.step_periodic_adjoint(U32, lam, dx, dt, cfg, block=8)
    g = gpu_adjoint(c, U32, lam, dx, dt)
    assert normwise(g, o).max() <= 1e-4, normwise(g, o)
    check_clean(c)


@pytest.mark.parametrize("precision", F64)
@pytest.mark.parametrize("limiter", ["none", "minmod"])
def test_adjoint_dot_product_against_gpu_central_differences(limiter, precision):
    """<w, (S(U+eps v) - S(U-eps v)) / 2 eps> = <J^T w, v> on a smooth field, all on the GPU."""
    shape = (16, 16, 16)
    c = ctx(precision, limiter)
    dx = 1.0 / 16
    U, _ = workloads.sound_wave(shape, amp=1e-3, kvec=(1, 1, 1), phase=0.3)
    U = U.numpy()
    dt = 0.8 * oracle.cfl_periodic(U, dx, oracle.config(limiter=limiter))
    rng = np.random.default_rng(9)
    for _ in range(4):
        v = rng.standard_normal(U.shape) * np.abs(U).max(axis=(1, 2, 3), keepdims=True)
        w = rng.standard_normal(U.shape)
        eps = 1e-6
        outs = []
        for s in (+1, -1):
            a = dev(U + s * eps * v)
            b = torch.empty_like(a)
            hy.hydro_step(c, hy.patch(a, 0, dx), hy.patch(b, 0, dx), dts(dt))
            outs.append(b.cpu().numpy())
        Jv = (outs[0] - outs[1]) / (2 * eps)
        JTw = gpu_adjoint(c, U, w, dx, dt)
        lhs, rhs = np.vdot(w, Jv), np.vdot(JTw, v)
        assert abs(lhs - rhs) <= 1e-7 * np.abs(w * Jv).sum(), (lhs, rhs)
    check_clean(c)


def _loss_setup(n, amp=1e-3):
    W, _ = workloads.sound_wave((n, n, n), amp=amp, kvec=(1, 1, 1), phase=0.3)
    q = oracle.recover(W.numpy())
    T, _ = workloads.sound_wave((n, n, n), amp=2 * amp, kvec=(1, 0, 1), phase=1.1)
    target = oracle.recover(T.numpy())[0]
    return q, target


@pytest.mark.parametrize("precision,limiter,eps,tol", [("fp64", "none", 1e-6, 1e-6), ("fp64", "minmod", 1e-8, 1e-5),
                                                       ("fp64", "minmod", 1e-6, 1e-4), ("df64", "minmod", 1e-8, 1e-5)])
def test_checkpointed_gradient_64cube_40steps_vs_central_differences(precision, limiter, eps, tol):
    """Loss sum (rho_40 - rho_target)^2 on the 64^3 periodic grid, 40 steps, checkpoint every 8;
    gradient w.r.t. rho0 and v0 against central differences over 64 random directions,
    replaying the recorded dt sequence.  The unlimited scheme is smooth: eps = 1e-6.  MinMod has
    kinks (a*b = 0 near every extremum of the wave): central differences measure a derivative only
    along directions where the loss is smooth at the scale eps, which a second difference at eps/2
    detects; directions that cross a kink are counted (they must be a minority) and the rest must
    agree: within 1e-5 at eps = 1e-8, and within 1e-4 at the configuration's eps = 1e-6 (kinks
    crossed inside a direction's smooth-looking stretch add O(eps) to the difference)."""
    n, nsteps = 64, 40
    c = ctx(precision, limiter)
    q, target = _loss_setup(n)
    rho0 = torch.tensor(q[0], device="cuda", requires_grad=True)
    vel0 = torch.tensor(q[1:4], device="cuda", requires_grad=True)
    p0 = torch.tensor(q[4], device="cuda")
    tgt = torch.tensor(target, device="cuda")
    sim = hag.Simulation(c, (n, n, n), 1.0 / n, nsteps, checkpoint_every=8)
    loss = ((sim(rho0, vel0, p0) - tgt) ** 2).sum()
    loss.backward()
    dts_rec = sim.last_dts.clone()
    g_rho, g_vel = rho0.grad.detach().clone(), vel0.grad.detach().clone()
    gen = torch.Generator(device="cuda").manual_seed(4)

    def fd(dr, dv, e):
        with torch.no_grad():
            lp = ((sim.forward_only(rho0 + e * dr, vel0 + e * dv, p0, dts=dts_rec) - tgt) ** 2).sum()
            lm = ((sim.forward_only(rho0 - e * dr, vel0 - e * dv, p0, dts=dts_rec) - tgt) ** 2).sum()
        return ((lp - lm) / (2 * e)).item()

    errs, kinked = [], 0
    for _ in range(64):
        dr = torch.randn(rho0.shape, generator=gen, device="cuda", dtype=torch.float64)
        dv = torch.randn(vel0.shape, generator=gen, device="cuda", dtype=torch.float64) * 1e-3
        an = ((g_rho * dr).sum() + (g_vel * dv).sum()).item()
        f1 = fd(dr, dv, eps)
        if limiter != "none":
            f2 = fd(dr, dv, 0.5 * eps)
            if abs(f1 - f2) > 0.5 * tol * abs(f1):
                kinked += 1
                continue
        errs.append(abs(f1 - an) / max(abs(an), 1e-30))
    assert kinked <= (0 if limiter == "none" else 16), kinked
    assert max(errs) <= tol, (max(errs), kinked)
    check_clean(c)


@pytest.mark.parametrize("precision", F64)
def test_checkpointed_gradient_matches_oracle_chain(precision):
    """Small case (12^3, 5 steps, checkpoint every 2): the autograd gradient equals the oracle's
    forward run + chained one-step adjoints + prim->cons adjoint."""
    n, nsteps = 12, 5
    c = ctx(precision, "minmod")
    q, target = _loss_setup(n, amp=0.05)
    dx = 1.0 / n
    rho0 = torch.tensor(q[0], device="cuda", requires_grad=True)
    vel0 = torch.tensor(q[1:4], device="cuda", requires_grad=True)
    p0 = torch.tensor(q[4], device="cuda", requires_grad=True)
    tgt = torch.tensor(target, device="cuda")
    sim = hag.Simulation(c, (n, n, n), dx, nsteps, checkpoint_every=2)
    loss = ((sim(rho0, vel0, p0) - tgt) ** 2).sum()
    loss.backward()
    # oracle chain
    cfg = oracle.config()
    U = oracle.prim_to_cons(q, cfg)
    states, dtl = [], []
    for _ in range(nsteps):
        dt = oracle.cfl_periodic(U, dx, cfg)
        states.append(U)
        dtl.append(dt)
        U = oracle.step_periodic(U, dx, dt, cfg)
    np.testing.assert_allclose(sim.last_dts.cpu().numpy()[:nsteps], dtl, rtol=1e-12)
    lam = np.zeros_like(U)
    lam[0] = 2 * (U[0] - target)
    for k in range(nsteps - 1, -1, -1):
        lam = oracle.step_periodic_adjoint(states[k], lam, dx, dtl[k], cfg, block=6)
    gq = oracle.prim_to_cons_adjoint(q, lam, cfg)
    got = np.concatenate([rho0.grad.cpu().numpy()[None], vel0.grad.cpu().numpy(), p0.grad.cpu().numpy()[None]])
    assert normwise(got, gq).max() <= 1e-10, normwise(got, gq)
    check_clean(c)


@pytest.mark.parametrize("limiter", ["none", "minmod"])
def test_fp32_checkpointed_gradient_64cube_40steps_vs_fp64(limiter):
    """The 64^3 / 40-step checkpointed gradient in FP32 against the same gradient in FP64 (central
    differences in FP32 at eps = 1e-6 would measure rounding, not a derivative).  Sound wave of
    amplitude 0.05 against a target wave of twice that amplitude, so the loss residual is O(0.1) and
    FP32 rounding moves it by ~1e-6 relative.  Unlimited slopes: every component of the gradient
    within 1e-4 (normwise) of the FP64 one.  MinMod: the two trajectories, 1e-7 apart, may take
    different sides of a limiter kink in a few cells, where the derivative itself jumps; the
    gradient agrees within 1e-4 in the 2-norm, and in the max norm up to the cells at such kinks."""
    n, nsteps = 64, 40
    q, target = _loss_setup(n, amp=0.05)
    grads = {}
    for precision in ("fp64", "fp32"):
        c = ctx(precision, limiter)
        rho0 = torch.tensor(q[0], device="cuda", requires_grad=True)
        vel0 = torch.tensor(q[1:4], device="cuda", requires_grad=True)
        p0 = torch.tensor(q[4], device="cuda")
        tgt = torch.tensor(target, device="cuda")
        sim = hag.Simulation(c, (n, n, n), 1.0 / n, nsteps, checkpoint_every=8)
        loss = ((sim(rho0, vel0, p0).double() - tgt) ** 2).sum()
        loss.backward()
        grads[precision] = [rho0.grad.double().cpu().numpy(), vel0.grad.double().cpu().numpy()]
        check_clean(c)
    for g32, g64 in zip(grads["fp32"], grads["fp64"]):
        l2 = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
        mx = np.abs(g32 - g64).max() / np.abs(g64).max()
        if limiter == "none":
            assert mx <= 1e-4, (mx, l2)
        else:
            assert l2 <= 1e-4, (mx, l2)
