"""GPU parity of the MHD step (ideal MHD with GLM cleaning) against the MHD oracle (oracle/mhd.py),
through the C ABI: periodic boxes element by element for each limiter and precision, a circularly
polarised Alfven wave over a period, the fused dt, conservation, a 256^3 box on sampled windows,
batched patches with two ghost layers, and the argument checks."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mhd as omhd
import workloads
from hydro_testlib import check_clean, ctx, dts

import paper_1412_0934_gb300 as hy

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df64": 1e-12, "fp32": 1e-5, "mixed": 1e-5}


def normwise(g, o):
    return np.array([np.abs(g[f] - o[f]).max() / max(np.abs(o[f]).max(), 1e-300) for f in range(9)])


def gpu_step(c, U, dx, dt, dt_next=False):
    a = torch.as_tensor(U).to(device="cuda", dtype=c.dtype).contiguous()
    b = torch.empty_like(a)
    dn = torch.empty(1, dtype=torch.float64, device="cuda") if dt_next else None
    hy.hydro_mhd_step(c, a, b, dx, dts(dt), dn)
    torch.cuda.synchronize()
    return b, (dn.item() if dt_next else None)


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32", "mixed"])
@pytest.mark.parametrize("limiter", ["minmod", "mc", "none"])
def test_mhd_step_matches_oracle(precision, limiter):
    shape = (14, 12, 18)
    U = workloads.mhd_state(shape, seed=61, beta=0.5, mach=1.5, psi_amp=0.05).numpy()
    dx = 1.0 / 18
    cfg = oracle.config(limiter=limiter)
    dt = omhd.cfl_periodic(U, dx, cfg)
    c = ctx(precision, limiter=limiter)
    b, dn = gpu_step(c, U, dx, dt, dt_next=True)
    check_clean(c)
    ref = omhd.step_periodic(U, dx, dt, cfg, limiter=limiter)
    err = normwise(b.double().cpu().numpy(), ref)
    assert err.max() <= TOL[precision], err
    d2 = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_mhd_cfl_dt(c, b, dx, d2)
    torch.cuda.synchronize()
    assert dn == d2.item()
    if precision in ("fp64", "df64"):
        dref = omhd.cfl_periodic(ref, dx, cfg)
        assert abs(dn - dref) <= 1e-12 * dref


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_alfven_wave_period_matches_oracle(precision):
    """A circularly polarised Alfven wave over one period (32 cells per wavelength), the GPU
    chaining its own fused dt: within 1e-9 of the oracle's run and within the scheme's error of the
    exact solution (the initial state)."""
    n = 32
    x = (np.arange(n) + 0.5) / n
    ph = 2 * np.pi * x
    q = np.zeros((9, 4, 4, n))
    q[0], q[4], q[5] = 1.0, 0.1, 1.0
    q[6], q[7] = 0.1 * np.sin(ph), 0.1 * np.cos(ph)
    q[2], q[3] = -q[6], -q[7]
    cfg = oracle.config(limiter="mc")
    U0 = omhd.conserved(q, cfg)
    dx = 1.0 / n
    c = ctx(precision, limiter="mc")
    a = torch.as_tensor(U0).cuda().contiguous()
    b = torch.empty_like(a)
    dtd = torch.empty(2, dtype=torch.float64, device="cuda")
    hy.hydro_mhd_cfl_dt(c, a, dx, dtd[0:1])
    U, t = U0.copy(), 0.0
    while True:
        dt = dtd[0].item()
        if t + dt >= 1.0:
            dt = 1.0 - t
        dtd[0] = dt
        hy.hydro_mhd_step(c, a, b, dx, dtd[0:1], dtd[1:2])
        U = omhd.step_periodic(U, dx, dt, cfg, limiter="mc")
        a, b = b, a
        t += dt
        dtd[0] = dtd[1]
        if t >= 1.0 - 1e-14:
            break
    torch.cuda.synchronize()
    check_clean(c)
    g = a.cpu().numpy()
    assert np.abs(g - U).max() <= 1e-9, np.abs(g - U).max()
    assert np.abs(g[6] - U0[6]).mean() < 2e-3


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32", "mixed"])
def test_mhd_conservation(precision):
    U = workloads.mhd_state((16, 16, 16), seed=62, beta=1.0, mach=1.0).numpy()
    dx = 1.0 / 16
    c = ctx(precision)
    a = torch.as_tensor(U).to(device="cuda", dtype=c.dtype).contiguous()
    b = torch.empty_like(a)
    d = torch.empty(1, dtype=torch.float64, device="cuda")
    tot0 = a.double().sum(dim=(1, 2, 3))
    scale = a.double().abs().sum(dim=(1, 2, 3))
    steps = 100 if precision in ("fp32", "mixed") else 10
    for _ in range(steps):
        hy.hydro_mhd_cfl_dt(c, a, dx, d)
        hy.hydro_mhd_step(c, a, b, dx, d)
        a, b = b, a
    torch.cuda.synchronize()
    check_clean(c)
    rel = ((a.double().sum(dim=(1, 2, 3)) - tot0).abs() / scale)[:8].max().item()
    assert rel <= (1e-6 if precision in ("fp32", "mixed") else 1e-12), rel


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32", "mixed"])
def test_mhd_step_several_tiles_and_chunks(precision):
    """A box of several 16 x 16 column tiles and z chunks, ragged in every axis (35 x 21 x 37 cells),
    on a rough state (white noise of 5% on rho and on the internal energy): every cell against the oracle, and the fused dt
    against the standalone one."""
    shape = (37, 21, 35)
    U = workloads.mhd_state(shape, seed=68, beta=0.5, mach=2.0, psi_amp=0.05).numpy()
    rng = np.random.default_rng(69)
    kin = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
    eint = U[4] - kin - 0.5 * (U[5] ** 2 + U[6] ** 2 + U[7] ** 2)
    f = 1 + 0.05 * rng.standard_normal(U[0].shape)  # rho and m scaled alike: velocities kept
    U[0:4] *= f
    U[4] += (f - 1) * kin + 0.05 * rng.standard_normal(U[0].shape) * eint
    dx = 1.0 / 35
    cfg = oracle.config()
    dt = omhd.cfl_periodic(U, dx, cfg)
    c = ctx(precision)
    b, dn = gpu_step(c, U, dx, dt, dt_next=True)
    check_clean(c)
    ref = omhd.step_periodic(U, dx, dt, cfg)
    err = normwise(b.double().cpu().numpy(), ref)
    assert err.max() <= TOL[precision], err
    d2 = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_mhd_cfl_dt(c, b, dx, d2)
    torch.cuda.synchronize()
    assert dn == d2.item()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mhd_full_size_sampled_windows(precision):
    """256^3 MHD step (the bench's magnetised-gas box); each sampled 8^3 block equals the oracle's
    step of the 12^3 window around it (stencil radius 2): per field, the largest difference over the
    blocks within 1e-12 (FP64) or 1e-5 (FP32) of the oracle's largest value there (the normwise
    metric; psi grows tenfold in this first step, the field B not being divergence-free)."""
    n = 256
    U = workloads.mhd_state(n, seed=63, beta=0.5, mach=2.0).numpy()
    dx = 1.0 / n
    cfg = oracle.config()
    dt = omhd.cfl_periodic(U, dx, cfg)
    c = ctx(precision)
    b, dn = gpu_step(c, U, dx, dt, dt_next=True)
    check_clean(c)
    g = b.double().cpu().numpy()
    rng = np.random.default_rng(64)
    corners = [(0, 0, 0), (n - 8, n - 8, n - 8)] + [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(6)]
    diff, scale = np.zeros(9), np.zeros(9)
    for (x, y, z) in corners:
        ix = np.arange(x - 2, x + 10) % n
        iy = np.arange(y - 2, y + 10) % n
        iz = np.arange(z - 2, z + 10) % n
        win = U[:, iz][:, :, iy][:, :, :, ix]
        ref = omhd.step_periodic(win, dx, dt, cfg)[:, 2:10, 2:10, 2:10]
        got = g[:, iz[2:10]][:, :, iy[2:10]][:, :, :, ix[2:10]]
        diff = np.maximum(diff, np.abs(got - ref).max(axis=(1, 2, 3)))
        scale = np.maximum(scale, np.abs(ref).max(axis=(1, 2, 3)))
    err = diff / scale
    assert err.max() <= TOL[precision], err


def _ghosted(U, origin, dims, g):
    o = np.asarray(origin)
    _, NZ, NY, NX = U.shape
    ix = np.arange(o[0] - g, o[0] + dims[0] + g) % NX
    iy = np.arange(o[1] - g, o[1] + dims[1] + g) % NY
    iz = np.arange(o[2] - g, o[2] + dims[2] + g) % NZ
    return U[:, iz][:, :, iy][:, :, :, ix]


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32", "mixed"])
def test_mhd_patches_match_oracle(precision):
    """Patches with two ghost layers (sizes 1 to 40, a 2:1 box, one patch wrapping the parent, one
    wider than a 32-column tile, dx and dt per patch) in one batched call: each against the
    oracle's ghosted-patch step; outputs with and without ghost layers; the fused per-patch dt
    equals hydro_mhd_cfl_patches bit for bit."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    parent = workloads.mhd_state((30, 26, 34), seed=66, beta=0.5, mach=1.5, psi_amp=0.05).numpy()
    rng = np.random.default_rng(67)
    dims = [(16, 16, 16), (20, 9, 40), (5, 13, 7), (1, 2, 3), (12, 12, 24), (8, 8, 8), (40, 11, 6)]
    origins = [tuple(int(v) for v in rng.integers(0, 26, 3)) for _ in dims]
    origins[0] = (30, 22, 27)
    cfg = oracle.config()
    c = ctx(precision)
    host, ins, outs, dtl = [], [], [], []
    for k, (d, o) in enumerate(zip(dims, origins)):
        dx = 1.0 / (16 * (1 + k % 3))
        Ug = _ghosted(parent, o, d, 2)
        host.append((Ug, dx))
        dtl.append(0.8 * omhd.cfl_patch(Ug, dx, cfg))
        a = torch.as_tensor(Ug).to(device="cuda", dtype=dtype).contiguous()
        ng_out = 2 if k % 2 else 0
        b = torch.full((9, d[2] + 2 * ng_out, d[1] + 2 * ng_out, d[0] + 2 * ng_out), 7.0, dtype=dtype, device="cuda")
        ins.append(hy.MhdPatch(a, 2, dx))
        outs.append(hy.MhdPatch(b, ng_out, dx))
    dn = torch.empty(len(dims), dtype=torch.float64, device="cuda")
    hy.hydro_mhd_step_patches(c, ins, outs, dts(*dtl), dn)
    torch.cuda.synchronize()
    check_clean(c)
    for (Ug, dx), po, dtp in zip(host, outs, dtl):
        g = torch.stack(po.tensors).double().cpu().numpy()
        ng = po.c.ng
        gi = g[:, ng:g.shape[1] - ng, ng:g.shape[2] - ng, ng:g.shape[3] - ng]
        ref = omhd.step_patch(Ug, dx, dtp, cfg)
        err = normwise(gi, ref)
        assert err.max() <= TOL[precision], (Ug.shape, err)
        if ng:
            assert (g[:, :2] == 7.0).all() and (g[:, -2:] == 7.0).all()
    # the CFL of the results, through patches that carry two ghost layers
    res = []
    for po, (Ug, dx) in zip(outs, host):
        t = torch.stack(po.tensors)
        ng = po.c.ng
        full = torch.zeros((9,) + tuple(s + 4 - 2 * ng for s in t.shape[1:]), dtype=dtype, device="cuda")
        full[:, 2:-2, 2:-2, 2:-2] = t[:, ng:t.shape[1] - ng, ng:t.shape[2] - ng, ng:t.shape[3] - ng]
        res.append(hy.MhdPatch(full.contiguous(), 2, dx))
    d2 = torch.empty_like(dn)
    hy.hydro_mhd_cfl_patches(c, res, d2)
    torch.cuda.synchronize()
    assert torch.equal(dn, d2)
    if precision in ("fp64", "df64"):
        for k, (po, (Ug, dx)) in enumerate(zip(res, host)):
            want = omhd.cfl_patch(torch.stack(po.tensors).cpu().numpy(), dx, cfg)
            assert abs(dn[k].item() - want) <= 1e-12 * want


def test_mhd_argument_checks_and_bad_dt():
    U = torch.as_tensor(workloads.mhd_state((8, 8, 8), seed=65).numpy()).cuda().contiguous()
    for precision, limiter in (("fp64", "ppm"),):
        c = ctx(precision, limiter=limiter)
        with pytest.raises(hy.HydroError):
            hy.hydro_mhd_step(c, U, torch.empty_like(U), 0.1, dts(0.01))
    c = ctx("fp64")
    with pytest.raises(hy.HydroError):  # in and out overlap
        hy.hydro_mhd_step(c, U, U, 0.1, dts(0.01))
    out = torch.full_like(U, 7.0)
    hy.hydro_mhd_step(c, U, out, 0.1, dts(-1.0))
    torch.cuda.synchronize()
    rc, bits = hy.hydro_get_error(c)
    assert bits & hy.EBIT_BAD_DT
    assert (out == 7.0).all()
