"""GPU parity of the PPM step against the PPM oracle (oracle/ppm.py), through the C ABI: periodic
boxes element by element (several tiles, a ragged tile edge, several z chunks), batched patches with
three ghost layers, a 256^3 box on sampled windows, the fused dt, conservation, the graph-captured
run, the ghost-layer check and the calls that reject a PPM context."""
import numpy as np
import pytest
import torch

import oracle
from oracle import ppm as oppm
import workloads
from hydro_testlib import check_clean, ctx, dev, dts, normwise

import paper_1412_0934_gb300 as hy

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-5, "fp32": 1e-5}


def ppm_step(c, U, dx, dt, dt_next=False):
    a = dev(U, c.dtype)
    b = torch.empty_like(a)
    dn = torch.empty(1, dtype=torch.float64, device="cuda") if dt_next else None
    hy.hydro_step(c, hy.patch(a, 0, dx), hy.patch(b, 0, dx), dts(dt), dn)
    torch.cuda.synchronize()
    return b, (dn.item() if dt_next else None)


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "fp32"])
@pytest.mark.parametrize("case", ["turbulent", "white"])
def test_ppm_step_matches_oracle(precision, case):
    shape = (37, 18, 20)  # x: a full 16-wide tile and a ragged one; z: a 32-plane chunk and 5 more
    if case == "turbulent":
        U = workloads.turbulent_state(shape, seed=41, mach=5.0, sedov=True).numpy()
    else:
        U = workloads.white_velocity_state(shape, seed=42).numpy()
    dx = 1.0 / 20
    cfg = oracle.config()
    dt = oracle.cfl_periodic(U, dx, cfg)
    c = ctx(precision, limiter="ppm")
    b, dn = ppm_step(c, U, dx, dt, dt_next=True)
    check_clean(c)
    ref = oppm.step_periodic(U, dx, dt, cfg)
    err = normwise(b.double().cpu().numpy(), ref)
    assert err.max() <= TOL[precision], err
    # fused dt: the CFL of U^{n+1}, bit-identical to hydro_cfl_dt on the result
    d2 = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, hy.patch(b, 0, dx), d2)
    torch.cuda.synchronize()
    assert dn == d2.item()
    if precision in ("fp64", "df64"):
        dref = oracle.cfl_periodic(ref, dx, cfg)
        assert abs(dn - dref) <= 1e-12 * dref


def test_ppm_differs_from_plm_and_each_zchunk_agrees():
    """The PPM context really runs the parabolic reconstruction (its result is the PPM oracle's,
    not the PLM one), and the z chunking does not change the bits."""
    shape = (24, 16, 16)
    U = workloads.turbulent_state(shape, seed=43, mach=2.0, sedov=False).numpy()
    dx = 1.0 / 16
    cfg = oracle.config()
    dt = oracle.cfl_periodic(U, dx, cfg)
    c = ctx("fp64", limiter="ppm")
    outs = []
    for zc in (1, 3, 8, 32):
        hy.hydro_set_tuning(c, 0, zc)
        outs.append(ppm_step(c, U, dx, dt)[0])
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    g = outs[0].cpu().numpy()
    assert normwise(g, oppm.step_periodic(U, dx, dt, cfg)).max() <= 1e-12
    assert normwise(g, oracle.step_periodic(U, dx, dt, cfg)).max() > 1e-6
    check_clean(c)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ppm_graph_run_and_conservation(precision):
    shape = (32, 32, 32)
    U = workloads.turbulent_state(shape, seed=44, mach=5.0, sedov=True).numpy()
    dx = 1.0 / 32
    c = ctx(precision, limiter="ppm")
    a0 = dev(U, c.dtype)
    tot0 = a0.double().sum(dim=(1, 2, 3))
    scale = a0.double().abs().sum(dim=(1, 2, 3))
    res = []
    for graph in (True, False):
        a = a0.clone()
        b = torch.empty_like(a)
        hist = torch.empty(21, dtype=torch.float64, device="cuda")
        hy.hydro_run(c, hy.patch(a, 0, dx), hy.patch(b, 0, dx), 20, hist, use_graph=graph)
        torch.cuda.synchronize()
        res.append((a.clone(), hist.clone()))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    rel = ((res[0][0].double().sum(dim=(1, 2, 3)) - tot0).abs() / scale).max().item()
    assert rel <= (1e-12 if precision == "fp64" else 1e-6), rel
    check_clean(c)


def test_ppm_full_size_sampled_windows():
    """256^3 FP64 PPM step; each sampled 8^3 block equals the oracle's step of a 14^3 window around
    it (the stencil radius is 3, so the window's own wrap does not reach the block)."""
    n = 256
    U = workloads.turbulent_state(n, seed=45, mach=5.0, sedov=True)
    dx = 1.0 / n
    cfg = oracle.config()
    Un = U.numpy()
    dt = oracle.cfl_periodic(Un, dx, cfg)
    c = ctx("fp64", limiter="ppm")
    b, _ = ppm_step(c, Un, dx, dt)
    check_clean(c)
    g = b.cpu().numpy()
    rng = np.random.default_rng(46)
    corners = [(0, 0, 0), (n - 8, n - 8, n - 8), (n // 2 - 4, n // 2 - 4, n // 2 - 4)]  # the Sedov cell's block
    corners += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(5)]
    for (x, y, z) in corners:
        ix = np.arange(x - 3, x + 11) % n
        iy = np.arange(y - 3, y + 11) % n
        iz = np.arange(z - 3, z + 11) % n
        win = Un[:, iz][:, :, iy][:, :, :, ix]
        ref = oppm.step_periodic(win, dx, dt, cfg)[:, 3:11, 3:11, 3:11]
        got = g[:, iz[3:11]][:, :, iy[3:11]][:, :, :, ix[3:11]]
        err = np.abs(got - ref).max(axis=(1, 2, 3)) / np.abs(Un).max(axis=(1, 2, 3))
        assert err.max() <= 1e-12, ((x, y, z), err)


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "fp32"])
def test_ppm_batched_patches_match_oracle(precision):
    """Patches with three ghost layers (cubes and 2:1 boxes, ragged tiles, several z chunks, one
    patch wrapping the parent) in one persistent launch, per-patch dt; each against the oracle's
    ghosted-patch step; the fused per-patch dt equals hydro_cfl_dt bit for bit."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    # Mach 3: at Mach 5 one PPM step leaves a few cells of these patches with negative internal
    # energy (in the oracle as well), which the fused CFL's recovery flags
    parent = workloads.turbulent_state((40, 36, 44), seed=47, mach=3.0, sedov=True)
    rng = np.random.default_rng(48)
    dims = [(16, 16, 16), (20, 9, 40), (5, 33, 7), (1, 2, 3), (24, 24, 12), (8, 8, 16)]
    origins = [tuple(int(v) for v in rng.integers(0, 40, 3)) for _ in dims]
    origins[0] = (38, 34, 39)
    cfg = oracle.config()
    host, ins, outs, keep, dtl = [], [], [], [], []
    for k, (d, o) in enumerate(zip(dims, origins)):
        dx = 1.0 / (32 * (1 + k % 3))
        Ug = workloads.ghosted_from_periodic(parent, o, d, ghost=3).numpy()
        host.append((Ug, dx))
        dtl.append(0.7 * oracle.cfl_patch(Ug[:, 1:-1, 1:-1, 1:-1], dx, cfg))
        a = dev(Ug, dtype)
        b = torch.full_like(a, 7.0)
        keep += [a, b]
        ins.append(hy.patch(a, 3, dx))
        outs.append(hy.patch(b, 3, dx))
    c = ctx(precision, limiter="ppm")
    dn = torch.empty(len(dims), dtype=torch.float64, device="cuda")
    for zc in (8, 32):
        hy.hydro_set_tuning(c, 0, zc)
        hy.hydro_step(c, ins, outs, dts(*dtl), dn)
        torch.cuda.synchronize()
        check_clean(c)
        for (Ug, dx), po, dtp in zip(host, outs, dtl):
            g = torch.stack(po.tensors).double().cpu().numpy()
            ref = oppm.step_patch(Ug, dx, dtp, cfg)
            err = normwise(g[:, 3:-3, 3:-3, 3:-3], ref)
            assert err.max() <= TOL[precision], (zc, Ug.shape, err)
            assert (g[:, :3] == 7.0).all() and (g[:, -3:] == 7.0).all()  # ghosts of out untouched
    dn2 = torch.empty_like(dn)
    hy.hydro_cfl_dt(c, outs, dn2)
    torch.cuda.synchronize()
    assert torch.equal(dn, dn2)


def test_ghost_layers_must_match_the_reconstruction():
    U = workloads.white_velocity_state(8, seed=1)
    g2, g3 = (dev(workloads.ghosted_from_periodic(U, (0, 0, 0), (8, 8, 8), ghost=g).numpy()) for g in (2, 3))
    for limiter, bad in (("ppm", g2), ("minmod", g3)):
        c = ctx("fp64", limiter=limiter)
        ng = 2 if bad is g2 else 3
        with pytest.raises(hy.HydroError):
            hy.hydro_step(c, hy.patch(bad, ng, 0.1), hy.patch(torch.empty_like(bad), ng, 0.1), dts(0.01))


def test_ppm_context_rejects_the_radius_two_calls():
    c = ctx("fp64", limiter="ppm")
    U = workloads.white_velocity_state(8, seed=1).numpy()
    g = torch.zeros((5, 2, 6, 6, 6), dtype=torch.float64, device="cuda")
    o = torch.zeros((5, 2, 2, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(hy.HydroError):
        hy.hydro_step_octs(c, g, o, 0.1, dts(0.01))
    p = dev(U)
    with pytest.raises(hy.HydroError):
        hy.hydro_adjoint_step(c, hy.patch(p, 0, 0.1), dts(0.01), hy.patch(p.clone(), 0, 0.1),
                              hy.patch(torch.empty_like(p), 0, 0.1))
    check_clean(c)
