"""Parity at the benchmark's full sizes, in the launch configuration bench.py times, on sampled
outputs the oracle computes one by one: each sampled cell from its own 5^3 periodic neighbourhood
(the step's stencil radius is 2), each sampled patch or oct group whole.
  - 512^3 Mach-5 turbulence + Sedov cell, MinMod (the headline workload): the CFL dt of the whole
    box (oracle over every cell), one step in double-float, FP64, FP32 and mixed at the tuning the
    autotuner picks for this box (as bench.py runs it), and in double-float at fixed tile shapes, and
    the fused dt of the result (oracle over every cell again);
  - 1024^3 Mach-10 MC FP32 (the first step of the graph-captured run): the step on samples, the dt
    at the cell the GPU's dt comes from and a lower bound at every sampled cell;
  - the 4096-patch mixed-precision set in one persistent launch, per-patch dt, and 262144 oct groups;
  - the 256^3 level stored oct-major (2,097,152 octs), its device-built Morton order and neighbour
    table, every oct stepped through the table (mixed), sampled octs against the oracle's step
    through its own table;
  - the 4096-patch set with three ghost layers under PPM (mixed), sampled patches whole."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from hydro_testlib import ctx

import paper_1412_0934_gb300 as hy

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df64": 1e-12, "fp32": 1e-5, "mixed": 1e-5}
DT_TOL = {"fp64": 1e-13, "df64": 1e-12, "fp32": 1e-6, "mixed": 1e-6}


def sample_cells(shape, count, seed):
    """Random cells plus the box's corners, cells on both sides of tile and z-chunk seams, and the 7^3
    block around the box centre: the Sedov cell of the turbulence boxes, whose blast sets the time
    step, so that elsewhere one step changes the state by little and the error there says little."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    cells = [tuple(int(rng.integers(0, m)) for m in shape) for _ in range(count)]
    for dz in range(-3, 4):
        for dy in range(-3, 4):
            for dx in range(-3, 4):
                cells.append(((nz // 2 + dz) % nz, (ny // 2 + dy) % ny, (nx // 2 + dx) % nx))
    for z in (0, 1, 31, 32, 63, 64, 127, 128, nz - 1):
        for y in (0, 15, 16, ny - 1):
            for x in (0, 15, 16, 31, 32, nx - 1):
                cells.append((z % nz, y % ny, x % nx))
    return np.array(cells)


def neighbourhoods(U, cells):
    """(S, 5, 5, 5, 5) periodic 5^3 neighbourhoods of the cells (z, y, x), gathered on U's device."""
    _, NZ, NY, NX = U.shape
    c = torch.as_tensor(cells, device=U.device, dtype=torch.long)
    r = torch.arange(-2, 3, device=U.device)
    iz = (c[:, 0, None] + r) % NZ
    iy = (c[:, 1, None] + r) % NY
    ix = (c[:, 2, None] + r) % NX
    flat = (iz[:, :, None, None] * NY + iy[:, None, :, None]) * NX + ix[:, None, None, :]
    return U.reshape(5, -1)[:, flat].permute(1, 0, 2, 3, 4).double().cpu().numpy()


def oracle_cells(nbs, dx, dt, cfg):
    return np.stack([oracle.step_patch(nb, dx, dt, cfg)[:, 0, 0, 0] for nb in nbs])


def fieldwise(got, want):
    scale = np.maximum(np.abs(want).max(axis=0), 1e-300)
    return (np.abs(got - want) / scale).max(axis=0)


@pytest.mark.parametrize("precision,tuning", [("df64", "auto"), ("df64", (0, 128)), ("df64", (3, 128)),
                                              ("df64", (4, 64)), ("fp64", "auto"), ("fp32", "auto"),
                                              ("mixed", "auto")])
def test_512_headline_step_sampled(precision, tuning):
    """The headline step at the tuning bench.py runs it with (the autotuner's choice on this machine), and
    at fixed tile shapes: 16x16, 32x16, and 16x16 with one block per SM."""
    n = 512
    dx = 1.0 / n
    cfg = oracle.config()
    c = ctx(precision)
    dtype = torch.float32 if precision == "fp32" else torch.float64
    U = workloads.turbulent_state(n, seed=2, mach=5.0, sedov=True, device="cuda").to(dtype).contiguous()
    d = torch.empty(2, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, hy.patch(U, 0, dx), d[0:1])
    out = torch.empty_like(U)
    if tuning == "auto":
        hy.hydro_autotune(c, hy.patch(U, 0, dx), hy.patch(out, 0, dx), d[0:1])
    else:
        hy.hydro_set_tuning(c, *tuning)
    Uh = U.double().cpu().numpy()
    assert d[0].item() == pytest.approx(oracle.cfl_periodic(Uh, dx, cfg), rel=DT_TOL[precision])
    del Uh
    hy.hydro_step(c, hy.patch(U, 0, dx), hy.patch(out, 0, dx), d[0:1], d[1:2])
    torch.cuda.synchronize()
    cells = sample_cells((n, n, n), 3000, seed=11)
    want = oracle_cells(neighbourhoods(U, cells), dx, d[0].item(), cfg)
    ci = torch.as_tensor(cells, device="cuda")
    got = out[:, ci[:, 0], ci[:, 1], ci[:, 2]].double().cpu().numpy().T
    err = fieldwise(got, want)
    assert err.max() <= TOL[precision], err
    Oh = out.double().cpu().numpy()
    assert d[1].item() == pytest.approx(oracle.cfl_periodic(Oh, dx, cfg), rel=DT_TOL[precision])
    rc, bits = hy.hydro_get_error(c)
    assert rc == hy.HYDRO_OK, bits


def test_1024_mach10_mc_fp32_step_sampled():
    n = 1024
    dx = 1.0 / n
    cfg = oracle.config(limiter="mc")
    c = ctx("fp32", "mc")
    hy.hydro_set_tuning(c, 0, 128)
    U = workloads.turbulent_state(n, seed=5, mach=10.0, sigma_rho=1.5, p_over_rho=1e-5, sedov=False,
                                  device="cuda").float().contiguous()
    d = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, hy.patch(U, 0, dx), d)
    dt = d.item()
    # the cell the dt comes from (largest |u|+|v|+|w|+3c, located here with torch) and samples
    W = U.double()
    rho = W[0]
    ke = (W[1] ** 2 + W[2] ** 2 + W[3] ** 2) / rho
    p = ((5.0 / 3.0 - 1.0) * (W[4] - 0.5 * ke)).clamp_min(1e-14)
    s = (W[1].abs() + W[2].abs() + W[3].abs()) / rho + 3.0 * torch.sqrt((5.0 / 3.0) * p / rho)
    top = np.array(np.unravel_index(int(torch.argmax(s).item()), (n, n, n)))
    del W, rho, ke, p, s
    cells = np.concatenate([top[None], sample_cells((n, n, n), 2000, seed=12)])
    nbs = neighbourhoods(U, cells)
    dts_o = np.array([oracle.cfl_patch(nb, dx, cfg) for nb in nbs])  # a 1-cell interior: the cell's dt
    assert dt == pytest.approx(dts_o[0], rel=DT_TOL["fp32"])
    assert (dts_o >= dt * (1 - DT_TOL["fp32"])).all()
    out = torch.empty_like(U)
    hy.hydro_step(c, hy.patch(U, 0, dx), hy.patch(out, 0, dx), d)
    torch.cuda.synchronize()
    want = oracle_cells(nbs, dx, dt, cfg)
    ci = torch.as_tensor(cells, device="cuda")
    got = out[:, ci[:, 0], ci[:, 1], ci[:, 2]].double().cpu().numpy().T
    err = fieldwise(got, want)
    assert err.max() <= TOL["fp32"], err


def test_4096_patches_and_262144_octs_mixed_sampled():
    cfg = oracle.config()
    c = ctx("mixed")
    parent = workloads.turbulent_state(256, seed=3, sedov=False, device="cuda")
    descs = workloads.patch_set(4096, seed=3)
    origins = workloads.patch_origins(descs, parent.shape[1:], seed=3)
    ins, outs, keep = [], [], []
    for dsc, o in zip(descs, origins):
        Ug = workloads.ghosted_from_periodic(parent, o, (dsc["nx"], dsc["ny"], dsc["nz"])).contiguous()
        Vg = torch.empty_like(Ug)
        keep.append((Ug, Vg))
        ins.append(hy.patch(Ug, 2, dsc["dx"], dsc["level"]))
        outs.append(hy.patch(Vg, 2, dsc["dx"], dsc["level"]))
    dt = torch.empty(len(ins), dtype=torch.float64, device="cuda")
    dn = torch.empty_like(dt)
    hy.hydro_cfl_dt(c, ins, dt)
    hy.hydro_step(c, ins, outs, dt, dn)
    torch.cuda.synchronize()
    rng = np.random.default_rng(13)
    big = sorted(range(len(descs)), key=lambda i: -descs[i]["nx"] * descs[i]["ny"] * descs[i]["nz"])[:4]
    picks = sorted(set(big) | set(int(i) for i in rng.choice(len(descs), 20, replace=False)))
    dth, dnh = dt.cpu().numpy(), dn.cpu().numpy()
    for i in picks:
        Ug, Vg = keep[i]
        Uh = Ug.cpu().numpy()
        dx = descs[i]["dx"]
        assert dth[i] == pytest.approx(oracle.cfl_patch(Uh, dx, cfg), rel=DT_TOL["mixed"])
        want = oracle.step_patch(Uh, dx, dth[i], cfg)
        got = Vg[:, 2:-2, 2:-2, 2:-2].cpu().numpy()
        err = fieldwise(got.reshape(5, -1).T, want.reshape(5, -1).T)
        assert err.max() <= TOL["mixed"], (i, err)
        # fused dt of the result: the oracle's CFL of the updated interior (ghosts: any values
        # give the same dt, the CFL reads the interior only)
        Vh = Vg.cpu().numpy()
        Vh[:, 2:-2, 2:-2, 2:-2] = got
        assert dnh[i] == pytest.approx(oracle.cfl_patch(Vh, dx, cfg), rel=DT_TOL["mixed"])
    del keep, ins, outs
    # oct groups
    G = 262144
    og = workloads.oct_origins(G, parent.shape[1:], seed=3)
    g = workloads.gather_octs(parent, og).contiguous()
    go = torch.empty((5, G, 2, 2, 2), dtype=torch.float64, device="cuda")
    dto = torch.tensor([0.5 * dth.min()], dtype=torch.float64, device="cuda")
    dxo = 1.0 / 256
    hy.hydro_step_octs(c, g, go, dxo, dto)
    torch.cuda.synchronize()
    sel = rng.choice(G, 1500, replace=False)
    gh = g[:, torch.as_tensor(sel, device="cuda")].permute(1, 0, 2, 3, 4).cpu().numpy()
    want = np.stack([oracle.step_patch(b, dxo, dto.item(), cfg) for b in gh])  # (S, 5, 2, 2, 2)
    got = go[:, torch.as_tensor(sel, device="cuda")].permute(1, 0, 2, 3, 4).cpu().numpy()
    err = fieldwise(got.transpose(0, 2, 3, 4, 1).reshape(-1, 5), want.transpose(0, 2, 3, 4, 1).reshape(-1, 5))
    assert err.max() <= TOL["mixed"], err
    rc, bits = hy.hydro_get_error(c)
    assert rc == hy.HYDRO_OK, bits


def test_256_level_octs_through_the_table_mixed_sampled():
    from oracle import octs as ooct
    cfg = oracle.config()
    c = ctx("mixed")
    parent = workloads.turbulent_state(256, seed=3, sedov=False, device="cuda")
    no = 128 ** 3
    V = parent.reshape(5, 128, 2, 128, 2, 128, 2).permute(0, 1, 3, 5, 2, 4, 6).reshape(5, no, 8).contiguous()
    idx = torch.arange(no, device="cuda", dtype=torch.int32)
    pos = torch.stack([idx % 128, (idx // 128) % 128, idx // (128 * 128)], dim=1).contiguous()
    order = torch.empty(no, dtype=torch.int32, device="cuda")
    nbr = torch.empty((no, 27), dtype=torch.int32, device="cuda")
    hy.hydro_octs_build(c, pos, (128, 128, 128), order, nbr)
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, hy.patch(parent, 0, 1.0 / 256), dt)
    out = torch.empty_like(V)
    hy.hydro_step_octs_table(c, V, out, nbr, order, 1.0 / 256, dt)
    torch.cuda.synchronize()
    rc, bits = hy.hydro_get_error(c)
    assert rc == hy.HYDRO_OK, bits
    # order: oct numbering x fastest, so the Morton order is the key order of the positions
    rng = np.random.default_rng(21)
    sel = np.concatenate([[0, no - 1, 127, 128 * 128 - 1], rng.choice(no, 300, replace=False)])
    posh = pos.cpu().numpy()
    assert np.array_equal(order.cpu().numpy(), ooct.sfc_order(posh))
    # sampled octs: the oracle gathers each 6^3 stencil through its own neighbour table entries
    nb = nbr.cpu().numpy()
    for o in sel[:8]:
        X, Y, Z = posh[o]
        want = [((X + dx) % 128) + 128 * (((Y + dy) % 128) + 128 * ((Z + dz) % 128))
                for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        assert np.array_equal(nb[o], want)
    Vh = V[:, torch.as_tensor(np.unique(nb[sel]), device="cuda").long()]
    lookup = {int(k): i for i, k in enumerate(np.unique(nb[sel]))}
    Vsub = Vh.cpu().numpy()
    d = dt.item()
    got = out[:, torch.as_tensor(sel, device="cuda").long()].cpu().numpy()  # (5, S, 8)
    want = np.empty_like(got)
    for k, o in enumerate(sel):
        table = np.array([[lookup[int(n)] for n in nb[o]]])
        G = ooct.gather_stencil(Vsub, table, 0)
        want[:, k] = oracle.step_patch(G, 1.0 / 256, d, cfg).reshape(5, 8)
    err = fieldwise(got.transpose(1, 2, 0).reshape(-1, 5), want.transpose(1, 2, 0).reshape(-1, 5))
    assert err.max() <= TOL["mixed"], err


def test_4096_patches_ppm_mixed_sampled():
    from oracle import ppm as oppm
    cfg = oracle.config()
    c = ctx("mixed", limiter="ppm")
    # the bench's patch set and state (Mach 5: the scheme floors a few cells' pressure, both sides)
    parent = workloads.turbulent_state(256, seed=3, sedov=False, device="cuda")
    descs = workloads.patch_set(4096, seed=3)
    origins = workloads.patch_origins(descs, parent.shape[1:], seed=3)
    ins, outs, keep = [], [], []
    for dsc, o in zip(descs, origins):
        Ug = workloads.ghosted_from_periodic(parent, o, (dsc["nx"], dsc["ny"], dsc["nz"]), ghost=3).contiguous()
        Vg = torch.empty_like(Ug)
        keep.append((Ug, Vg))
        ins.append(hy.patch(Ug, 3, dsc["dx"], dsc["level"]))
        outs.append(hy.patch(Vg, 3, dsc["dx"], dsc["level"]))
    dt = torch.empty(len(ins), dtype=torch.float64, device="cuda")
    dn = torch.empty_like(dt)
    hy.hydro_cfl_dt(c, ins, dt)
    hy.hydro_step(c, ins, outs, dt, dn)
    dn2 = torch.empty_like(dn)
    hy.hydro_cfl_dt(c, outs, dn2)
    torch.cuda.synchronize()
    assert torch.equal(dn, dn2)
    rng = np.random.default_rng(23)
    big = sorted(range(len(descs)), key=lambda i: -descs[i]["nx"] * descs[i]["ny"] * descs[i]["nz"])[:2]
    picks = sorted(set(big) | set(int(i) for i in rng.choice(len(descs), 10, replace=False)))
    dth = dt.cpu().numpy()
    for i in picks:
        Ug, Vg = keep[i]
        want = oppm.step_patch(Ug.cpu().numpy(), descs[i]["dx"], dth[i], cfg)
        got = Vg[:, 3:-3, 3:-3, 3:-3].cpu().numpy()
        err = fieldwise(got.reshape(5, -1).T, want.reshape(5, -1).T)
        assert err.max() <= TOL["mixed"], (i, err)
