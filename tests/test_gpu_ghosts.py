"""GPU coarse-to-fine ghost fill (hydro_fill_ghosts) against the oracle (oracle/amr.py): every
ghost cell of patches of mixed sizes whose ghosts wrap around the periodic coarse level and whose
origins lie outside [0, period); bitwise for double storage (the arithmetic is exact up to the same
roundings in the same order), float storage against the oracle on the float coarse level; the
interiors are left untouched; the fill from the coarse level interpolated in time within its step;
argument errors; the 4096-patch set on a 128^3 coarse level, sampled."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from hydro_testlib import check_clean, ctx
from oracle import amr

import paper_1412_0934_gb300 as hy

pytestmark = pytest.mark.gpu


def _patches(rng, n, period, sizes=(1, 2, 3, 5, 8)):
    dims = [tuple(int(rng.choice(sizes)) for _ in range(3)) for _ in range(n)]
    origins = [tuple(int(rng.integers(-6, p + 6)) for p in period) for _ in range(n)]
    return dims, origins


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64", "fp32"])
def test_ghost_fill_matches_oracle(precision):
    dtype = torch.float32 if precision == "fp32" else torch.float64
    c = ctx(precision)
    coarse = workloads.turbulent_state((6, 5, 7), seed=9, mach=3.0, sedov=False).to(dtype).contiguous()
    Uc = coarse.double().numpy()
    dxc = 1.0 / 7
    rng = np.random.default_rng(10)
    dims, origins = _patches(rng, 40, (14, 10, 12))
    tens = [torch.full((5, nz + 4, ny + 4, nx + 4), 7.0, dtype=dtype, device="cuda") for nx, ny, nz in dims]
    hy.hydro_fill_ghosts(c, hy.patch(coarse.cuda(), 0, dxc), [hy.patch(t, 2, dxc / 2) for t in tens], origins)
    torch.cuda.synchronize()
    for t, (nx, ny, nz), o in zip(tens, dims, origins):
        got = t.double().cpu().numpy()
        want = amr.fill_ghosts(Uc, np.full(got.shape, 7.0), o)
        if dtype == torch.float64:
            assert np.array_equal(got, want), o
        else:
            err = np.abs(got - want).max(axis=(1, 2, 3)) / np.abs(Uc).max(axis=(1, 2, 3))
            assert err.max() <= 1e-6, (o, err)
        assert (got[:, 2:-2, 2:-2, 2:-2] == 7.0).all()
    check_clean(c)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_time_interpolated_ghost_fill_matches_oracle(precision):
    """hydro_fill_ghosts_time against the oracle's fill from the coarse level at a fraction of its
    step (bitwise for double storage); theta = 1 and 0 give the plain fills of the two states."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    c = ctx(precision)
    old = workloads.turbulent_state((6, 5, 7), seed=11, mach=3.0, sedov=False).to(dtype).contiguous()
    new = workloads.turbulent_state((6, 5, 7), seed=12, mach=3.0, sedov=False).to(dtype).contiguous()
    Uo, Un = old.double().numpy(), new.double().numpy()
    dxc = 1.0 / 7
    rng = np.random.default_rng(13)
    dims, origins = _patches(rng, 25, (14, 10, 12))
    co, cn = hy.patch(old.cuda(), 0, dxc), hy.patch(new.cuda(), 0, dxc)
    for theta in (0.0, 0.375, 0.7, 1.0):
        tens = [torch.full((5, nz + 4, ny + 4, nx + 4), 7.0, dtype=dtype, device="cuda") for nx, ny, nz in dims]
        fine = [hy.patch(t, 2, dxc / 2) for t in tens]
        hy.hydro_fill_ghosts_time(c, co, cn, theta, fine, origins)
        torch.cuda.synchronize()
        for t, o in zip(tens, origins):
            got = t.double().cpu().numpy()
            want = amr.fill_ghosts_time(Uo, Un, theta, np.full(got.shape, 7.0), o)
            if dtype == torch.float64:
                assert np.array_equal(got, want), (theta, o)
            else:
                err = np.abs(got - want).max(axis=(1, 2, 3)) / np.abs(Un).max(axis=(1, 2, 3))
                assert err.max() <= 1e-6, (theta, o, err)
        if theta in (0.0, 1.0):
            plain = [torch.full_like(t, 7.0) for t in tens]
            hy.hydro_fill_ghosts(c, co if theta == 0.0 else cn, [hy.patch(t, 2, dxc / 2) for t in plain], origins)
            torch.cuda.synchronize()
            for t, p in zip(tens, plain):
                assert torch.equal(t, p)
    with pytest.raises(hy.HydroError):
        hy.hydro_fill_ghosts_time(c, co, cn, 1.5, [hy.patch(tens[0], 2, dxc / 2)], origins[:1])
    check_clean(c)


def test_ghost_fill_argument_errors():
    c = ctx("fp64")
    coarse = torch.zeros((5, 4, 4, 4), dtype=torch.float64, device="cuda")
    fine = torch.zeros((5, 6, 6, 6), dtype=torch.float64, device="cuda")
    o = (ctypes.c_int * 3)(0, 0, 0)
    good = hy.patch(fine, 2, 0.125)
    for cp, fp in ((hy.patch(coarse, 0, 0.25), hy.patch(fine, 2, 0.1)),  # dx not half the coarse dx
                   (hy.Patch(coarse, 0, 0.25), hy.patch(fine, 0, 0.125)),  # fine without ghosts
                   (hy.patch(fine, 2, 0.25), good)):  # coarse with ghosts
        rc = hy.lib().hydro_fill_ghosts(c.handle, ctypes.byref(cp.c), ctypes.byref(fp.c), o, 1)
        assert rc == hy.HYDRO_ERR_ARG


def test_ghost_fill_4096_patches_on_128cube_sampled():
    c = ctx("mixed")
    coarse = workloads.turbulent_state(128, seed=3, sedov=False, device="cuda")
    dxc = 1.0 / 128
    descs = workloads.patch_set(4096, seed=3)
    rng = np.random.default_rng(14)
    origins = [(int(rng.integers(0, 256)), int(rng.integers(0, 256)), int(rng.integers(0, 256))) for _ in descs]
    tens = [torch.full((5, d["nz"] + 4, d["ny"] + 4, d["nx"] + 4), 7.0, dtype=torch.float64, device="cuda")
            for d in descs]
    hy.hydro_fill_ghosts(c, hy.patch(coarse, 0, dxc), [hy.patch(t, 2, dxc / 2) for t in tens], origins)
    torch.cuda.synchronize()
    Uc = coarse.cpu().numpy()
    for i in list(rng.choice(len(descs), 24, replace=False)) + [0, len(descs) - 1]:
        got = tens[i].cpu().numpy()
        want = amr.fill_ghosts(Uc, np.full(got.shape, 7.0), origins[i])
        assert np.array_equal(got, want), i
    check_clean(c)


def _partition(rng, period, pieces):
    """Blocks tiling the periodic level: cut positions per axis (x, y, z) -> list of (origin, dims)."""
    cuts = []
    for P, k in zip(period, pieces):
        c = np.sort(rng.choice(np.arange(1, P), k - 1, replace=False)) if k > 1 else np.array([], dtype=int)
        edges = np.concatenate([[0], c, [P]])
        cuts.append(list(zip(edges[:-1], np.diff(edges))))
    return [((int(x0), int(y0), int(z0)), (int(nx), int(ny), int(nz)))
            for z0, nz in cuts[2] for y0, ny in cuts[1] for x0, nx in cuts[0]]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_exchange_then_fill_matches_oracle(precision):
    """Coarse fill, then the same-level exchange, on blocks tiling a periodic fine level with a
    third of them removed (their neighbours' ghosts stay prolonged), origins shifted by whole
    periods, and one axis of a single block (the block's own periodic image)."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    c = ctx(precision)
    rng = np.random.default_rng(21)
    coarse = workloads.turbulent_state((5, 4, 6), seed=12, mach=3.0, sedov=False).to(dtype).contiguous()
    Uc = coarse.double().numpy()
    period = (12, 8, 10)  # fine level (x, y, z) = 2 x coarse
    blocks = _partition(rng, period, (3, 1, 3))
    keep = [b for b in blocks if rng.random() > 0.33]
    origins = [(o[0] + int(rng.integers(-1, 2)) * period[0], o[1] + int(rng.integers(-1, 2)) * period[1],
                o[2] + int(rng.integers(-1, 2)) * period[2]) for o, _ in keep]
    fine = workloads.turbulent_state((10, 8, 12), seed=13, mach=3.0, sedov=False).to(dtype)
    tens, host = [], []
    for (o, (nx, ny, nz)), oo in zip(keep, origins):
        t = torch.zeros((5, nz + 4, ny + 4, nx + 4), dtype=dtype)
        t[:, 2:-2, 2:-2, 2:-2] = fine[:, o[2]:o[2] + nz, o[1]:o[1] + ny, o[0]:o[0] + nx]
        host.append(t.double().numpy())
        tens.append(t.cuda())
    dxc = 1.0 / 6
    pf = [hy.patch(t, 2, dxc / 2) for t in tens]
    hy.hydro_fill_ghosts(c, hy.patch(coarse.cuda(), 0, dxc), pf, origins)
    hy.hydro_exchange_ghosts(c, pf, origins, period)
    torch.cuda.synchronize()
    want = [amr.fill_ghosts(Uc, h, o) for h, o in zip(host, origins)]
    want = amr.exchange_ghosts(want, origins, period)
    for t, w in zip(tens, want):
        got = t.double().cpu().numpy()
        if dtype == torch.float64:
            assert np.array_equal(got, w)
        else:
            assert np.abs(got - w).max() <= 1e-6 * np.abs(w).max()
    check_clean(c)


def test_exchange_reassembles_a_tiled_level_bitwise():
    c = ctx("fp64")
    rng = np.random.default_rng(22)
    period = (40, 24, 32)
    level = workloads.turbulent_state((32, 24, 40), seed=14, mach=2.0, sedov=False)
    blocks = _partition(rng, period, (4, 2, 3))
    tens = []
    for o, (nx, ny, nz) in blocks:
        t = torch.full((5, nz + 4, ny + 4, nx + 4), -1.0, dtype=torch.float64)
        t[:, 2:-2, 2:-2, 2:-2] = level[:, o[2]:o[2] + nz, o[1]:o[1] + ny, o[0]:o[0] + nx]
        tens.append(t.cuda())
    hy.hydro_exchange_ghosts(c, [hy.patch(t, 2, 1.0 / 40) for t in tens], [o for o, _ in blocks], period)
    torch.cuda.synchronize()
    for t, (o, (nx, ny, nz)) in zip(tens, blocks):
        want = workloads.ghosted_from_periodic(level, o, (nx, ny, nz))
        assert torch.equal(t.cpu(), want)
