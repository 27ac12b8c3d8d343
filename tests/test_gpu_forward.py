"""GPU parity of the forward step (uniform periodic grid, ghosted patches, batched patches, oct
groups, CFL dt) against the FP64 oracle, element by element on seeded inputs, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from hydro_testlib import cfl, check_clean, ctx, dev, dts, normwise, step_periodic

import paper_1412_0934_gb300 as hy

pytestmark = pytest.mark.gpu

TOL64 = 1e-12  # FP64: relative (normwise per field) per step
TOL32 = 1e-5  # FP32 / MIXED after one step


def ocfg(limiter="minmod"):
    return oracle.config(limiter=limiter)


def _inputs(limiter, shape):
    """TVD limiters: k^-4 turbulence with a Sedov cell, and white-noise velocities.  Unlimited
    slopes: smooth data only (k^-4 turbulence without the blast, a 3D sound wave).  Unlimited
    slopes across the blast or on white noise are ill-conditioned -- the oracle itself moves by
    ~1e-12 under a 1-ulp input perturbation there (test_oracle_conditioning.py)."""
    if limiter == "none":
        wave, _ = workloads.sound_wave(shape, amp=0.1, kvec=(1, 1, 1), phase=0.3)
        return [workloads.turbulent_state(shape, seed=2, mach=5.0, sedov=False).numpy(), wave.numpy()]
    return [workloads.turbulent_state(shape, seed=2, mach=5.0, sedov=True).numpy(),
            workloads.white_velocity_state(shape, seed=1).numpy()]


F64 = ["fp64", "df64"]  # native double, and double-float arithmetic on a double state


@pytest.mark.parametrize("precision", F64)
@pytest.mark.parametrize("limiter", ["minmod", "mc", "none"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (9, 13, 20), (5, 3, 37)])
def test_fp64_one_step_matches_oracle(precision, limiter, shape):
    dx = 1.0 / shape[2]
    c = ctx(precision, limiter)
    for U in _inputs(limiter, shape):
        dt = oracle.cfl_periodic(U, dx, ocfg(limiter))
        o = oracle.step_periodic(U, dx, dt, ocfg(limiter))
        for tile in range(hy.NUM_TILES):
            hy.hydro_set_tuning(c, tile, 8)
            g, _ = step_periodic(c, U, dx, dt)
            assert normwise(g, o).max() <= TOL64, (tile, normwise(g, o))
    check_clean(c)


ALL = ["fp64", "df64", "mixed", "fp32"]


@pytest.mark.parametrize("precision", ALL)
@pytest.mark.parametrize("shape", [(12, 40, 70), (37, 21, 19)])
def test_every_tile_shape_matches_oracle(precision, shape):
    """Every compiled tile shape (16x16, 32x8, 8x8, 32x16, and 16x16 with one block per SM) in every
    policy, on boxes that span several tiles with ragged tails in x and y and z chunks with a ragged
    last chunk, against the oracle (FP32 from the state rounded to float); the fused dt of the result
    is the same bits for every tile shape (a maximum, whatever the order of its atomic folds)."""
    dx = 1.0 / shape[2]
    U = workloads.turbulent_state(shape, seed=2, mach=5.0, sedov=True).numpy()
    dt = oracle.cfl_periodic(U, dx, ocfg())
    Uin = U.astype(np.float32).astype(np.float64) if precision == "fp32" else U
    o = oracle.step_periodic(U, dx, dt, ocfg())
    tol = TOL64 if precision in F64 else TOL32
    c = ctx(precision)
    dnext = set()
    for tile in range(hy.NUM_TILES):
        for zc in (8, 5):
            hy.hydro_set_tuning(c, tile, zc)
            g, dn = step_periodic(c, Uin, dx, dt, dt_next=True)
            assert normwise(g, o).max() <= tol, (tile, zc, normwise(g, o))
            dnext.add(dn)
    assert len(dnext) == 1, dnext
    with pytest.raises(hy.HydroError):
        hy.hydro_set_tuning(c, hy.NUM_TILES, 8)
    check_clean(c)


@pytest.mark.parametrize("precision", ALL)
def test_autotuned_step_matches_oracle(precision, tmp_path):
    """hydro_autotune on a box and on a patch set, then the step at the tuning it chose, against the
    oracle; a cache file written by the first call gives the same tuning to a second context."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    tol = TOL64 if precision in F64 else TOL32
    shape = (24, 48, 72)
    dx = 1.0 / shape[2]
    U = workloads.turbulent_state(shape, seed=2, mach=5.0, sedov=True).numpy()
    Uin = U.astype(np.float32).astype(np.float64) if precision == "fp32" else U
    dt = oracle.cfl_periodic(U, dx, ocfg())
    o = oracle.step_periodic(U, dx, dt, ocfg())
    c = ctx(precision)
    a = dev(Uin, dtype)
    b = torch.empty_like(a)
    cache = str(tmp_path / "tuning.txt")
    hy.hydro_autotune(c, hy.patch(a, 0, dx), hy.patch(b, 0, dx), dts(dt), cache_path=cache)
    tuned = hy.hydro_get_tuning(c)
    assert 0 <= tuned[0] < hy.NUM_TILES and tuned[1] >= 1
    g, _ = step_periodic(c, Uin, dx, dt)
    assert normwise(g, o).max() <= tol, (tuned, normwise(g, o))
    c2 = ctx(precision)
    hy.hydro_set_tuning(c2, (tuned[0] + 1) % hy.NUM_TILES, 3)
    hy.hydro_autotune(c2, hy.patch(a, 0, dx), hy.patch(b, 0, dx), dts(dt), cache_path=cache)
    assert hy.hydro_get_tuning(c2) == tuned
    # a patch set
    host, ins, outs = _patch_batch(16, 9, precision, dtype, edges=(8, 16, 24, 40))
    dt_list = [0.7 * oracle.cfl_patch(Ug, d["dx"], ocfg()) for Ug, d in host]
    hy.hydro_autotune(c, ins, outs, dts(*dt_list))
    for po in outs:
        for t in po.tensors:
            t.zero_()
    hy.hydro_step(c, ins, outs, dts(*dt_list))
    torch.cuda.synchronize()
    for (Ug, d), po, dtp in zip(host, outs, dt_list):
        out = torch.stack(po.tensors).double().cpu().numpy()[:, 2:-2, 2:-2, 2:-2]
        Ur = Ug.astype(np.float32).astype(np.float64) if precision == "fp32" else Ug
        assert normwise(out, oracle.step_patch(Ur, d["dx"], dtp, ocfg())).max() <= tol, hy.hydro_get_tuning(c)
    check_clean(c)


@pytest.mark.parametrize("precision", F64)
def test_fp64_cfl_matches_oracle_and_fused_is_bitwise(precision):
    U = workloads.white_velocity_state((20, 24, 28), seed=3).numpy()
    dx = 1.0 / 28
    c = ctx(precision)
    d_gpu = cfl(c, U, dx)
    assert d_gpu == pytest.approx(oracle.cfl_periodic(U, dx, ocfg()), rel=1e-14 if precision == "fp64" else 1e-12)
    # the fused epilogue of a step on U0 gives the dt of U1; the standalone kernel on U1 the same bits
    U1, dnext = step_periodic(c, U, dx, 0.5 * d_gpu, dt_next=True)
    assert dnext == cfl(c, U1, dx)
    check_clean(c)


def _cfl_cases(shape, seed=4):
    """States for the fused CFL maximum: near ties (a uniform flow whose speeds differ by ~1e-9),
    cold fast gas (internal energy ~1e-9 of the kinetic: no float speed estimate is sure), a fast
    jet (Mach ~80, internal energy ~3e-4 of the kinetic: unsure) holding the maximum inside warm gas
    at the same pressure, and flow along x alone (zero y and z momenta in and out)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    one = np.ones(shape)
    cases = {}
    cases["near_ties"] = (one, 0.5 + 1e-9 * rng.standard_normal(shape), 0.1 * one, -0.2 * one, one)
    rho = np.exp(0.3 * rng.standard_normal(shape))
    cases["cold_fast"] = (rho, 1.0 + 1e-7 * rng.standard_normal(shape), 0.3 + 1e-7 * rng.standard_normal(shape),
                          -0.2 * one, 1e-9 * one)
    u = 0.1 * rng.standard_normal(shape)
    jet = (slice(nz // 3, nz // 3 + 2), slice(ny // 2, ny // 2 + 3), slice(None))
    u[jet] = 100.0 + 1e-3 * rng.standard_normal(u[jet].shape)
    cases["fast_jet"] = (one, u, 0.05 * rng.standard_normal(shape), 0.05 * rng.standard_normal(shape), one)
    rx = np.exp(0.5 * rng.standard_normal(nx)) * one
    ux = 0.5 * rng.standard_normal(nx) * one
    cases["x_only"] = (rx, ux, 0 * one, 0 * one, one)
    out = {}
    for k, (r, vx, vy, vz, pr) in cases.items():
        E = pr / (GAMMA_ - 1.0) + 0.5 * r * (vx * vx + vy * vy + vz * vz)
        out[k] = np.stack([r, r * vx, r * vy, r * vz, E])
    return out


GAMMA_ = 5.0 / 3.0


@pytest.mark.parametrize("precision", F64)
def test_fused_cfl_max_on_near_ties_and_unsure_estimates(precision):
    """The fused CFL of the FP64 step takes the exact speed only of cells whose float estimate is
    unsure or near the warp's running maximum (double-float takes every cell's); on states built to
    stress that choice (thousands of near ties, estimates unsure everywhere, an unsure cell holding
    the maximum, zero momenta) the fused dt is, for every tile shape, the same bits as the
    standalone CFL of the result and within 1e-13 of the oracle's CFL of it."""
    shape = (10, 36, 40)
    dx = 1.0 / shape[2]
    c = ctx(precision)
    for name, U in _cfl_cases(shape).items():
        dt = 0.5 * oracle.cfl_periodic(U, dx, ocfg())
        seen = set()
        for tile in range(hy.NUM_TILES):
            hy.hydro_set_tuning(c, tile, 4)
            U1, dn = step_periodic(c, U, dx, dt, dt_next=True)
            assert dn == cfl(c, U1, dx), (name, tile)
            assert dn == pytest.approx(oracle.cfl_periodic(U1, dx, ocfg()), rel=1e-13), (name, tile)
            seen.add(dn)
        assert len(seen) == 1, (name, seen)
        check_clean(c)


@pytest.mark.parametrize("precision", F64)
def test_fp64_ten_steps_config1(precision):
    """32^3, lognormal density (sigma 0.5), white velocities (0.3 c_s), P = 1, MinMod, CFL 0.8:
    ten steps with each side taking its own CFL dt."""
    U0 = workloads.white_velocity_state(32, seed=1).numpy()
    dx = 1.0 / 32
    c = ctx(precision)
    a = dev(U0)
    b = torch.empty_like(a)
    hist = torch.empty(11, dtype=torch.float64, device="cuda")
    hy.hydro_run(c, hy.patch(a, 0, dx), hy.patch(b, 0, dx), 10, hist, use_graph=False)
    torch.cuda.synchronize()
    g = a.cpu().numpy()  # 10 steps: result back in a
    o, odts = oracle.run_periodic(U0, dx, 10, ocfg())
    np.testing.assert_allclose(hist.cpu().numpy()[:10], odts, rtol=1e-12)
    assert normwise(g, o).max() <= 10 * TOL64
    check_clean(c)


def test_graph_run_matches_eager_run_bitwise():
    U0 = workloads.turbulent_state(24, seed=2, mach=5.0, sedov=True).numpy()
    dx = 1.0 / 24
    res = []
    for graph in (False, True, True):
        c = ctx("fp64")
        a = dev(U0)
        b = torch.empty_like(a)
        hist = torch.empty(8, dtype=torch.float64, device="cuda")
        hy.hydro_run(c, hy.patch(a, 0, dx), hy.patch(b, 0, dx), 7, hist, use_graph=graph)
        torch.cuda.synchronize()
        res.append((b.cpu().numpy(), hist.cpu().numpy()))
        check_clean(c)
    for r in res[1:]:
        np.testing.assert_array_equal(r[0], res[0][0])
        np.testing.assert_array_equal(r[1], res[0][1])


@pytest.mark.parametrize("precision", F64)
def test_ghosted_patch_equals_periodic_box(precision):
    U = workloads.white_velocity_state((12, 16, 20), seed=4).numpy()
    dx = 1.0 / 20
    dt = 0.5 * oracle.cfl_periodic(U, dx, ocfg())
    Ug = oracle.fill_ghosts_periodic(U)
    c = ctx(precision)
    a = dev(Ug)
    out = torch.zeros_like(a)
    hy.hydro_step(c, hy.patch(a, 2, dx), hy.patch(out, 2, dx), dts(dt))
    torch.cuda.synchronize()
    g = out[:, 2:-2, 2:-2, 2:-2].cpu().numpy()
    assert normwise(g, oracle.step_patch(Ug, dx, dt, ocfg())).max() <= TOL64
    # ghost layers of the output are untouched
    assert float(out[:, :2].abs().max()) == 0.0
    check_clean(c)


def _patch_batch(npatch, seed, precision, dtype, edges=(4, 8, 12, 16, 24), max_level=3):
    parent = workloads.turbulent_state(32, seed=seed, mach=5.0, sedov=False)
    descs = workloads.patch_set(npatch, seed=seed, edges=edges, max_level=max_level)
    origins = workloads.patch_origins(descs, parent.shape[1:], seed=seed)
    ins, outs, host = [], [], []
    for d, o in zip(descs, origins):
        Ug = workloads.ghosted_from_periodic(parent, o, (d["nx"], d["ny"], d["nz"])).numpy()
        host.append((Ug, d))
        t = dev(Ug, dtype)
        ins.append(hy.patch(t, 2, d["dx"], d["level"]))
        outs.append(hy.patch(torch.zeros_like(t), 2, d["dx"], d["level"]))
    return host, ins, outs


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "fp32"])
def test_batched_patches_match_oracle(precision):
    dtype = torch.float32 if precision == "fp32" else torch.float64
    host, ins, outs = _patch_batch(24, 5, precision, dtype, edges=(4, 8, 12, 16, 24, 40))
    c = ctx(precision)
    dt_list = [0.7 * oracle.cfl_patch(Ug, d["dx"], ocfg()) for Ug, d in host]
    dt = dts(*dt_list)
    dn = torch.empty(len(host), dtype=torch.float64, device="cuda")
    for tile in range(hy.NUM_TILES):
        hy.hydro_set_tuning(c, tile, 8 if tile % 2 else 5)
        hy.hydro_step(c, ins, outs, dt, dn)
        torch.cuda.synchronize()
        tol = TOL64 if precision in F64 else TOL32
        for (Ug, d), po, dtp in zip(host, outs, dt_list):
            out = torch.stack(po.tensors).double().cpu().numpy()[:, 2:-2, 2:-2, 2:-2]
            o = oracle.step_patch(Ug, d["dx"], dtp, ocfg())
            assert normwise(out, o).max() <= tol, (precision, tile, d, normwise(out, o))
    # per-patch dt of U^{n+1}: fused and standalone agree bitwise
    dn2 = torch.empty_like(dn)
    hy.hydro_cfl_dt(c, outs, dn2)
    torch.cuda.synchronize()
    assert torch.equal(dn, dn2)
    check_clean(c)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("limiter", ["minmod", "mc"])
def test_reduced_precision_one_step(precision, limiter):
    """FP32 state rounded from the FP64 initial state, one step, vs the FP64 oracle."""
    U = workloads.turbulent_state(32, seed=2, mach=5.0, sedov=True).numpy()
    dx = 1.0 / 32
    dt = oracle.cfl_periodic(U, dx, ocfg(limiter))
    c = ctx(precision, limiter)
    Uin = U.astype(np.float32).astype(np.float64) if precision == "fp32" else U
    g, _ = step_periodic(c, Uin, dx, dt)
    o = oracle.step_periodic(U, dx, dt, ocfg(limiter))
    assert normwise(g, o).max() <= TOL32, normwise(g, o)
    check_clean(c)


def test_fp32_conservation_100_steps():
    U0 = workloads.turbulent_state(32, seed=2, mach=5.0, sedov=False).numpy()
    dx = 1.0 / 32
    c = ctx("fp32")
    a = dev(U0, torch.float32)
    b = torch.empty_like(a)
    tot0 = a.double().sum(dim=(1, 2, 3))
    scale = a.double().abs().sum(dim=(1, 2, 3))
    hist = torch.empty(101, dtype=torch.float64, device="cuda")
    hy.hydro_run(c, hy.patch(a, 0, dx), hy.patch(b, 0, dx), 100, hist)
    torch.cuda.synchronize()
    tot = a.double().sum(dim=(1, 2, 3))
    rel = ((tot - tot0).abs() / scale).max().item()
    assert rel <= 1e-6, rel
    check_clean(c)


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "fp32"])
def test_octs_match_oracle_and_uniform_grid(precision):
    dtype = torch.float32 if precision == "fp32" else torch.float64
    parent = workloads.white_velocity_state(16, seed=6)
    dx = 1.0 / 16
    U = parent.numpy()
    dt = 0.6 * oracle.cfl_periodic(U, dx, ocfg())
    origins = workloads.oct_origins(37, parent.shape[1:], seed=6)
    gathered = workloads.gather_octs(parent, origins)  # (5, G, 6, 6, 6)
    c = ctx(precision)
    gd = gathered.to(device="cuda", dtype=dtype).contiguous()
    od = torch.zeros((5, gd.shape[1], 2, 2, 2), dtype=dtype, device="cuda")
    hy.hydro_step_octs(c, gd, od, dx, dts(dt))
    torch.cuda.synchronize()
    full = oracle.step_periodic(U, dx, dt, ocfg())
    tol = {"fp64": 1e-13, "df64": TOL64}.get(precision, TOL32)
    g = od.double().cpu().numpy()
    for k, (ox, oy, oz) in enumerate(origins):
        o = full[:, oz:oz + 2, oy:oy + 2, ox:ox + 2]
        err = np.abs(g[:, k] - o).max(axis=(1, 2, 3)) / np.abs(full).max(axis=(1, 2, 3))
        assert err.max() <= tol, (k, err)
    check_clean(c)


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "fp32"])
def test_octs_from_level_grid_equal_gathered_octs(precision):
    """hydro_step_octs_level (stencils read in place from the periodic level, wrapped) gives the
    bits of hydro_step_octs on the gathered stencils; origins on the grid's edges included; an
    origin outside the grid flags HYDRO_EBIT_BAD_TILE and leaves its group unwritten."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    shape = (12, 10, 14)
    parent = workloads.turbulent_state(shape, seed=7, mach=2.0, sedov=False)
    dx = 1.0 / 14
    dt = 0.6 * oracle.cfl_periodic(parent.numpy(), dx, ocfg())
    rng = np.random.default_rng(8)
    origins = np.stack([rng.integers(0, 14, 61), rng.integers(0, 10, 61), rng.integers(0, 12, 61)], axis=1)
    origins[:4] = [[0, 0, 0], [13, 9, 11], [12, 8, 10], [1, 9, 0]]
    c = ctx(precision)
    gd = workloads.gather_octs(parent, origins).to(device="cuda", dtype=dtype).contiguous()
    og = torch.zeros((5, len(origins), 2, 2, 2), dtype=dtype, device="cuda")
    hy.hydro_step_octs(c, gd, og, dx, dts(dt))
    level = parent.to(device="cuda", dtype=dtype).contiguous()
    ol = torch.zeros_like(og)
    od = torch.as_tensor(origins, dtype=torch.int32, device="cuda").contiguous()
    hy.hydro_step_octs_level(c, hy.patch(level, 0, dx), od, ol, dts(dt))
    torch.cuda.synchronize()
    assert torch.equal(ol, og)
    check_clean(c)
    bad = od.clone()
    bad[5] = torch.tensor([14, 0, 0], dtype=torch.int32)
    ob = torch.full_like(og, 7.0)
    hy.hydro_step_octs_level(c, hy.patch(level, 0, dx), bad, ob, dts(dt))
    torch.cuda.synchronize()
    rc, bits = hy.hydro_get_error(c)
    assert bits & hy.EBIT_BAD_TILE
    assert torch.equal(ob[:, 5], torch.full_like(ob[:, 5], 7.0))
    keep = [k for k in range(len(origins)) if k != 5]
    assert torch.equal(ob[:, keep], og[:, keep])


def test_error_word_flags_and_argument_errors():
    U = workloads.white_velocity_state(8, seed=1).numpy()
    c = ctx("fp64")
    a = dev(U)
    b = torch.empty_like(a)
    # dt <= 0: flagged on the device, nothing written
    hy.hydro_step(c, hy.patch(a, 0, 0.1), hy.patch(b, 0, 0.1), dts(0.0))
    rc, bits = hy.hydro_get_error(c)
    assert rc == hy.HYDRO_ERR_UNPHYSICAL and bits & hy.EBIT_BAD_DT
    hy.hydro_clear_error(c)
    check_clean(c)
    # a non-finite cell is flagged
    a[0, 3, 3, 3] = float("nan")
    hy.hydro_step(c, hy.patch(a, 0, 0.1), hy.patch(b, 0, 0.1), dts(1e-3))
    rc, bits = hy.hydro_get_error(c)
    assert bits & hy.EBIT_NONFINITE
    hy.hydro_clear_error(c)
    # negative internal energy is flagged (and floored)
    a = dev(U)
    a[4, 2, 2, 2] = 0.0
    hy.hydro_step(c, hy.patch(a, 0, 0.1), hy.patch(b, 0, 0.1), dts(1e-3))
    rc, bits = hy.hydro_get_error(c)
    assert bits & hy.EBIT_P_FLOOR
    hy.hydro_clear_error(c)
    # host-side argument errors: aliasing, bad ghost width, wrong strides
    with pytest.raises(hy.HydroError) as e:
        hy.hydro_step(c, hy.patch(a, 0, 0.1), hy.patch(a, 0, 0.1), dts(1e-3))
    assert e.value.status == hy.HYDRO_ERR_ARG
    with pytest.raises(hy.HydroError):
        hy.hydro_step(c, hy.patch(a, 1, 0.1), hy.patch(b, 1, 0.1), dts(1e-3))
    with pytest.raises(hy.HydroError):
        hy.hydro_step(c, hy.patch(a, 0, -0.1), hy.patch(b, 0, -0.1), dts(1e-3))
    with pytest.raises(hy.HydroError):  # FP32 context given FP64 data of odd alignment is fine; a bad dx is not
        hy.hydro_cfl_dt(c, hy.patch(a, 0, 0.0), dts(0.0))
    check_clean(c)


@pytest.mark.parametrize("precision", ALL)
def test_odd_sizes_odd_strides_and_unaligned_views(precision):
    """Ghosted patches of odd sizes stored as views with odd row strides that start one element into
    their buffer, and a periodic box of odd size stored the same way: the paired (vector) halo loads
    fall back to single-cell loads wherever a pair is not adjacent or not aligned in memory, and every
    tile shape still gives the oracle's step."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    tol = TOL64 if precision in F64 else TOL32
    rnd = (lambda a: a.astype(np.float32).astype(np.float64)) if precision == "fp32" else (lambda a: a)
    parent = workloads.turbulent_state(16, seed=8, mach=3.0, sedov=False)
    dims = [(5, 7, 9), (13, 3, 11), (1, 1, 1), (17, 19, 6)]
    origins = [(3, 5, 7), (15, 0, 2), (8, 8, 8), (0, 11, 13)]

    def view_of(arr, pad):
        F, Z, Y, X = arr.shape
        buf = torch.zeros((F, Z, Y, X + pad), dtype=dtype, device="cuda")
        v = buf[:, :, :, 1:1 + X]
        v.copy_(torch.as_tensor(arr))
        return buf, v

    c = ctx(precision)
    keep, ins, outs, host = [], [], [], []
    for (nx, ny, nz), o in zip(dims, origins):
        Ug = rnd(workloads.ghosted_from_periodic(parent, o, (nx, ny, nz)).numpy())
        dx = 1.0 / 64
        b1, vin = view_of(Ug, 2)   # row stride nx + 6: odd for odd nx
        b2, vout = view_of(np.zeros_like(Ug), 4)
        keep += [b1, b2]
        ins.append(hy.patch(vin, 2, dx))
        outs.append(hy.patch(vout, 2, dx))
        host.append((Ug, dx, vout))
    dt_list = [0.7 * oracle.cfl_patch(Ug, dx, ocfg()) for Ug, dx, _ in host]
    U = rnd(workloads.turbulent_state((7, 9, 11), seed=9, mach=3.0, sedov=True).numpy())
    bp, vp = view_of(U, 2)
    bq, vq = view_of(np.zeros_like(U), 2)
    dtp = oracle.cfl_periodic(U, 1.0 / 11, ocfg())
    want_p = oracle.step_periodic(U, 1.0 / 11, dtp, ocfg())
    for tile in range(hy.NUM_TILES):
        hy.hydro_set_tuning(c, tile, 4)
        hy.hydro_step(c, ins, outs, dts(*dt_list))
        hy.hydro_step(c, hy.patch(vp, 0, 1.0 / 11), hy.patch(vq, 0, 1.0 / 11), dts(dtp))
        torch.cuda.synchronize()
        for (Ug, dx, vout), dt in zip(host, dt_list):
            got = vout.double().cpu().numpy()[:, 2:-2, 2:-2, 2:-2]
            assert normwise(got, oracle.step_patch(Ug, dx, dt, ocfg())).max() <= tol, (tile, Ug.shape)
        assert normwise(vq.double().cpu().numpy(), want_p).max() <= tol, tile
    check_clean(c)


@pytest.mark.parametrize("precision", ["df64", "fp32"])
def test_writes_stay_inside_the_output_interior(precision):
    """Canary-padded buffers: each output field lives inside a larger buffer whose every other element
    (the padding around the box in x, y and z, and the output patch's own ghost layers) holds a
    sentinel; after steps with every tile shape and several z chunks, batched and uniform, every
    sentinel is intact: no write lands outside the interior it belongs to."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    sentinel = -12345.0
    c = ctx(precision)
    parent = workloads.turbulent_state(16, seed=10, mach=3.0, sedov=False)
    dims = [(9, 5, 7), (16, 16, 16), (3, 20, 5)]
    ins, outs, bufs = [], [], []
    for k, (nx, ny, nz) in enumerate(dims):
        Ug = workloads.ghosted_from_periodic(parent, (k, 2 * k, 3 * k), (nx, ny, nz)).to(dtype)
        ins.append(hy.patch(Ug.to("cuda").contiguous(), 2, 1.0 / 64))
        buf = torch.full((5, nz + 4 + 6, ny + 4 + 6, nx + 4 + 6), sentinel, dtype=dtype, device="cuda")
        outs.append(hy.patch(buf[:, 3:-3, 3:-3, 3:-3], 2, 1.0 / 64))
        bufs.append(buf)
    dt = torch.empty(len(ins), dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, ins, dt)
    U = workloads.turbulent_state((11, 13, 15), seed=11, mach=3.0, sedov=True).to("cuda", dtype)
    pbuf = torch.full((5, 11 + 4, 13 + 4, 15 + 4), sentinel, dtype=dtype, device="cuda")
    pout = pbuf[:, 2:-2, 2:-2, 2:-2]
    dtp = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, hy.patch(U.contiguous(), 0, 1.0 / 15), dtp)
    for tile in range(hy.NUM_TILES):
        for zc in (3, 32):
            hy.hydro_set_tuning(c, tile, zc)
            hy.hydro_step(c, ins, outs, dt)
            hy.hydro_step(c, hy.patch(U.contiguous(), 0, 1.0 / 15), hy.patch(pout, 0, 1.0 / 15), dtp)
    torch.cuda.synchronize()
    for (nx, ny, nz), buf in zip(dims, bufs):
        inner = torch.zeros_like(buf, dtype=torch.bool)
        inner[:, 5:5 + nz, 5:5 + ny, 5:5 + nx] = True  # the interior: 3 padding + 2 ghost layers in
        assert bool((buf[~inner] == sentinel).all())
        assert not bool((buf[inner] == sentinel).any())
    inner = torch.zeros_like(pbuf, dtype=torch.bool)
    inner[:, 2:-2, 2:-2, 2:-2] = True
    assert bool((pbuf[~inner] == sentinel).all()) and not bool((pbuf[inner] == sentinel).any())
    check_clean(c)


def test_double_float_exponent_range():
    """The double-float policy keeps the exponent range of float (include/hydro.h at HYDRO_FP64_DF).
    The step is scale-covariant (U -> a U scales every flux and update by a, floors scaled alike), so
    the oracle's step of U, times a, is the step of a U: at a = 1e-10 and 1e12 (momentum squares
    ~1e-23 and ~1e22, inside the range) double-float matches it within 1e-12, as FP64 does; at
    a = 1e25 the momentum squares (~1e47) overflow float, and the step flags HYDRO_EBIT_NONFINITE
    instead of returning silent garbage, while native FP64 steps it to the scaled oracle result.
    (Below the range, e.g. a = 1e-20, the squares ~1e-43 underflow and lose their precision: the
    step then is neither FP64-accurate nor guaranteed to flag.)"""
    U = workloads.turbulent_state((12, 16, 20), seed=2, mach=5.0, sedov=False).numpy()
    dx = 1.0 / 20
    dt = 0.5 * oracle.cfl_periodic(U, dx, ocfg())  # the same for a U: velocities and sound speeds keep
    o = oracle.step_periodic(U, dx, dt, ocfg())
    for a, precision, ok in ((1e-10, "df64", True), (1e12, "df64", True), (1e-10, "fp64", True),
                             (1e25, "fp64", True), (1e25, "df64", False)):
        c = ctx(precision, rho_floor=1e-10 * a, p_floor=1e-14 * a)
        g, _ = step_periodic(c, a * U, dx, dt)
        rc, bits = hy.hydro_get_error(c)
        if ok:
            assert rc == hy.HYDRO_OK and bits == 0, (a, precision, bits)
            assert normwise(g / a, o).max() <= TOL64, (a, precision, normwise(g / a, o))
        else:
            assert bits & hy.EBIT_NONFINITE, (a, precision, bits)
        hy.hydro_finalize(c)


@pytest.mark.parametrize("precision", ALL)
def test_tile_shape_per_patch_class(precision, tmp_path):
    """A batch with patches of all three patch-shape classes (an x or y edge of 8; an edge of 24 or 40;
    edges multiples of 16), each class stepped with its own tile shape and z chunk (one persistent
    launch per class, each over its own work-list segment), against the oracle, with the fused dt
    equal to the standalone CFL's bits; hydro_set_tuning puts every class back on the context's
    tuning; the autotuner's choice, per class included, comes back from its cache file."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    tol = TOL64 if precision in F64 else TOL32
    host, ins, outs = _patch_batch(30, 12, precision, dtype, edges=(8, 16, 24, 32, 40))

    def klass(d):
        nx, ny = d["nx"], d["ny"]
        return 0 if min(nx, ny) <= 8 else (1 if nx % 16 or ny % 16 else 2)

    assert {klass(d) for _, d in host} == {0, 1, 2}
    c = ctx(precision)
    for k, (t, z) in enumerate([(2, 8), (1, 5), (3, 16)]):
        hy.hydro_set_class_tuning(c, k, t, z)
    assert hy.hydro_get_class_tuning(c, 1) == (1, 5)
    dt_list = [0.7 * oracle.cfl_patch(Ug, d["dx"], ocfg()) for Ug, d in host]
    dn = torch.empty(len(host), dtype=torch.float64, device="cuda")
    hy.hydro_step(c, ins, outs, dts(*dt_list), dn)
    l0 = hy.hydro_launch_count(c)
    hy.hydro_step(c, ins, outs, dts(*dt_list), dn)  # the work-list cached: one launch per class
    assert hy.hydro_launch_count(c) - l0 == 3
    torch.cuda.synchronize()
    for (Ug, d), po, dtp in zip(host, outs, dt_list):
        out = torch.stack(po.tensors).double().cpu().numpy()[:, 2:-2, 2:-2, 2:-2]
        Ur = Ug.astype(np.float32).astype(np.float64) if precision == "fp32" else Ug
        assert normwise(out, oracle.step_patch(Ur, d["dx"], dtp, ocfg())).max() <= tol, d
    dn2 = torch.empty_like(dn)
    hy.hydro_cfl_dt(c, outs, dn2)
    torch.cuda.synchronize()
    assert torch.equal(dn, dn2)
    hy.hydro_set_tuning(c, 0, 8)
    assert all(hy.hydro_get_class_tuning(c, k) == (0, 8) for k in range(hy.NUM_PATCH_CLASSES))
    with pytest.raises(hy.HydroError):
        hy.hydro_set_class_tuning(c, hy.NUM_PATCH_CLASSES, 0, 8)
    cache = str(tmp_path / "tuning.txt")
    hy.hydro_autotune(c, ins, outs, dts(*dt_list), cache_path=cache)
    tuned = [hy.hydro_get_class_tuning(c, k) for k in range(hy.NUM_PATCH_CLASSES)]
    c2 = ctx(precision)
    hy.hydro_autotune(c2, ins, outs, dts(*dt_list), cache_path=cache)
    assert [hy.hydro_get_class_tuning(c2, k) for k in range(hy.NUM_PATCH_CLASSES)] == tuned
    assert hy.hydro_get_tuning(c2) == hy.hydro_get_tuning(c)
    check_clean(c)
