"""GPU parity of the oct-level chunk builder (Morton order, neighbour table) and of the step of
octs read through the table, against oracle/octs.py, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from oracle import octs as ooct
import workloads
from hydro_testlib import check_clean, ctx, dts

import paper_1412_0934_gb300 as hy

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def ipos(p):
    return torch.as_tensor(np.asarray(p), dtype=torch.int32).cuda().contiguous()


def build(c, pos, dims, with_nbr=True):
    n = len(pos)
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    nbr = torch.empty((n, 27), dtype=torch.int32, device="cuda") if with_nbr else None
    hy.hydro_octs_build(c, ipos(pos), dims, order, nbr)
    torch.cuda.synchronize()
    return order.cpu().numpy(), (nbr.cpu().numpy() if with_nbr else None)


@pytest.mark.parametrize("dims,count", [((7, 5, 6), 130), ((16, 16, 16), 4096), ((1, 1, 1), 1), ((3, 1, 2), 6),
                                        ((1024, 2, 3), 2000), ((37, 29, 41), 12000)])
def test_build_matches_oracle(dims, count):
    rng = np.random.default_rng(sum(dims) + count)
    total = dims[0] * dims[1] * dims[2]
    flat = rng.choice(total, count, replace=False)
    pos = np.stack([flat % dims[0], (flat // dims[0]) % dims[1], flat // (dims[0] * dims[1])], axis=1)
    c = ctx("fp64")
    order, nbr = build(c, pos, dims)
    check_clean(c)
    assert np.array_equal(order, ooct.sfc_order(pos))
    assert np.array_equal(nbr, ooct.neighbour_table(pos, dims))
    order2, _ = build(c, pos, dims, with_nbr=False)
    assert np.array_equal(order2, order)
    check_clean(c)


def test_build_flags_bad_positions():
    c = ctx("fp64")
    build(c, [[1, 2, 3], [0, 0, 0], [1, 2, 3]], (4, 4, 4))
    rc, bits = hy.hydro_get_error(c)
    assert bits & hy.EBIT_BAD_TILE
    hy.hydro_clear_error(c)
    order, _ = build(c, [[0, 0, 0], [4, 0, 0]], (4, 4, 4))
    rc, bits = hy.hydro_get_error(c)
    assert bits & hy.EBIT_BAD_TILE
    assert order[0] == 0 and order[1] == -1
    hy.hydro_clear_error(c)
    with pytest.raises(hy.HydroError):
        build(c, [[0, 0, 0]], (1025, 1, 1))
    with pytest.raises(hy.HydroError):
        build(c, [[0, 0, 0]], (0, 1, 1))


def level_octs(shape, seed):
    U = workloads.turbulent_state(shape, seed=seed, mach=2.0, sedov=False).numpy()
    V, pos = ooct.level_to_octs(U)
    rng = np.random.default_rng(seed + 1)
    perm = rng.permutation(len(pos))
    return U, V[:, perm], pos[perm]


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "fp32"])
def test_table_step_matches_oracle_and_gathered_octs(precision):
    """Octs of a shuffled oct-major level stepped through the device-built table: equal to the
    oracle's step through its table, and bit-equal to hydro_step_octs on the same stencils
    gathered; octs not listed keep their contents."""
    dtype = torch.float32 if precision == "fp32" else torch.float64
    shape = (12, 10, 14)
    dims = (7, 5, 6)
    U, V, pos = level_octs(shape, seed=21)
    dx = 1.0 / 14
    cfg = oracle.config()
    dt = 0.6 * oracle.cfl_periodic(U, dx, cfg)
    c = ctx(precision)
    order, nbr = build(c, pos, dims)
    onbr = ooct.neighbour_table(pos, dims)
    oorder = ooct.sfc_order(pos)
    assert np.array_equal(order, oorder) and np.array_equal(nbr, onbr)
    listed = oorder[np.sort(np.random.default_rng(22).choice(len(oorder), 97, replace=False))]
    Vd = torch.as_tensor(V).to(device="cuda", dtype=dtype).contiguous()
    out = torch.full_like(Vd, 7.0)
    hy.hydro_step_octs_table(c, Vd, out, torch.as_tensor(nbr).cuda().contiguous(), ipos(listed), dx, dts(dt))
    torch.cuda.synchronize()
    check_clean(c)
    g = out.double().cpu().numpy()
    rest = np.setdiff1d(np.arange(len(pos)), listed)
    assert np.all(g[:, rest] == 7.0)
    ref = ooct.step_octs_table(V, onbr, listed, dx, dt, cfg)
    tol = {"fp64": 1e-13, "df64": TOL64}.get(precision, TOL32)
    err = np.abs(g[:, listed] - ref).max(axis=(1, 2)) / np.abs(ref).max(axis=(1, 2))
    assert err.max() <= tol, err
    # the same stencils gathered and stepped by hydro_step_octs: the same bits
    Vc = Vd.double().cpu().numpy()
    gath = np.stack([ooct.gather_stencil(Vc, onbr, o) for o in listed], axis=1)
    gd = torch.as_tensor(gath).to(device="cuda", dtype=dtype).contiguous()
    og = torch.zeros((5, len(listed), 2, 2, 2), dtype=dtype, device="cuda")
    hy.hydro_step_octs(c, gd, og, dx, dts(dt))
    torch.cuda.synchronize()
    assert torch.equal(out[:, torch.as_tensor(listed).cuda().long()].reshape(og.shape), og)
    check_clean(c)


def test_table_step_of_whole_level_equals_uniform_step():
    """Every oct of the level, listed in Morton order: the reassembled level equals the uniform
    periodic step of the level (FP64)."""
    shape = (16, 12, 20)
    dims = (10, 6, 8)
    U, V, pos = level_octs(shape, seed=23)
    dx = 1.0 / 20
    cfg = oracle.config()
    dt = 0.6 * oracle.cfl_periodic(U, dx, cfg)
    c = ctx("fp64")
    order, nbr = build(c, pos, dims)
    assert np.array_equal(order, ooct.sfc_order(pos))
    Vd = torch.as_tensor(V).cuda().contiguous()
    out = torch.empty_like(Vd)
    hy.hydro_step_octs_table(c, Vd, out, torch.as_tensor(nbr).cuda().contiguous(), ipos(order), dx, dts(dt))
    torch.cuda.synchronize()
    check_clean(c)
    g = out.cpu().numpy()
    back = np.empty_like(g)
    # each stored oct's index in the unshuffled numbering (x fastest, then y, then z)
    back[:, pos[:, 0] + dims[0] * (pos[:, 1] + dims[1] * pos[:, 2])] = g
    full = oracle.step_periodic(U, dx, dt, cfg)
    err = np.abs(ooct.octs_to_level(back, shape) - full).max(axis=(1, 2, 3)) / np.abs(full).max(axis=(1, 2, 3))
    assert err.max() <= 1e-13, err


def test_missing_neighbour_and_bad_list_skip_the_oct():
    shape = (12, 10, 14)
    dims = (7, 5, 6)
    U, V, pos = level_octs(shape, seed=24)
    keep = np.ones(len(pos), bool)
    keep[5] = False  # a hole in the level
    pos_h, V_h = pos[keep], V[:, keep]
    c = ctx("fp64")
    order, nbr = build(c, pos_h, dims)
    check_clean(c)
    onbr = ooct.neighbour_table(pos_h, dims)
    assert np.array_equal(nbr, onbr)
    lacking = np.nonzero((onbr < 0).any(axis=1))[0]
    assert len(lacking) == 26
    lack = set(int(o) for o in lacking)
    ok = [int(o) for o in ooct.sfc_order(pos_h) if int(o) not in lack][:40]
    bad = [int(o) for o in lacking[::5]]
    listed = np.array(ok[:20] + bad + ok[20:] + [len(pos_h) + 3], dtype=np.int32)
    Vd = torch.as_tensor(V_h).cuda().contiguous()
    out = torch.full_like(Vd, 7.0)
    dx = 1.0 / 14
    dt = 0.6 * oracle.cfl_periodic(U, dx, oracle.config())
    hy.hydro_step_octs_table(c, Vd, out, torch.as_tensor(nbr).cuda().contiguous(), ipos(listed), dx, dts(dt))
    torch.cuda.synchronize()
    rc, bits = hy.hydro_get_error(c)
    assert bits & hy.EBIT_BAD_TILE
    g = out.cpu().numpy()
    assert np.all(g[:, bad] == 7.0)
    ref = ooct.step_octs_table(V_h, onbr, ok, dx, dt, oracle.config())
    err = np.abs(g[:, ok] - ref).max(axis=(1, 2)) / np.abs(ref).max(axis=(1, 2))
    assert err.max() <= 1e-13
    # overlapping in and out: an argument error, nothing launched
    with pytest.raises(hy.HydroError):
        hy.hydro_step_octs_table(c, Vd, Vd, torch.as_tensor(nbr).cuda().contiguous(), ipos(listed), dx, dts(dt))
