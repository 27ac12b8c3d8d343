"""Pins of the coarse-to-fine ghost fill oracle (oracle/amr.py) by what the prolongation must
satisfy: the eight children of a coarse cell average to it; a field linear across a cell's
neighbours is reproduced exactly at the fine centres; no fine value leaves the range of its parent
and the parent's face neighbours (MinMod slopes); a constant field stays constant; the ghost fill
of a patch agrees with the whole-level prolongation, including ghosts that wrap around the
periodic level; the fill from the coarse level interpolated in time between two of its states."""
import numpy as np
import pytest

from oracle import amr


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((5,) + shape) + np.array([3.0, 0.0, 0.0, 0.0, 5.0])[:, None, None, None]


def test_children_average_to_parent():
    Uc = _field((6, 5, 7), 1)
    Uf = amr.prolong_box(Uc)
    avg = Uf.reshape(5, 6, 2, 5, 2, 7, 2).mean(axis=(2, 4, 6))
    assert np.abs(avg - Uc).max() <= 1e-15 * np.abs(Uc).max() * 8


def test_linear_field_reproduced_at_fine_centres():
    NZ, NY, NX = 6, 7, 8
    k, j, i = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    coef = np.array([[1.0, 0.5, -0.25, 2.0], [0.0, -1.0, 0.3, 0.1], [2.0, 0.2, 0.2, -0.7],
                     [-1.0, 0.0, 1.5, 0.4], [4.0, 0.9, -0.6, 0.05]])
    Uc = np.stack([c[0] + c[1] * i + c[2] * j + c[3] * k for c in coef])
    # fine cells whose parent and the parent's neighbours do not wrap
    f = np.array([[x, y, z] for z in range(2, 2 * NZ - 2) for y in range(2, 2 * NY - 2) for x in range(2, 2 * NX - 2)])
    got = amr.prolong_cells(Uc, f)
    pos = f / 2.0 - 0.25  # fine centres in coarse index units
    want = np.stack([c[0] + c[1] * pos[:, 0] + c[2] * pos[:, 1] + c[3] * pos[:, 2] for c in coef])
    assert np.abs(got - want).max() <= 1e-13


def test_no_new_extrema_and_constant_field():
    Uc = _field((5, 6, 4), 2)
    NZ, NY, NX = Uc.shape[1:]
    f = np.array([[x, y, z] for z in range(2 * NZ) for y in range(2 * NY) for x in range(2 * NX)])
    got = amr.prolong_cells(Uc, f)
    C = f // 2
    lo = np.full(got.shape, np.inf)
    hi = np.full(got.shape, -np.inf)
    for e in ([0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]):
        c = np.mod(C + np.array(e), [NX, NY, NZ])
        v = Uc[:, c[:, 2], c[:, 1], c[:, 0]]
        lo, hi = np.minimum(lo, v), np.maximum(hi, v)
    assert (got >= lo - 1e-14).all() and (got <= hi + 1e-14).all()
    const = np.ones((5, 3, 3, 3)) * np.array([1.5, -2.0, 0.0, 0.25, 7.0])[:, None, None, None]
    assert np.array_equal(amr.prolong_box(const), np.ones((5, 6, 6, 6)) * const[:, :1, :1, :1])


@pytest.mark.parametrize("origin", [(0, 0, 0), (5, 3, 1), (10, 12, 8)])
def test_patch_ghosts_agree_with_level_prolongation(origin):
    Uc = _field((6, 7, 6), 3)
    Uf = amr.prolong_box(Uc)  # fine level (12, 14, 12)
    nx, ny, nz = 4, 6, 4
    Ug = amr.fill_ghosts(Uc, np.zeros((5, nz + 4, ny + 4, nx + 4)), origin)
    ox, oy, oz = origin
    ix = np.mod(np.arange(ox - 2, ox + nx + 2), 12)
    iy = np.mod(np.arange(oy - 2, oy + ny + 2), 14)
    iz = np.mod(np.arange(oz - 2, oz + nz + 2), 12)
    ref = Uf[:, iz][:, :, iy][:, :, :, ix]
    interior = np.zeros(Ug.shape[1:], dtype=bool)
    interior[2:-2, 2:-2, 2:-2] = True
    assert np.array_equal(Ug[:, interior], np.zeros((5, interior.sum())))
    assert np.abs(Ug[:, ~interior] - ref[:, ~interior]).max() <= 1e-15 * np.abs(ref).max()


def test_time_interpolated_ghosts():
    """The coarse level between its states: the end points are the plain fills bit for bit; the
    midpoint is symmetric in the two states; a change of the coarse state that is uniform in space
    (so no slope changes) moves every ghost by theta times that change."""
    Uo = _field((6, 7, 6), 5)
    c = np.array([0.3, -0.2, 0.1, 0.05, 0.7])[:, None, None, None]
    Un = Uo + c
    Ug = np.zeros((5, 8, 10, 8))
    origin = (3, 9, 11)
    assert np.array_equal(amr.fill_ghosts_time(Uo, Un, 0.0, Ug, origin), amr.fill_ghosts(Uo, Ug, origin))
    assert np.array_equal(amr.fill_ghosts_time(Uo, Un, 1.0, Ug, origin), amr.fill_ghosts(Un, Ug, origin))
    Ur = _field((6, 7, 6), 6)
    assert np.array_equal(amr.fill_ghosts_time(Uo, Ur, 0.5, Ug, origin), amr.fill_ghosts_time(Ur, Uo, 0.5, Ug, origin))
    base = amr.fill_ghosts(Uo, Ug, origin)
    ghost = np.ones(Ug.shape[1:], dtype=bool)
    ghost[2:-2, 2:-2, 2:-2] = False
    for theta in (0.25, 0.5, 0.8):
        got = amr.fill_ghosts_time(Uo, Un, theta, Ug, origin)
        want = base + theta * c
        assert np.abs(got[:, ghost] - want[:, ghost]).max() <= 1e-14
        assert np.array_equal(got[:, ~ghost], Ug[:, ~ghost])


def test_sibling_exchange_reassembles_a_partitioned_level():
    """A periodic fine level cut into patches that tile it exactly: after the exchange every
    patch's ghosts equal the level's own cells around it (cut independently, with wrap)."""
    rng = np.random.default_rng(5)
    NZ, NY, NX = 8, 6, 10
    level = rng.standard_normal((5, NZ, NY, NX))
    cuts = [(x0, y0, z0, nx, ny, nz) for z0, nz in ((0, 3), (3, 5)) for y0, ny in ((0, 6),)
            for x0, nx in ((0, 4), (4, 2), (6, 4))]
    patches, origins = [], []
    for x0, y0, z0, nx, ny, nz in cuts:
        Ug = np.zeros((5, nz + 4, ny + 4, nx + 4))
        Ug[:, 2:-2, 2:-2, 2:-2] = level[:, z0:z0 + nz, y0:y0 + ny, x0:x0 + nx]
        patches.append(Ug)
        origins.append((x0, y0, z0))
    done = amr.exchange_ghosts(patches, origins, (NX, NY, NZ))
    for Ug, (x0, y0, z0, nx, ny, nz) in zip(done, cuts):
        ix = np.mod(np.arange(x0 - 2, x0 + nx + 2), NX)
        iy = np.mod(np.arange(y0 - 2, y0 + ny + 2), NY)
        iz = np.mod(np.arange(z0 - 2, z0 + nz + 2), NZ)
        assert np.array_equal(Ug, level[:, iz][:, :, iy][:, :, :, ix])


def test_sibling_exchange_leaves_uncovered_ghosts():
    """Two patches apart on a large level: nothing covers their ghosts, which keep their values;
    touching along x, each patch's x ghosts on that side take the other's first two columns."""
    a = np.full((5, 7, 7, 7), 1.0)
    b = np.full((5, 7, 7, 7), 2.0)
    a[:, 2:-2, 2:-2, 2:-2] = 10.0
    b[:, 2:-2, 2:-2, 2:-2] = 20.0
    far = amr.exchange_ghosts([a, b], [(0, 0, 0), (20, 20, 20)], (40, 40, 40))
    assert np.array_equal(far[0], a) and np.array_equal(far[1], b)
    near = amr.exchange_ghosts([a, b], [(0, 0, 0), (3, 0, 0)], (40, 40, 40))
    assert (near[0][:, 2:-2, 2:-2, 5:7] == 20.0).all() and (near[0][:, 2:-2, 2:-2, :2] == 1.0).all()
    assert (near[1][:, 2:-2, 2:-2, 0:2] == 10.0).all() and (near[1][:, 0:2] == 2.0).all()


def _composite_step(reflux_on):
    """Coarse 16^3 periodic level and one fine patch (refinement 2) over the coarse box
    [4, 12)^3, stepped once on the coarse level and twice on the fine one (ghosts prolonged from
    the coarse level at t and, linearly in time, at t + dt/2), then refluxed and averaged down.
    Mach 0.5, density contrast sigma 0.5: with faster flow or stronger contrasts the separately
    interpolated density, momenta and energy of prolonged ghosts can put the energy below the
    kinetic energy, and the pressure floor would act there."""
    import oracle
    import workloads
    Uc = workloads.turbulent_state((16, 16, 16), seed=31, mach=0.5, sigma_rho=0.5, sedov=False).numpy()
    dxc = 1.0 / 16
    cfg = oracle.config()
    dtc = 0.5 * oracle.cfl_periodic(Uc, dxc, cfg)
    oc, nc = (4, 4, 4), (8, 8, 8)
    ofine = tuple(2 * o for o in oc)
    Ucg = workloads.ghosted_from_periodic(torch_tensor(Uc), oc, nc).numpy()
    Rc = dtc * oracle.patch_boundary_fluxes(Ucg, dxc, dtc, cfg)
    Uc1 = oracle.step_periodic(Uc, dxc, dtc, cfg)
    fine_level = amr.prolong_box(Uc)
    Uf = fine_level[:, 8:24, 8:24, 8:24]
    dxf, dtf = dxc / 2, dtc / 2
    Rf = np.zeros_like(Rc, shape=(5, 2 * 3 * 16 * 16))
    for sub, Ut in enumerate((Uc, 0.5 * (Uc + Uc1))):
        Ug = np.zeros((5, 20, 20, 20))
        Ug[:, 2:-2, 2:-2, 2:-2] = Uf
        Ug = amr.fill_ghosts(Ut, Ug, ofine)
        Rf = Rf + dtf * oracle.patch_boundary_fluxes(Ug, dxf, dtf, cfg)
        Uf = oracle.step_patch(Ug, dxf, dtf, cfg)
    U = amr.reflux(Uc1, oc, nc, Rc, Rf, dxc) if reflux_on else Uc1
    return Uc, amr.average_down(U, Uf, oc)


def torch_tensor(a):
    import torch
    return torch.as_tensor(a)


def test_refluxed_composite_step_conserves_to_round_off():
    U0, U1 = _composite_step(True)
    scale = np.abs(U0).sum(axis=(1, 2, 3))
    drift = np.abs(U1.sum(axis=(1, 2, 3)) - U0.sum(axis=(1, 2, 3))) / scale
    assert drift.max() <= 1e-14, drift
    _, U2 = _composite_step(False)  # without the correction the composite level leaks
    leak = np.abs(U2.sum(axis=(1, 2, 3)) - U0.sum(axis=(1, 2, 3))) / scale
    assert leak.max() > 1e-9, leak
