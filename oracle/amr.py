"""Test infrastructure: the coarse-to-fine ghost fill of AMR patches (refinement ratio 2).

Only tests/ import this module; it shares nothing with the CUDA library.

The paper's Ramses GPU procedure builds chunks of patches whose boundary cells are interpolated
from the coarser level (Sec. 3); it prints no formula.  The reading here is the textbook
conservative piecewise-linear prolongation of each conserved variable (Berger & Colella 1989):
a fine cell inside coarse cell C whose centre sits s_d = +-1/4 of the coarse width from C's centre
along axis d receives
    U_f = U_C + s_x D_x + s_y D_y + s_z D_z,    D_d = minmod(U_C - U_{C-e_d}, U_{C+e_d} - U_C),
with minmod as in the scheme (0 when the one-sided differences have opposite signs or one is
zero, else the one of smaller magnitude, the first on a tie).  The eight children of C then
average to U_C, and a field linear across C's neighbours is reproduced exactly.

Index conventions: the coarse level is a periodic box Uc (5, NZ, NY, NX); the fine level has
twice as many cells per axis and the same period, so fine index f lies in coarse cell floor(f/2)
(wrapped), on its upper half when f is odd.
"""
import numpy as np


def minmod(a, b):
    return np.where(a * b <= 0.0, 0.0, np.where(np.abs(a) <= np.abs(b), a, b))


def prolong_cells(Uc, f):
    """U at fine cells with fine-level indices f (N, 3) as (x, y, z): returns (5, N)."""
    Uc = np.asarray(Uc, dtype=np.float64)
    _, NZ, NY, NX = Uc.shape
    f = np.asarray(f, dtype=np.int64)
    C = np.floor_divide(f, 2)
    s = np.where(np.mod(f, 2) == 1, 0.25, -0.25)
    n = np.array([NX, NY, NZ])
    C = np.mod(C, n)

    def at(c):
        return Uc[:, c[:, 2], c[:, 1], c[:, 0]]

    U0 = at(C)
    out = U0.copy()
    for d in range(3):
        e = np.zeros(3, dtype=np.int64)
        e[d] = 1
        Um = at(np.mod(C - e, n))
        Up = at(np.mod(C + e, n))
        out = out + s[None, :, d] * minmod(U0 - Um, Up - U0)
    return out


def fill_ghosts(Uc, Ug, origin):
    """Copy of the ghosted fine patch Ug (5, nz+4, ny+4, nx+4) with its 2 ghost layers filled from
    Uc; origin (x, y, z) = the fine-level index of the patch's first interior cell."""
    Ug = np.array(Ug, dtype=np.float64)
    _, GZ, GY, GX = Ug.shape
    k, j, i = np.meshgrid(np.arange(GZ), np.arange(GY), np.arange(GX), indexing="ij")
    ghost = (i < 2) | (i >= GX - 2) | (j < 2) | (j >= GY - 2) | (k < 2) | (k >= GZ - 2)
    idx = np.stack([i[ghost], j[ghost], k[ghost]], axis=1)
    f = idx - 2 + np.asarray(origin, dtype=np.int64)[None, :]
    vals = prolong_cells(Uc, f)
    for v in range(5):
        Ug[v][ghost] = vals[v]
    return Ug


def coarse_at(Uc_old, Uc_new, theta):
    """The coarse level at a fraction theta (0..1) of its step, linear in time between its states
    before and after the step: (1 - theta) U_old + theta U_new, each product and the sum rounded
    once.  A fine level subcycling inside one coarse step takes its ghosts from this state (the
    paper's time refinement: a finer level advances by smaller steps between the coarse ones, Sec. 2)."""
    w0 = 1.0 - float(theta)
    return w0 * np.asarray(Uc_old, dtype=np.float64) + float(theta) * np.asarray(Uc_new, dtype=np.float64)


def fill_ghosts_time(Uc_old, Uc_new, theta, Ug, origin):
    """fill_ghosts from the coarse level interpolated in time to the fraction theta of its step."""
    return fill_ghosts(coarse_at(Uc_old, Uc_new, theta), Ug, origin)


def prolong_box(Uc):
    """The whole fine level (5, 2NZ, 2NY, 2NX) prolonged from the periodic coarse box."""
    _, NZ, NY, NX = Uc.shape
    k, j, i = np.meshgrid(np.arange(2 * NZ), np.arange(2 * NY), np.arange(2 * NX), indexing="ij")
    f = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    return prolong_cells(Uc, f).reshape(5, 2 * NZ, 2 * NY, 2 * NX)


def exchange_ghosts(patches, origins, period):
    """Ghost cells of each ghosted patch covered by the interior of a patch of the same level (another
    one, or the patch itself across the period) take that interior's values (the level periodic
    with `period` (x, y, z) fine cells); other ghosts are left as they are.  patches: list of (5, nz+4, ny+4, nx+4) arrays; origins: their
    first interior cells (x, y, z).  Returns new arrays.  Patch interiors must not overlap."""
    P = np.asarray(period, dtype=np.int64)
    out = [np.array(p, dtype=np.float64) for p in patches]
    dims = [np.array([p.shape[3] - 4, p.shape[2] - 4, p.shape[1] - 4]) for p in patches]
    for a, (Ua, oa) in enumerate(zip(out, origins)):
        _, GZ, GY, GX = Ua.shape
        k, j, i = np.meshgrid(np.arange(GZ), np.arange(GY), np.arange(GX), indexing="ij")
        ghost = (i < 2) | (i >= GX - 2) | (j < 2) | (j >= GY - 2) | (k < 2) | (k >= GZ - 2)
        f = np.stack([i[ghost], j[ghost], k[ghost]], axis=1) - 2 + np.asarray(oa)[None, :]
        f = np.mod(f, P)
        vals = Ua[:, ghost]
        for b, (Ub, ob) in enumerate(zip(patches, origins)):  # b == a: the patch's own periodic image
            rel = np.mod(f - np.asarray(ob)[None, :], P)  # position inside b's interior, if any
            inside = np.all(rel < dims[b][None, :], axis=1)
            if inside.any():
                r = rel[inside]
                vals[:, inside] = np.asarray(Ub)[:, r[:, 2] + 2, r[:, 1] + 2, r[:, 0] + 2]
        Ua[:, ghost] = vals
    return out


# ------------------------------------------------------------------ flux registers and refluxing
# A patch's boundary-face register, per field: x-low [nz][ny], x-high [nz][ny], y-low [nz][nx],
# y-high [nz][nx], z-low [ny][nx], z-high [ny][nx] (the layout of oracle.patch_boundary_fluxes).
# Registers hold time-integrated fluxes (sum over steps of dt * F).

def _faces(R, n):
    """Split a (5, R) register of a box with interior n = (nx, ny, nz) into the six face arrays."""
    nx, ny, nz = n
    sizes = [nz * ny, nz * ny, nz * nx, nz * nx, ny * nx, ny * nx]
    shapes = [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]
    out, a = [], 0
    for s, sh in zip(sizes, shapes):
        out.append(R[:, a:a + s].reshape((5,) + sh))
        a += s
    return out


def reflux(Uc, origin_c, n_c, Rc, Rf, dxc):
    """Coarse level Uc (5, NZ, NY, NX), periodic, after a coarse step whose fluxes through the
    boundary faces of the coarse box B (origin_c, n_c (x, y, z)) integrate to the register Rc; the
    fine patch covering B (refinement 2) integrated Rf through the same faces.  Each coarse cell
    outside B across one of those faces is corrected from the coarse to the fine flux integral:
        U_C += s / dxc * (Rc_face - (1/4) sum of the 4 fine faces' Rf),
    s = +1 when the face is C's upper face (C below B), -1 when it is its lower face.  Cells
    inside B are left to average_down.  Returns a new array."""
    U = np.array(Uc, dtype=np.float64)
    _, NZ, NY, NX = U.shape
    ox, oy, oz = origin_c
    nx, ny, nz = n_c
    fc = _faces(np.asarray(Rc), (nx, ny, nz))
    ff = _faces(np.asarray(Rf), (2 * nx, 2 * ny, 2 * nz))

    def avg(F):  # (5, 2a, 2b) fine faces -> (5, a, b) coarse-face means
        return 0.25 * (F[:, 0::2, 0::2] + F[:, 1::2, 0::2] + F[:, 0::2, 1::2] + F[:, 1::2, 1::2])

    for side, s in ((0, 1.0), (1, -1.0)):
        d = s / dxc * (fc[side] - avg(ff[side]))  # x faces [k][j]
        x = (ox - 1) % NX if side == 0 else (ox + nx) % NX
        for k in range(nz):
            for j in range(ny):
                U[:, (oz + k) % NZ, (oy + j) % NY, x] += d[:, k, j]
        d = s / dxc * (fc[2 + side] - avg(ff[2 + side]))  # y faces [k][i]
        y = (oy - 1) % NY if side == 0 else (oy + ny) % NY
        for k in range(nz):
            for i in range(nx):
                U[:, (oz + k) % NZ, y, (ox + i) % NX] += d[:, k, i]
        d = s / dxc * (fc[4 + side] - avg(ff[4 + side]))  # z faces [j][i]
        z = (oz - 1) % NZ if side == 0 else (oz + nz) % NZ
        for j in range(ny):
            for i in range(nx):
                U[:, z, (oy + j) % NY, (ox + i) % NX] += d[:, j, i]
    return U


def average_down(Uc, Uf, origin_c):
    """Coarse cells of the box at origin_c (x, y, z) covered by the fine interior Uf (5, 2nz, 2ny,
    2nx) replaced by the mean of their eight children.  Returns a new array."""
    U = np.array(Uc, dtype=np.float64)
    _, NZ, NY, NX = U.shape
    _, FZ, FY, FX = Uf.shape
    m = np.asarray(Uf, dtype=np.float64).reshape(5, FZ // 2, 2, FY // 2, 2, FX // 2, 2)
    mean = 0.125 * m.sum(axis=(2, 4, 6))
    ox, oy, oz = origin_c
    iz = (oz + np.arange(FZ // 2)) % NZ
    iy = (oy + np.arange(FY // 2)) % NY
    ix = (ox + np.arange(FX // 2)) % NX
    U[np.ix_(range(5), iz, iy, ix)] = mean
    return U
