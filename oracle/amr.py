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
