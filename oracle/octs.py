"""Test infrastructure: the oct bookkeeping of one AMR level for the device chunk builder --
the space-filling-curve (Morton) order of the level's octs, their neighbour table, and the step
of octs whose 6^3 stencils are read through that table.

Only tests/ import this module; it shares nothing with the CUDA library.

The paper's Ramses GPU procedure (Sec. 3, Fig. 1) orders the cells of a level along the
space-filling curve before cutting them into chunks, and gathers each oct's neighbourhood into a
6^3 buffer; it prints no formula.  Readings:
  - An oct at oct coordinates (X, Y, Z) holds the 2^3 cells 2X..2X+1, 2Y..2Y+1, 2Z..2Z+1 of the
    level.  Storage is oct-major: field f of cell (i, j, k) of oct o is U[f, o, (k*2 + j)*2 + i].
  - Morton key: the bits of X, Y and Z interleaved, x lowest: key bit 3b is bit b of X, bit 3b+1
    is bit b of Y, bit 3b+2 is bit b of Z.
  - SFC order: the oct indices sorted by increasing key (distinct positions have distinct keys).
  - Neighbour table: nbr[o, ((dz+1)*3 + (dy+1))*3 + (dx+1)] is the index of the oct at
    (X+dx, Y+dy, Z+dz), wrapped on the level's periodic oct dims, or -1 when the level has no oct
    there; entry 13 is o itself.
  - The 6^3 stencil of an oct (its cells and two ghost layers) is exactly the cells of its 27-oct
    neighbourhood: stencil cell (x, y, z), each 0..5, is cell (x%2, y%2, z%2) of the neighbour at
    offset (x//2 - 1, y//2 - 1, z//2 - 1).
"""
import numpy as np

from . import step_patch


def morton_key(X, Y, Z, bits=10):
    """Morton keys of oct coordinates (arrays of non-negative ints below 2**bits), bit by bit."""
    X, Y, Z = (np.asarray(a, dtype=np.int64) for a in (X, Y, Z))
    key = np.zeros(np.broadcast(X, Y, Z).shape, dtype=np.int64)
    for b in range(bits):
        key |= ((X >> b) & 1) << (3 * b)
        key |= ((Y >> b) & 1) << (3 * b + 1)
        key |= ((Z >> b) & 1) << (3 * b + 2)
    return key


def sfc_order(pos):
    """Oct indices of pos (n, 3) as (X, Y, Z) in increasing Morton key."""
    pos = np.asarray(pos, dtype=np.int64)
    key = morton_key(pos[:, 0], pos[:, 1], pos[:, 2])
    if len(np.unique(key)) != len(key):
        raise ValueError("two octs at one position")
    return np.argsort(key, kind="stable")


def neighbour_table(pos, dims):
    """(n, 27) neighbour indices of the octs at pos (n, 3) on a periodic level of dims (X, Y, Z)
    octs, -1 where no oct exists."""
    pos = np.asarray(pos, dtype=np.int64)
    where = {}
    for o, p in enumerate(pos):
        t = tuple(int(a) for a in p)
        if t in where:
            raise ValueError("two octs at one position")
        where[t] = o
    nbr = np.full((len(pos), 27), -1, dtype=np.int64)
    for o, (X, Y, Z) in enumerate(pos):
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    q = ((X + dx) % dims[0], (Y + dy) % dims[1], (Z + dz) % dims[2])
                    nbr[o, ((dz + 1) * 3 + (dy + 1)) * 3 + (dx + 1)] = where.get(q, -1)
    return nbr


def level_to_octs(U):
    """Oct-major copy (5, n, 8) of a level U (5, NZ, NY, NX) with even sizes, octs numbered
    x fastest, then y, then z; also returns their positions (n, 3)."""
    U = np.asarray(U)
    _, NZ, NY, NX = U.shape
    Z, Y, X = NZ // 2, NY // 2, NX // 2
    V = U.reshape(5, Z, 2, Y, 2, X, 2).transpose(0, 1, 3, 5, 2, 4, 6).reshape(5, Z * Y * X, 8)
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    pos = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    return np.ascontiguousarray(V), pos


def octs_to_level(V, shape):
    """Inverse of level_to_octs for a level of shape (NZ, NY, NX)."""
    NZ, NY, NX = shape
    Z, Y, X = NZ // 2, NY // 2, NX // 2
    return np.ascontiguousarray(np.asarray(V).reshape(5, Z, Y, X, 2, 2, 2).transpose(0, 1, 4, 2, 5, 3, 6)
                                .reshape(5, NZ, NY, NX))


def gather_stencil(V, nbr, o):
    """The 6^3 ghosted stencil (5, 6, 6, 6) of oct o, read from oct-major V through nbr."""
    G = np.empty((5, 6, 6, 6), dtype=np.float64)
    for z in range(6):
        for y in range(6):
            for x in range(6):
                n = nbr[o, ((z // 2) * 3 + y // 2) * 3 + x // 2]
                if n < 0:
                    raise ValueError("oct %d lacks a neighbour" % o)
                G[:, z, y, x] = V[:, n, ((z % 2) * 2 + y % 2) * 2 + x % 2]
    return G


def step_octs_table(V, nbr, octs, dx, dt, cfg=None):
    """U^{n+1} (5, len(octs), 8) of the listed octs, each stepped on its 6^3 stencil gathered
    through the neighbour table (the same discrete step as a ghosted 2^3 patch)."""
    V = np.asarray(V, dtype=np.float64)
    out = np.empty((5, len(octs), 8), dtype=np.float64)
    for g, o in enumerate(octs):
        out[:, g] = step_patch(gather_stencil(V, nbr, o), dx, dt, cfg).reshape(5, 8)
    return out
