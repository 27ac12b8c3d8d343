"""Pins of the oct-level oracle (oracle/octs.py): Morton order against a recursive octant walk,
the neighbour table against a pairwise geometric search, and the step of octs read through the
table against the pinned uniform-grid step of the same level."""
import numpy as np
import pytest

import oracle
from oracle import octs
import workloads


def z_walk(level):
    """Positions of the 2^level cube in the order of a recursive octant walk (octant i has
    x = i & 1, y = (i >> 1) & 1, z = i >> 2, visited in increasing i at every scale)."""
    if level == 0:
        return [(0, 0, 0)]
    half = 1 << (level - 1)
    sub = z_walk(level - 1)
    out = []
    for i in range(8):
        ox, oy, oz = (i & 1) * half, ((i >> 1) & 1) * half, (i >> 2) * half
        out += [(ox + x, oy + y, oz + z) for (x, y, z) in sub]
    return out


def test_morton_key_unit_values():
    assert octs.morton_key(1, 0, 0) == 1
    assert octs.morton_key(0, 1, 0) == 2
    assert octs.morton_key(0, 0, 1) == 4
    assert octs.morton_key(3, 3, 3) == 63
    for b in range(10):
        assert octs.morton_key(1 << b, 0, 0) == 8 ** b
        assert octs.morton_key(0, 1 << b, 0) == 2 * 8 ** b
        assert octs.morton_key(0, 0, 1 << b) == 4 * 8 ** b
    assert octs.morton_key(1023, 1023, 1023) == (1 << 30) - 1


def test_sfc_order_is_the_recursive_octant_walk():
    walk = np.array(z_walk(3))  # 8^3 positions
    rng = np.random.default_rng(11)
    perm = rng.permutation(len(walk))
    pos = walk[perm]
    order = octs.sfc_order(pos)
    assert np.array_equal(pos[order], walk)


def test_sfc_order_keeps_aligned_blocks_contiguous():
    """Every aligned 2^m block of a 16^3 level occupies consecutive places of the order."""
    rng = np.random.default_rng(12)
    g = np.stack(np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij"), -1).reshape(-1, 3)
    pos = g[rng.permutation(len(g))]
    ranked = pos[octs.sfc_order(pos)]
    for m in (1, 2, 3):
        block = ranked >> m
        # block ids change only at multiples of 8^m
        change = np.nonzero(np.any(block[1:] != block[:-1], axis=1))[0] + 1
        assert np.all(change % (8 ** m) == 0)


def test_duplicate_positions_rejected():
    with pytest.raises(ValueError):
        octs.sfc_order([[1, 2, 3], [0, 0, 0], [1, 2, 3]])
    with pytest.raises(ValueError):
        octs.neighbour_table([[1, 2, 3], [1, 2, 3]], (4, 4, 4))


def test_neighbour_table_against_pairwise_search():
    dims = (6, 5, 7)
    rng = np.random.default_rng(13)
    allpos = np.stack(np.meshgrid(np.arange(6), np.arange(5), np.arange(7), indexing="ij"), -1).reshape(-1, 3)
    pos = allpos[rng.choice(len(allpos), 120, replace=False)]
    nbr = octs.neighbour_table(pos, dims)
    n = len(pos)
    expect = np.full((n, 27), -1)
    for a in range(n):
        for b in range(n):
            d = [(int(pos[b, k]) - int(pos[a, k])) % dims[k] for k in range(3)]
            # offset -1, 0 or +1 along each axis reaches b (sizes >= 3: at most one offset does)
            off = []
            for k in range(3):
                m = [s for s in (-1, 0, 1) if s % dims[k] == d[k]]
                off.append(m[0] if m else None)
            if None not in off:
                expect[a, ((off[2] + 1) * 3 + off[1] + 1) * 3 + off[0] + 1] = b
    assert np.array_equal(nbr, expect)
    assert np.array_equal(nbr[:, 13], np.arange(n))


def test_level_oct_round_trip():
    U = np.arange(5 * 4 * 6 * 8, dtype=np.float64).reshape(5, 4, 6, 8)
    V, pos = octs.level_to_octs(U)
    assert V.shape == (5, 2 * 3 * 4, 8)
    o = 1 + 4 * (2 + 3 * 1)  # oct (1, 2, 1)
    assert tuple(pos[o]) == (1, 2, 1)
    for k in range(2):
        for j in range(2):
            for i in range(2):
                assert np.array_equal(V[:, o, (k * 2 + j) * 2 + i], U[:, 2 + k, 4 + j, 2 + i])
    assert np.array_equal(octs.octs_to_level(V, U.shape[1:]), U)


def test_table_step_equals_uniform_grid_step():
    """Every oct of a periodic 8x6x10 level stepped through the table gives the uniform-grid step
    of the level, cell for cell; the octs' storage order does not matter."""
    shape = (8, 6, 10)
    U = workloads.turbulent_state(shape, seed=14, mach=2.0, sedov=False).numpy()
    dx = 1.0 / 10
    cfg = oracle.config()
    dt = 0.6 * oracle.cfl_periodic(U, dx, cfg)
    V, pos = octs.level_to_octs(U)
    rng = np.random.default_rng(15)
    perm = rng.permutation(len(pos))  # shuffled storage
    Vs, ps = V[:, perm], pos[perm]
    nbr = octs.neighbour_table(ps, (5, 3, 4))
    out = octs.step_octs_table(Vs, nbr, octs.sfc_order(ps), dx, dt, cfg)
    back = np.empty_like(V)
    back[:, perm[octs.sfc_order(ps)]] = out
    full = oracle.step_periodic(U, dx, dt, cfg)
    err = np.abs(octs.octs_to_level(back, shape) - full).max() / np.abs(full).max()
    assert err <= 1e-15, err


def test_missing_neighbour_rejected():
    pos = np.array([[0, 0, 0], [1, 0, 0]])
    nbr = octs.neighbour_table(pos, (4, 4, 4))
    assert nbr[0, 14] == 1 and nbr[0, 12] == -1
    with pytest.raises(ValueError):
        octs.gather_stencil(np.zeros((5, 2, 8)), nbr, 0)
