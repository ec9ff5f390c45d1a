"""Pins of the oracle's depth-first order of the nested grids (Sec. 2.1,
Sec. 9.1): a recursive octree partition (a different algorithm) gives the
same order, every cell of every level is contiguous, and every particle lies
in its sub-cell."""
import math

import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs


def _fine(p, n_c):
    """Top cell and sub-cell (0..1023) per axis, from the stated rule."""
    L = p["L"]
    ks, gs = [], []
    for a in ("x", "y", "z"):
        s = (np.asarray(p[a], dtype=np.float64) * n_c) / L
        k = np.clip(np.floor(s).astype(np.int64), 0, n_c - 1)
        g = np.clip(np.floor(s * 1024.0).astype(np.int64), 1024 * k, 1024 * k + 1023) - 1024 * k
        ks.append(k)
        gs.append(g)
    return ks, gs


def _recursive_order(idx, gx, gy, gz, depth):
    """Depth-first order by splitting a cell into its 8 children (child index
    x + 2 y + 4 z of the halves) down to depth 10."""
    if depth == 10 or len(idx) <= 1:
        return sorted(idx)
    b = 9 - depth
    out = []
    for child in range(8):
        cx, cy, cz = child & 1, (child >> 1) & 1, (child >> 2) & 1
        sub = [i for i in idx if ((gx[i] >> b) & 1) == cx and ((gy[i] >> b) & 1) == cy
               and ((gz[i] >> b) & 1) == cz]
        out += _recursive_order(sub, gx, gy, gz, depth + 1)
    return out


@pytest.mark.parametrize("case", ["lattice", "clustered"])
def test_tree_order_equals_recursive_partition(orc, case):
    p = inputs.lattice(7, seed=2) if case == "lattice" else inputs.clustered(1500, n_spheres=3, seed=4)
    n_c = 3
    (kx, ky, kz), (gx, gy, gz) = _fine(p, n_c)
    cell = kx + n_c * (ky + n_c * kz)
    expect = []
    for c in range(n_c ** 3):
        expect += _recursive_order([int(i) for i in np.where(cell == c)[0]], gx, gy, gz, 0)
    cs, perm = orc.tree_order(p["x"], p["y"], p["z"], p["L"], n_c)
    assert perm.tolist() == expect
    assert np.array_equal(np.diff(cs), np.bincount(cell, minlength=n_c ** 3))


def test_every_cell_of_every_level_is_contiguous(orc):
    p = inputs.clustered(3000, n_spheres=4, seed=5)
    n_c = 4
    (kx, ky, kz), (gx, gy, gz) = _fine(p, n_c)
    cs, perm = orc.tree_order(p["x"], p["y"], p["z"], p["L"], n_c)
    for d in range(0, 11):
        sh = 10 - d
        lab = ((kx + n_c * (ky + n_c * kz)) * (1 << 30) + ((gx >> sh) << 20) + ((gy >> sh) << 10)
               + (gz >> sh))[perm]
        # each label appears in one run
        change = np.concatenate([[True], lab[1:] != lab[:-1]])
        assert len(np.unique(lab)) == int(change.sum()), d


def test_particles_lie_in_their_sub_cells(orc):
    p = inputs.clustered(2000, n_spheres=4, seed=6)
    n_c = 5
    L = p["L"]
    (kx, ky, kz), (gx, gy, gz) = _fine(p, n_c)
    sub = L / n_c / 1024
    for k, g, a in ((kx, gx, "x"), (ky, gy, "y"), (kz, gz, "z")):
        lo = (1024 * k + g) * sub
        x = np.asarray(p[a])
        # one rounding of the scaled coordinate: within a tiny fraction of a sub-cell
        assert np.all(x >= lo - 1e-9 * sub) and np.all(x < lo + sub * (1 + 1e-9))


def test_edges_and_empty(orc):
    L = 1.0
    x = np.array([0.0, math.nextafter(1.0, 0.0), 0.5, 0.5])
    y = np.array([0.0, math.nextafter(1.0, 0.0), 0.5, 0.5])
    cs, perm = orc.tree_order(x, y, y, L, 2)
    assert perm.tolist() == [0, 2, 3, 1]  # cell 0, cell 7 (0.5 starts it), ties by index, last cell
    cs0, perm0 = orc.tree_order(np.zeros(0), np.zeros(0), np.zeros(0), L, 3)
    assert len(perm0) == 0 and cs0[-1] == 0
