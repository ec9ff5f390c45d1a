"""Pins of the oracle's cell grid (Sec. 2.1, the Verlet-list grid): every
particle sits in the cell that contains it, the order is a stable sort by cell
id, and the neighbour search agrees with brute force."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs


def _geometric_cells(x, L, n_c):
    # independent check: the cell k of x satisfies k L/n_c <= x < (k+1) L/n_c
    # up to one rounding of the boundary
    return x, L / n_c


@pytest.mark.parametrize("n_c", [3, 7, 11])
def test_stable_sort_and_containment(orc, n_c):
    p = inputs.clustered(3000, n_spheres=5, seed=3)
    L = p["L"]
    cs, perm = orc.build_cells(p["x"], p["y"], p["z"], L, n_c)
    n = p["x"].shape[0]
    assert sorted(perm.tolist()) == list(range(n))
    assert cs[0] == 0 and cs[-1] == n
    # per-axis containment, checked geometrically with a one-ulp slack
    c = L / n_c
    cell_of = np.empty(n, dtype=np.int64)
    for cell in range(n_c ** 3):
        seg = perm[cs[cell]:cs[cell + 1]]
        cell_of[seg] = cell
        # stable: ascending input index inside the cell
        assert np.all(np.diff(seg) > 0)
    kx = cell_of % n_c
    ky = (cell_of // n_c) % n_c
    kz = cell_of // (n_c * n_c)
    for k, x in ((kx, p["x"]), (ky, p["y"]), (kz, p["z"])):
        assert np.all(x >= k * c - 1e-15)
        assert np.all(x < (k + 1) * c + 1e-15)
    # the order equals Python's stable sort of the cell ids
    ref = sorted(range(n), key=lambda i: cell_of[i])
    assert perm.tolist() == ref


def test_boundaries(orc):
    L, n_c = 1.0, 5
    assert orc.cell_coord(0.0, L, n_c) == 0
    assert orc.cell_coord(0.2, L, n_c) == 1          # exactly on a face -> upper cell
    assert orc.cell_coord(np.nextafter(0.2, 0.0), L, n_c) == 0
    assert orc.cell_coord(np.nextafter(1.0, 0.0), L, n_c) == n_c - 1
    assert orc.cell_coord(1.0, L, n_c) == n_c - 1    # clamp
    assert orc.wrap(-1e-3, 1.0) == pytest.approx(1.0 - 1e-3)
    assert orc.wrap(1.0, 1.0) == 0.0


def test_empty_and_single(orc):
    cs, perm = orc.build_cells(np.zeros(0), np.zeros(0), np.zeros(0), 1.0, 3)
    assert perm.shape == (0,) and np.all(cs == 0)
    cs, perm = orc.build_cells([0.9], [0.1], [0.5], 1.0, 3)
    assert perm.tolist() == [0]
    cell = 2 + 3 * (0 + 3 * 1)
    assert cs[cell] == 0 and cs[cell + 1] == 1


def test_range_search_matches_brute_force(orc):
    p = inputs.clustered(1500, n_spheres=3, seed=1)
    rng = np.random.default_rng(0)
    t = rng.choice(1500, 60, replace=False)
    R = rng.uniform(0.01, 0.3, 60)
    a = orc.neighbours(p, t, R, brute=False)
    b = orc.neighbours(p, t, R, brute=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
