"""Pins of the friends-of-friends oracle (Sec. 7.1) against things other
than itself: connected components of the brute-force friendship graph from
scipy, closed-form chains, the periodic wrap, and the canonical labels."""
import numpy as np
import pytest

import oracle
from paper_2305_13380_gb300 import inputs


def _brute_labels(x, y, z, L, b):
    # O(N^2) friendship matrix with the same FP64 predicate (minimum image,
    # r2 = dx*dx + dy*dy + dz*dz < b*b), components by scipy, each labelled
    # with its smallest index
    sp = pytest.importorskip("scipy.sparse")
    cg = pytest.importorskip("scipy.sparse.csgraph")

    def mi(d):
        return np.where(d > 0.5 * L, d - L, np.where(d < -0.5 * L, d + L, d))
    dx = mi(x[:, None] - x[None, :])
    dy = mi(y[:, None] - y[None, :])
    dz = mi(z[:, None] - z[None, :])
    adj = (dx * dx + dy * dy + dz * dz) < b * b
    np.fill_diagonal(adj, False)
    n_comp, lab = cg.connected_components(sp.csr_matrix(adj), directed=False)
    first = np.full(n_comp, len(x), dtype=np.int64)
    np.minimum.at(first, lab, np.arange(len(x)))
    return first[lab].astype(np.int32)


@pytest.mark.parametrize("case", ["uniform", "clustered", "lattice_edge"])
def test_fof_matches_brute_force_components(case):
    if case == "uniform":
        rng = np.random.default_rng(3)
        p = {k: rng.random(1500) for k in "xyz"}
        L, b = 1.0, 0.6 * 1500 ** (-1.0 / 3.0)
    elif case == "clustered":
        p = inputs.clustered(1500, n_spheres=4, seed=2)
        L, b = float(p["L"]), 0.2 * 1500 ** (-1.0 / 3.0)
    else:
        # a jittered lattice with b at the spacing: many pairs sit at the
        # linking length, where the FP64 predicate decides
        p = inputs.lattice(11, seed=4)
        L, b = float(p["L"]), 1.0 / 11
    x, y, z = (np.asarray(p[k], dtype=np.float64) for k in "xyz")
    got = oracle.fof(x, y, z, L, b)
    ref = _brute_labels(x, y, z, L, b)
    assert np.array_equal(got, ref)
    assert 1 < len(np.unique(got)) < len(x)


def test_fof_chain_closed_form():
    n, b = 20, 0.01
    x = 0.2 + np.arange(n) * 0.9 * b
    y = np.full(n, 0.5)
    z = np.full(n, 0.5)
    assert np.array_equal(oracle.fof(x, y, z, 1.0, b), np.zeros(n, dtype=np.int32))
    x2 = 0.2 + np.arange(n) * 1.1 * b
    assert np.array_equal(oracle.fof(x2, y, z, 1.0, b), np.arange(n, dtype=np.int32))


def test_fof_links_across_the_periodic_boundary():
    x = np.array([0.995, 0.5, 0.005])
    y = np.array([0.5, 0.5, 0.5])
    z = np.array([0.5, 0.5, 0.5])
    # 0.995 and 0.005 are 0.01 apart through the boundary
    assert oracle.fof(x, y, z, 1.0, 0.02).tolist() == [0, 1, 0]
    assert oracle.fof(x, y, z, 1.0, 0.009).tolist() == [0, 1, 2]


def test_fof_labels_are_smallest_indices_and_follow_a_permutation():
    p = inputs.clustered(800, n_spheres=3, seed=5)
    x, y, z = (np.asarray(p[k], dtype=np.float64) for k in "xyz")
    b = 0.3 * 800 ** (-1.0 / 3.0)
    g = oracle.fof(x, y, z, 1.0, b)
    idx = np.arange(len(x))
    assert np.all(g <= idx) and np.array_equal(g[g], g)
    # relabelling the particles permutes the partition, not its shape
    perm = np.random.default_rng(1).permutation(len(x))
    g2 = oracle.fof(x[perm], y[perm], z[perm], 1.0, b)
    same_a = g[perm][:, None] == g[perm][None, :]
    same_b = g2[:, None] == g2[None, :]
    assert np.array_equal(same_a, same_b)


def test_fof_rejects_a_linking_length_above_a_third_of_the_box():
    with pytest.raises(RuntimeError):
        oracle.fof(np.array([0.1]), np.array([0.1]), np.array([0.1]), 1.0, 0.4)
