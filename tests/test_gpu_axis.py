"""Sorted interactions on the uniform grid (SPH_FLAG_AXIS_SORT, Sec. 2.2):
the density filter walks each neighbour cell along the axis linking it to
the target's cell and stops at the search radius.  The neighbour sets are
those of the plain filter (identical pair counts), the sums run in another
order, and everything matches the FP64 oracle at the usual tolerance."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

from gpu_common import as_f32, compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


CASES = {
    "lattice16": lambda: inputs.lattice(16),
    "lattice8_3cells": lambda: inputs.lattice(8, seed=7, sigma_v=0.05),
    "lattice6_2cells": lambda: inputs.lattice(6, seed=6, sigma_v=0.05),
    "mildly_clustered": lambda: inputs.clustered(6000, n_spheres=4, seed=9, a_min=0.03, a_max=0.06),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_axis_sort_matches_oracle_and_plain_filter(orc, case):
    p = CASES[case]()
    q = as_f32(p)
    g = run_gpu(p, count_pairs=True, axis=True)
    plain = run_gpu(p, count_pairs=True)
    od, of = orc.density_force(q, q["h0"])
    compare(g, od, of)
    # the same neighbour sets: pair counts agree exactly
    assert g["pairs"] == plain["pairs"]
    # and the same values up to the order of the sums
    for k in ("h", "rho", "f", "P", "c"):
        assert np.allclose(g[k], plain[k], rtol=5e-6, atol=0), k


def test_axis_sort_with_overflowing_lists(orc):
    # strongly clustered gas on a uniform grid: cells far wider than the
    # densest supports, so lists overflow and those lanes take the direct
    # path; the sorted walk must leave that path intact
    p = inputs.clustered(6000, n_spheres=4, seed=9)
    q = as_f32(p)
    g = run_gpu(p, count_pairs=True, axis=True)
    plain = run_gpu(p, count_pairs=True)
    assert g["pairs"] == plain["pairs"]
    from paper_2305_13380_gb300 import sph
    od, of = orc.density_force(q, q["h0"])
    cell = p["L"] / sph.sph_cells_sync(g["_ctx"], g["_cells"])
    vmax = float(np.sqrt(q["vx"] ** 2 + q["vy"] ** 2 + q["vz"] ** 2).max())
    compare(g, od, of, cell=cell, vmax=vmax)


def test_axis_sort_step_and_pool(orc):
    # a KDK step of two boxes in one pool with the flag, against each box
    # stepped alone with the flag (bitwise) and against the oracle step
    import torch
    from paper_2305_13380_gb300 import pool, sph
    from test_gpu_step import _oracle_state, _pool
    boxes = [inputs.lattice(12, seed=4), inputs.lattice(10, seed=5)]
    prm = sph.sph_default_params(flags=sph.SPH_FLAG_AXIS_SORT)
    P = pool.Pool(boxes, prm)
    P.start()
    P.step()
    got = P.host()
    for s, b in enumerate(boxes):
        S = pool.Pool([b], prm, stream=P.stream)
        S.start()
        S.step()
        one = S.host()
        sl = P.sim_slice(s)
        for k in ("x", "vx", "h", "rho", "ax", "du_dt", "v_sig"):
            assert np.array_equal(got[k][sl], one[k]), (s, k)
    assert P.status() == 0
    p = inputs.lattice(12, seed=4)
    st = _oracle_state(orc, p)
    off, box, arr = _pool([st])
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC | sph.SPH_FLAG_AXIS_SORT))
    sph.sph_step(ctx, sph.pool(off, box, arr))
    dt_gpu = float(arr["dt"].cpu()[0])
    dt = orc.step(st, 0.1)
    assert dt_gpu == pytest.approx(dt, rel=1e-5)
    g = {k: v.cpu().numpy() for k, v in arr.items()}
    assert np.allclose(g["h"], st["h"], rtol=1e-5)
    assert np.allclose(g["rho"], st["rho"], rtol=1e-5)
    arms = np.sqrt(np.mean(st["ax"] ** 2 + st["ay"] ** 2 + st["az"] ** 2))
    for k in ("ax", "ay", "az"):
        assert np.abs(g[k] - st[k]).max() < 1e-4 * arms
    torch.cuda.synchronize()
