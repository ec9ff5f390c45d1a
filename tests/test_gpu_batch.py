"""Batched simulations: one sph_step for a pool of independent boxes of
uneven size (jittered lattices and Plummer-clustered boxes), captured in a
CUDA graph and replayed."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

from gpu_common import as_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


def _boxes():
    # small boxes of the batched workload (even: lattice, odd: 4 Plummer spheres)
    return inputs.batch(6, seed0=0, n_min=1000, n_max=4000)


def _params(grid):
    from paper_2305_13380_gb300 import sph
    if grid == "nested":
        # the configuration the batched bench runs (its tuned choice)
        return sph.sph_default_params(flags=sph.SPH_FLAG_TREE, cell_margin=0.03, n_leaf=32)
    return sph.sph_default_params()


@pytest.mark.parametrize("grid", ["uniform", "nested"])
def test_graph_replay_equals_plain_steps(grid):
    from paper_2305_13380_gb300 import pool
    boxes = _boxes()
    a = pool.Pool(boxes, _params(grid))
    b = pool.Pool(boxes, _params(grid))
    a.start()
    b.start()
    b.capture()          # includes one warm-up step
    a.step()
    for _ in range(3):
        a.step()
        b.replay()
    ha, hb = a.host(), b.host()
    assert a.status() == 0 and b.status() == 0
    for k in ha:
        assert np.array_equal(ha[k], hb[k]), k


@pytest.mark.parametrize("grid", ["uniform", "nested"])
def test_batched_box_matches_oracle(orc, grid):
    """The first density + force of every box of the pool against the oracle.
    On the nested grids (the batched bench's configuration) every box holds
    the plain bounds; on one uniform grid the clustered boxes' densest
    particles sit in cells ~100 supports wide and get the coordinate floor."""
    from gpu_common import compare
    from paper_2305_13380_gb300 import pool
    boxes = _boxes()
    P = pool.Pool(boxes, _params(grid))
    P.start()
    assert P.status() == 0
    g = P.host(("h", "rho", "f", "div_v", "curl_v", "P", "c", "balsara", "ax", "ay", "az",
                "du_dt", "v_sig"))
    for s, p in enumerate(boxes):
        q = as_f32(p)
        od, of = orc.density_force(q, q["h0"])
        sl = P.sim_slice(s)
        gs = {k: v[sl] for k, v in g.items()}
        if s % 2 == 0 or grid == "nested":
            compare(gs, od, of)
        else:
            # clustered boxes sit on one uniform grid: add the coordinate floor
            from gpu_common import expected_nc
            nc = expected_nc(q["h0"], p["L"], n=len(p["x"]))
            vmax = float(np.sqrt(q["vx"] ** 2 + q["vy"] ** 2 + q["vz"] ** 2).max())
            compare(gs, od, of, cell=p["L"] / nc, vmax=vmax)


def test_split_group_equals_its_pools_alone(orc):
    """The batched bench's split: the lattice boxes on the uniform grid and the
    clustered boxes on nested grids, two pools forked onto their own streams
    and captured in one graph.  Each pool's results equal those of the same
    pool stepped alone (bitwise), and every box holds the plain bounds against
    the oracle."""
    from gpu_common import compare
    from paper_2305_13380_gb300 import pool, sph, tune
    boxes = _boxes()
    parts = tune.partition(boxes)
    assert [sorted(p) for p in parts] == [[0, 2, 4], [1, 3, 5]]
    prm = [_params("uniform"), _params("nested")]
    alone = [pool.Pool([boxes[i] for i in idx], prm[k]) for k, idx in enumerate(parts)]
    G = pool.Group([pool.Pool([boxes[i] for i in idx], prm[k]) for k, idx in enumerate(parts)])
    for A in alone:
        A.start()
    G.start()
    g0 = [P.host(("h", "rho", "f", "div_v", "curl_v", "P", "c", "balsara", "ax", "ay", "az", "du_dt",
                  "v_sig")) for P in G.pools]
    for k, idx in enumerate(parts):
        for j, s in enumerate(idx):
            q = as_f32(boxes[s])
            od, of = orc.density_force(q, q["h0"])
            sl = G.pools[k].sim_slice(j)
            compare({key: v[sl] for key, v in g0[k].items()}, od, of)
    G.capture()          # includes one warm-up step
    for A in alone:
        A.step()
    for _ in range(3):
        G.replay()
        for A in alone:
            A.step()
    G.synchronize()
    assert G.status() == 0 and all(A.status() == 0 for A in alone)
    assert G.pools[0].ctx is not G.pools[1].ctx
    for A, P in zip(alone, G.pools):
        ha, hp = A.host(), P.host()
        for key in ha:
            assert np.array_equal(ha[key], hp[key]), key
    assert sph.SPH_FLAG_TREE & G.pools[1].params.flags
