"""Parity at the full sizes of the workloads, in the configurations the bench
times: the cell lists and the nested grids' order of the 2M boxes byte for
byte, and sampled targets of the clustered and batched workloads checked one
by one against the oracle (the samples and the particles their force reads
chosen from the positions alone)."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

from gpu_common import GAMMA_K, as_f32, compare, run_gpu, support_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


def _sampled(orc, q, tg, bound=None):
    """Oracle density of the sampled targets, and their force with the oracle
    density of every particle the force reads: every j with
    r_tj < max(H_t, H_j), found with the position bound on H (a superset,
    nothing of the GPU's); the others keep h = 0, which no pair reaches."""
    n = len(q["x"])
    Hb, tree, X = support_bound(q) if bound is None else bound
    need = set(int(t) for t in tg)
    for t in tg:
        js = np.array(tree.query_ball_point(X[t], Hb.max()), dtype=np.int64)
        d = X[js] - X[t]
        d -= q["L"] * np.round(d / q["L"])
        r = np.sqrt((d ** 2).sum(1))
        need.update(int(j) for j in js[r < np.maximum(Hb[t], Hb[js])])
    need = np.array(sorted(need))
    od_need = orc.density(q, q["h0"], targets=need)
    assert np.all(GAMMA_K * od_need["h"] <= Hb[need])   # the bound holds
    state = {"h": np.zeros(n), "rho": np.ones(n), "f": np.ones(n), "P": np.zeros(n), "c": np.zeros(n),
             "B": np.zeros(n)}
    for k in state:
        state[k][need] = od_need[k]
    of = orc.force(q, state, targets=tg)
    pos = {int(j): k for k, j in enumerate(need)}
    sel = np.array([pos[int(t)] for t in tg])
    od = {k: v[sel] for k, v in od_need.items()}
    return od, of


def test_clustered_2M_sampled(orc):
    # 2^21 particles in 64 Plummer spheres + background: the bench's clustered
    # workload on nested grids; 120 targets spread over all levels
    p = inputs.clustered(1 << 21, n_spheres=64, seed=0)
    q = as_f32(p)
    g = run_gpu(p, tree=True)
    rng = np.random.default_rng(0)
    bound = support_bound(q)
    order = np.argsort(bound[0])
    # targets from the densest to the widest particles (by the position bound)
    tg = np.sort(np.unique(order[np.linspace(0, len(order) - 1, 120).astype(int)]))
    tg = np.unique(np.concatenate([tg, rng.choice(len(order), 20, replace=False)]))
    od, of = _sampled(orc, q, tg, bound)
    assert od["h"].max() / od["h"].min() > 50
    compare(g, od, of, idx=tg)


def test_batched_boxes_full_size(orc):
    # the 256 boxes of the batched workload in one pool on nested grids: the
    # small boxes whole, the largest box sampled
    from paper_2305_13380_gb300 import pool, sph
    boxes = inputs.batch(256, seed0=0)
    P = pool.Pool(boxes, sph.sph_default_params(flags=sph.SPH_FLAG_TREE))
    P.start()
    assert P.status() == 0
    g = P.host(("h", "rho", "f", "div_v", "curl_v", "P", "c", "balsara", "ax", "ay", "az",
                "du_dt", "v_sig"))
    sizes = np.array([len(b["x"]) for b in boxes])
    small = [int(s) for s in np.argsort(sizes)[:2]]
    clustered_small = [int(s) for s in np.argsort(sizes) if s % 2 == 1][:2]
    for s in sorted(set(small + clustered_small)):
        q = as_f32(boxes[s])
        od, of = orc.density_force(q, q["h0"])
        sl = P.sim_slice(s)
        compare({k: v[sl] for k, v in g.items()}, od, of)
    big = int(np.argmax(sizes))
    q = as_f32(boxes[big])
    sl = P.sim_slice(big)
    gb = {k: v[sl] for k, v in g.items()}
    tg = np.sort(np.random.default_rng(1).choice(sizes[big], 60, replace=False))
    od, of = _sampled(orc, q, tg)
    compare(gb, od, of, idx=tg)


def _gpu_cells(p, flags=0):
    import torch
    from paper_2305_13380_gb300 import sph
    ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), flags=flags))
    t = sph.to_device(p)
    cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], t["h0"])
    cs, perm = sph.sph_cells_copy(ctx, cells)
    assert sph.sph_status(ctx) == 0
    torch.cuda.synchronize()
    return cells.n_c, cs, perm


@pytest.mark.parametrize("case", ["lattice128", "clustered2M"])
def test_cells_bit_exact_2M(orc, case):
    """The uniform cell build of the 2M workloads (8-bit radix digits over
    ~18-21 key bits: three passes) against the oracle's counting sort."""
    from gpu_common import expected_nc
    p = inputs.lattice(128) if case == "lattice128" else inputs.clustered(1 << 21, n_spheres=64, seed=0)
    nc, cs, perm = _gpu_cells(p)
    assert nc == expected_nc(as_f32(p)["h0"], p["L"], n=len(p["x"]))
    ocs, operm = orc.build_cells(p["x"], p["y"], p["z"], p["L"], nc)
    assert np.array_equal(cs, ocs)
    assert np.array_equal(perm, operm)


def test_tree_order_bit_exact_2M(orc):
    """The nested grids' source order of the 2M clustered box (64-bit keys:
    top cell and the Morton code of the 1024^3 sub-cells) against the
    oracle's depth-first order."""
    from paper_2305_13380_gb300 import sph
    p = inputs.clustered(1 << 21, n_spheres=64, seed=0)
    nc, cs, perm = _gpu_cells(p, sph.SPH_FLAG_TREE)
    ocs, operm = orc.tree_order(p["x"], p["y"], p["z"], p["L"], nc)
    assert np.array_equal(cs, ocs)
    assert np.array_equal(perm, operm)
