"""Nested grids (SPH_FLAG_TREE) against the FP64 oracle: clustered inputs
whose smoothing lengths span decades, the list-free path, reverse pairs,
pools and the KDK step."""
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


@pytest.mark.parametrize("n_leaf", [16, 1, 64])
def test_tree_clustered_no_precision_floor(orc, n_leaf):
    # h spans more than 30x; coordinates relative to each target's own level
    # keep the uniform tolerance without the uniform grid's coordinate floor.
    # n_leaf = 1 splits as deep as the supports allow
    p = inputs.clustered(6000, n_spheres=4, seed=9)
    q = as_f32(p)
    g = run_gpu(p, tree=True, n_leaf=n_leaf, count_pairs=True)
    od, of = orc.density_force(q, q["h0"])
    assert od["h"].max() / od["h"].min() > 30
    rep = compare(g, od, of)
    assert abs(g["pairs"][0] - od["n_ngb"].sum()) <= 1e-4 * od["n_ngb"].sum()
    assert abs(g["pairs"][1] - of["n_pairs"].sum()) <= 1e-4 * of["n_pairs"].sum()
    print(rep)


def test_tree_strongly_clustered(orc):
    # the densest configuration of the clustered workload (64 spheres, scale
    # radii 0.002-0.02) at a size the oracle finishes in seconds
    p = inputs.clustered(20000, n_spheres=64, seed=1)
    q = as_f32(p)
    g = run_gpu(p, tree=True)
    od, of = orc.density_force(q, q["h0"])
    assert od["h"].max() / od["h"].min() > 50
    compare(g, od, of)


def test_tree_lattice(orc):
    # uniform h: the leaves are the top cells
    p = inputs.lattice(16)
    q = as_f32(p)
    g = run_gpu(p, tree=True, count_pairs=True)
    od, of = orc.density_force(q, q["h0"])
    compare(g, od, of)
    assert g["pairs"][1] == of["n_pairs"].sum()


@pytest.mark.parametrize("side", [6, 8])
def test_tree_small_boxes(orc, side):
    # 2 and 3 top cells per side: periodic images of the same cell
    p = inputs.lattice(side, seed=side, sigma_v=0.05)
    q = as_f32(p)
    g = run_gpu(p, tree=True)
    od, of = orc.density_force(q, q["h0"])
    compare(g, od, of)


def test_tree_list_free_path(orc):
    # starting guesses far off the converged h: too large (lists overflow)
    # for some particles, too small (the support outgrows the list radius)
    # for others; both take the list-free path and must give the same result
    p = inputs.clustered(6000, n_spheres=4, seed=9)
    q = as_f32(p)
    rng = np.random.default_rng(5)
    scale = np.where(rng.random(len(p["x"])) < 0.3, 1.6, 1.0)
    scale = np.where(rng.random(len(p["x"])) < 0.3, 0.85, scale)
    h_start = (q["h0"] * scale).astype(np.float32)
    g = run_gpu(p, tree=True, h_start=h_start)
    od, of = orc.density_force(q, h_start.astype(np.float64))
    compare(g, od, of)


def test_tree_two_spheres(orc):
    # the served workload's geometry: two dense spheres in a large empty box
    p = inputs.two_spheres(seed=3, n_min=4000, n_max=4000)
    q = as_f32(p)
    g = run_gpu(p, tree=True)
    od, of = orc.density_force(q, q["h0"])
    compare(g, od, of)


def test_tree_deterministic():
    # the reverse pairs are grouped by atomics; their sort makes the sums
    # run in a fixed order, so two evaluations agree bit for bit
    p = inputs.clustered(6000, n_spheres=4, seed=9)
    a = run_gpu(p, tree=True)
    b = run_gpu(p, tree=True)
    for k in ("h", "rho", "div_v", "curl_v", "ax", "ay", "az", "du_dt", "v_sig"):
        assert np.array_equal(a[k], b[k]), k


def test_tree_pool_equals_alone():
    # several boxes in one pool: each box's results equal its own run.  The
    # boxes start from converged smoothing lengths, so that no box needs the
    # rebuild that a synchronous first step repeats for the whole pool.
    import torch
    from paper_2305_13380_gb300 import pool, sph
    boxes = [inputs.clustered(3000, n_spheres=4, seed=s) for s in (1, 2)] + [inputs.lattice(12, seed=4)]
    prm = sph.sph_default_params(flags=sph.SPH_FLAG_TREE)
    for b in boxes:
        W = pool.Pool([b], prm)
        W.start()
        b["h0"] = W.host(("h",))["h"].copy()
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
    torch.cuda.synchronize()


def test_tree_step_matches_oracle(orc):
    import torch
    from paper_2305_13380_gb300 import sph
    from test_gpu_step import _oracle_state, _pool
    p = inputs.clustered(4000, n_spheres=4, seed=7)
    s = _oracle_state(orc, p)
    off, box, arr = _pool([s])
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC | sph.SPH_FLAG_TREE))
    sph.sph_step(ctx, sph.pool(off, box, arr))
    dt_gpu = float(arr["dt"].cpu()[0])
    dt = orc.step(s, 0.1)
    assert dt_gpu == pytest.approx(dt, rel=1e-5)
    g = {k: v.cpu().numpy() for k, v in arr.items()}
    assert np.allclose(g["h"], s["h"], rtol=1e-5)
    assert np.allclose(g["rho"], s["rho"], rtol=1e-5)
    arms = np.sqrt(np.mean(s["ax"] ** 2 + s["ay"] ** 2 + s["az"] ** 2))
    for k in ("ax", "ay", "az"):
        assert np.abs(g[k] - s[k]).max() < 1e-4 * arms
    torch.cuda.synchronize()


def test_tree_coarser_level_fallback(orc):
    # starting guesses half the converged h for a third of the particles put
    # them at levels whose cells are too small for their support; they are
    # re-solved one or more levels coarser inside the same call, so no
    # rebuild is needed and the results still match the oracle
    # (the top cells are sized by the converged h, so only levels below them
    # are too small)
    p = inputs.clustered(6000, n_spheres=4, seed=9)
    q = as_f32(p)
    h_conv = orc.density(q, q["h0"])["h"]
    rng = np.random.default_rng(11)
    h_start = (np.where(rng.random(len(p["x"])) < 0.33, 0.5, 1.0) * h_conv).astype(np.float32)
    g = run_gpu(p, tree=True, h_start=h_start)
    assert g["rebuilds"] == 0
    od, of = orc.density_force(q, h_start.astype(np.float64))
    compare(g, od, of)


def test_tree_rebuild_when_top_cells_too_small(orc):
    # every starting guess too small: the top grid itself is too fine, which
    # only a rebuild of the top cells fixes
    p = inputs.lattice(12, seed=4)
    p["h0"] = p["h0"] * 0.5
    q = as_f32(p)
    g = run_gpu(p, tree=True)
    assert g["rebuilds"] >= 1
    od, of = orc.density_force(q, q["h0"])
    compare(g, od, of)


@pytest.mark.parametrize("case", ["lattice16", "clustered6000", "clustered20000"])
def test_tree_order_bit_exact(orc, case):
    # the nested grids' source order (top cells, then depth-first below them,
    # ties by index) and the top cells' ranges equal the oracle's exactly
    import torch
    from paper_2305_13380_gb300 import sph
    if case == "lattice16":
        p = inputs.lattice(16)
    elif case == "clustered6000":
        p = inputs.clustered(6000, n_spheres=4, seed=9)
    else:
        p = inputs.clustered(20000, n_spheres=64, seed=1)
    ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), flags=sph.SPH_FLAG_TREE))
    t = sph.to_device(p)
    cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], t["h0"])
    cs, perm = sph.sph_cells_copy(ctx, cells)
    assert sph.sph_status(ctx) == 0
    torch.cuda.synchronize()
    ocs, operm = orc.tree_order(p["x"], p["y"], p["z"], p["L"], cells.n_c)
    assert np.array_equal(cs, ocs)
    assert np.array_equal(perm, operm)
