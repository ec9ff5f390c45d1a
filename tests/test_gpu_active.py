"""The loops on an active subset (Sec. 2.4, the per-particle time-step
hierarchy): only the masked particles are updated, every particle is a
neighbour.  Against the oracle on the same targets, and against the
unmasked loops, on the uniform grid and on the nested grids."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

from gpu_common import as_f32, compare

pytestmark = pytest.mark.gpu

SENTINEL = -7.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


GRIDS = ["uniform", "nested"]


def _run(p, masks, same_pointer=True, grid="uniform"):
    """Unmasked density (every particle's state), then the masked density and
    force for each mask; returns the unmasked results and the masked ones."""
    import torch
    from paper_2305_13380_gb300 import sph
    flags = sph.SPH_FLAG_SYNC | (sph.SPH_FLAG_TREE if grid == "nested" else 0)
    ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), flags=flags))
    t = sph.to_device(p)
    n = int(t["x"].shape[0])
    part = sph.particles(t)
    d0, f0 = sph.alloc_density(n), sph.alloc_force(n)
    h_in = t["h0"]
    for _ in range(8):  # rebuild until every support fits its cell
        cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], h_in)
        try:
            sph.sph_density(ctx, cells, part, h_in, sph.density_out(d0))
            break
        except sph.SPHError as e:
            if e.code != sph.SPH_E_REBUILD:
                raise
            h_in = d0["h"].clone()
    sph.sph_force(ctx, cells, part, sph.density_out(d0), sph.force_out(f0))
    base = {k: v.cpu().numpy() for k, v in d0.items()}
    base.update({k: v.cpu().numpy() for k, v in f0.items()})
    outs = []
    for m in masks:
        act = torch.tensor(m.astype(np.uint8), device="cuda")
        d = {k: v.clone() for k, v in d0.items()}
        f = {k: torch.full_like(v, SENTINEL) for k, v in f0.items()}
        for k in ("rho", "f", "div_v", "curl_v", "P", "c", "balsara"):
            d[k][torch.tensor(m, device="cuda")] = SENTINEL
        sph.sph_density_active(ctx, cells, part, h_in, act, sph.density_out(d))
        act_f = act if same_pointer else act.clone()
        sph.sph_force_active(ctx, cells, part, sph.density_out(d), act_f, sph.force_out(f))
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in d.items()}
        g.update({k: v.cpu().numpy() for k, v in f.items()})
        outs.append(g)
    return base, outs


def _blob(p, frac, seed):
    """A seeded spherical region holding about `frac` of the particles (the
    active set of a local event), plus a sprinkling of single particles."""
    rng = np.random.default_rng(seed)
    L = float(p["L"])
    c0 = rng.uniform(0, L, 3)
    d = [(np.asarray(p[k]) - c0[i] + 0.5 * L) % L - 0.5 * L for i, k in enumerate("xyz")]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    m = r < np.quantile(r, frac)
    m |= rng.random(len(r)) < 0.01
    return m


@pytest.mark.parametrize("grid", GRIDS)
def test_all_active_equals_unmasked(grid):
    p = inputs.lattice(16, seed=4, sigma_v=0.05)
    n = len(p["x"])
    base, (g,) = _run(p, [np.ones(n, bool)], grid=grid)
    for k in ("h", "rho", "f", "div_v", "curl_v", "P", "c", "balsara", "ax", "ay", "az", "du_dt", "v_sig"):
        assert np.array_equal(g[k], base[k]), k


@pytest.mark.parametrize("grid", GRIDS)
def test_none_active_changes_nothing(grid):
    p = inputs.lattice(12, seed=4, sigma_v=0.05)
    n = len(p["x"])
    base, (g,) = _run(p, [np.zeros(n, bool)], grid=grid)
    for k in ("ax", "ay", "az", "du_dt", "v_sig"):
        assert np.all(g[k] == SENTINEL), k
    assert np.array_equal(g["h"], base["h"])


@pytest.mark.parametrize("grid,same_pointer", [("uniform", True), ("uniform", False), ("nested", True)])
def test_active_subset_lattice(orc, grid, same_pointer):
    p = inputs.lattice(16, seed=7, sigma_v=0.05)
    m = _blob(p, 0.1, seed=3)
    base, (g,) = _run(p, [m], same_pointer, grid=grid)
    idx = np.where(m)[0]
    q = as_f32(p)
    od_all = orc.density(q, q["h0"])
    od = {k: v[idx] for k, v in od_all.items()}
    of = orc.force(q, od_all, targets=idx)
    compare(g, od, of, idx=idx)
    off = ~m
    for k in ("ax", "ay", "az", "du_dt", "v_sig"):
        assert np.all(g[k][off] == SENTINEL), k
    for k in ("rho", "P", "balsara"):
        assert np.all(g[k][off] == base[k][off]), k


@pytest.mark.parametrize("grid", GRIDS)
def test_active_subset_clustered(orc, grid):
    # on a uniform grid, clustered gas sends dense blocks to the overflow
    # kernels; on the nested grids the masked particles' supports span decades
    # and the unmasked ones send reverse pairs from supports beyond the lists
    p = inputs.clustered(6000, n_spheres=4, seed=9, a_min=0.03, a_max=0.06)
    masks = [_blob(p, 0.2, seed=5), np.random.default_rng(1).random(len(p["x"])) < 0.3]
    base, outs = _run(p, masks, grid=grid)
    q = as_f32(p)
    od_all = orc.density(q, q["h0"])
    for m, g in zip(masks, outs):
        idx = np.where(m)[0]
        od = {k: v[idx] for k, v in od_all.items()}
        of = orc.force(q, od_all, targets=idx)
        compare(g, od, of, idx=idx)
        assert np.all(g["v_sig"][~m] == SENTINEL)


def test_nested_force_needs_the_density_mask():
    """The nested grids' force reads the lists and reverse pairs of the
    density: a force under another mask than the density's (another pointer),
    or without a mask after a masked density, is refused."""
    import torch
    from paper_2305_13380_gb300 import sph
    p = inputs.lattice(8, seed=1)
    ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), flags=sph.SPH_FLAG_TREE | sph.SPH_FLAG_SYNC))
    t = sph.to_device(p)
    n = int(t["x"].shape[0])
    part = sph.particles(t)
    cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], t["h0"])
    d, f = sph.alloc_density(n), sph.alloc_force(n)
    act = torch.ones(n, dtype=torch.uint8, device="cuda")
    sph.sph_density_active(ctx, cells, part, t["h0"], act, sph.density_out(d))
    for call in (lambda: sph.sph_force_active(ctx, cells, part, sph.density_out(d), act.clone(), sph.force_out(f)),
                 lambda: sph.sph_force(ctx, cells, part, sph.density_out(d), sph.force_out(f))):
        with pytest.raises(sph.SPHError) as e:
            call()
        assert e.value.code == sph.SPH_E_INVAL
    sph.sph_force_active(ctx, cells, part, sph.density_out(d), act, sph.force_out(f))
