"""Time bins and the first time-step limiter (sph_time_bins) on the GPU
against the oracle.  The oracle decides the CFL bins in FP64 (the definition),
the kernel in FP32: they agree except where the CFL step lies within 1e-6 of a
bin boundary (a few FP32 roundings), where the kernel's bin may be one off.
The limited bins lie within what the oracle's limiter gives with those edge
bins moved either way and the force-pair radius moved by 1e-5 (pairs at the
edge of max(H_i, H_j) may fall either way), and equal the oracle's almost
everywhere."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

pytestmark = pytest.mark.gpu

CFL, DT_MAX, MAX_BIN = 0.1, 1.0, 30


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


def _gpu_bins(p, h, v):
    import torch
    from paper_2305_13380_gb300 import sph
    ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), flags=sph.SPH_FLAG_SYNC))
    t = sph.to_device(p)
    n = int(t["x"].shape[0])
    hd = torch.tensor(h, dtype=torch.float32, device="cuda")
    cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], hd)
    d = sph.alloc_density(n)
    d["h"].copy_(hd)
    for k in ("rho", "f", "P", "c", "balsara"):
        d[k].fill_(1.0)
    bins = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    sph.sph_time_bins(ctx, cells, sph.particles(t), sph.density_out(d),
                      torch.tensor(v, dtype=torch.float32, device="cuda"), CFL, DT_MAX, MAX_BIN, bins)
    return bins.cpu().numpy()


def _case(seed, v):
    p = inputs.lattice(12, seed=seed, sigma_v=0.05)
    rng = np.random.default_rng(seed)
    h = (np.asarray(p["h0"]) * rng.uniform(0.9, 1.1, len(p["x"]))).astype(np.float32)
    return p, h, np.asarray(v(rng, len(p["x"])), dtype=np.float32)


def _bounds(orc, p, h, v):
    b0 = orc.time_bins(h, v, CFL, DT_MAX, MAX_BIN)
    edge = orc.bin_edge_band(h, v, CFL, DT_MAX, MAX_BIN).astype(np.int32)
    lo = orc.limit_time_bins(p, h, np.maximum(b0 - edge, 0), scale=1 - 1e-5)
    hi = orc.limit_time_bins(p, h, np.minimum(b0 + edge, MAX_BIN), scale=1 + 1e-5)
    return b0, edge, lo, hi


def test_uniform_speed_gives_one_bin(orc):
    p, h, v = _case(1, lambda r, n: np.full(n, 3.0))
    g = _gpu_bins(p, h, v)
    b0, edge, lo, hi = _bounds(orc, p, h, v)
    assert np.all(g >= lo) and np.all(g <= hi)
    if not edge.any():
        assert np.array_equal(g, orc.limit_time_bins(p, h, b0))
    assert len(np.unique(b0)) <= 2


@pytest.mark.parametrize("seed", [2, 3])
def test_random_speeds_and_the_limiter(orc, seed):
    p, h, v = _case(seed, lambda r, n: np.exp(r.uniform(np.log(0.5), np.log(500.0), n)))
    g = _gpu_bins(p, h, v)
    b0, edge, lo, hi = _bounds(orc, p, h, v)
    assert np.all(g >= lo) and np.all(g <= hi)
    assert np.mean(g == orc.limit_time_bins(p, h, b0)) > 0.99
    assert np.all(g >= b0) and np.sum(g > b0) > 50   # the limiter acted


def test_one_fast_particle_raises_its_neighbours(orc):
    p, h, v = _case(4, lambda r, n: np.full(n, 1.0))
    v[17] = 1e4
    g = _gpu_bins(p, h, v)
    b0, edge, lo, hi = _bounds(orc, p, h, v)
    assert np.all(g >= lo) and np.all(g <= hi)
    if not edge.any():
        assert np.array_equal(g, orc.limit_time_bins(p, h, b0))
    assert g[17] == b0[17] and (g == b0[17] - 2).sum() > 30


def test_resting_particles_take_the_longest_bin(orc):
    p, h, v = _case(5, lambda r, n: np.zeros(n))
    assert np.all(_gpu_bins(p, h, v) == 0)


def test_cfl_bins_match_the_fp64_definition_off_the_edges(orc):
    """Without neighbours in reach (particles far apart), the limiter leaves
    the CFL bins alone: the kernel's FP32 bins equal the FP64 definition except
    within the edge band, including speeds placed exactly on and next to the
    bin boundaries."""
    rng = np.random.default_rng(9)
    n_side = 4
    p = inputs.lattice(n_side, seed=9, jitter=0.0, sigma_v=0.0)
    n = len(p["x"])
    h = np.full(n, 0.05, np.float32)      # supports far below the spacing
    c = CFL * orc.GAMMA_K
    # speeds whose CFL step falls on, just above and just below boundaries
    k = rng.integers(1, 20, n)
    v = (c * 0.05 / np.ldexp(DT_MAX, -k)).astype(np.float32)
    v[::3] = np.nextafter(v[::3], np.float32(np.inf))
    v[1::3] = np.nextafter(v[1::3], np.float32(0))
    g = _gpu_bins(p, h, v)
    b0 = orc.time_bins(h, v, CFL, DT_MAX, MAX_BIN)
    edge = orc.bin_edge_band(h, v, CFL, DT_MAX, MAX_BIN)
    assert np.array_equal(g[~edge], b0[~edge])
    assert np.all(np.abs(g[edge] - b0[edge]) <= 1)
    # random speeds: almost none on an edge, all equal
    v2 = np.exp(rng.uniform(0.0, 8.0, n)).astype(np.float32)
    g2 = _gpu_bins(p, h, v2)
    b2 = orc.time_bins(h, v2, CFL, DT_MAX, MAX_BIN)
    e2 = orc.bin_edge_band(h, v2, CFL, DT_MAX, MAX_BIN)
    assert np.array_equal(g2[~e2], b2[~e2])


def _gpu_bins_nested(p, v):
    """sph_time_bins on the nested grids, after the density and force of the
    same build (the limiter walks their lists and reverse pairs); returns the
    bins and the density's h."""
    import torch
    from paper_2305_13380_gb300 import sph
    ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), flags=sph.SPH_FLAG_SYNC | sph.SPH_FLAG_TREE))
    t = sph.to_device(p)
    n = int(t["x"].shape[0])
    part = sph.particles(t)
    d, f = sph.alloc_density(n), sph.alloc_force(n)
    h_in = t["h0"]
    for _ in range(8):  # rebuild until the top cells hold every support
        cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], h_in)
        try:
            sph.sph_density(ctx, cells, part, h_in, sph.density_out(d))
            break
        except sph.SPHError as e:
            if e.code != sph.SPH_E_REBUILD:
                raise
            h_in = d["h"].clone()
    sph.sph_force(ctx, cells, part, sph.density_out(d), sph.force_out(f))
    bins = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    sph.sph_time_bins(ctx, cells, part, sph.density_out(d), torch.tensor(v, dtype=torch.float32, device="cuda"),
                      CFL, DT_MAX, MAX_BIN, bins)
    return bins.cpu().numpy()


@pytest.mark.parametrize("case", ["clustered", "fast_particle"])
def test_limiter_on_the_nested_grids(orc, case):
    """The limiter over the nested grids' force pairs (lists and reverse
    pairs) against the oracle's brute force: clustered gas whose supports span
    decades, and one fast particle raising its neighbours.  The bins are
    decided from the oracle's own h (the GPU's agrees within 1e-5), so the
    edge band and the pair radius carry that difference too (1e-4)."""
    from gpu_common import as_f32
    if case == "clustered":
        p = inputs.clustered(3000, n_spheres=3, seed=11, a_min=0.03, a_max=0.08)
    else:
        p = inputs.lattice(12, seed=4, sigma_v=0.05)
    rng = np.random.default_rng(21)
    n = len(p["x"])
    v = np.exp(rng.uniform(np.log(0.5), np.log(50.0), n)).astype(np.float32)
    if case == "fast_particle":
        v[:] = 1.0
        v[17] = 1e4
    g = _gpu_bins_nested(p, v)
    q = as_f32(p)
    h = orc.density(q, q["h0"])["h"]
    b0 = orc.time_bins(h, v, CFL, DT_MAX, MAX_BIN)
    edge = orc.bin_edge_band(h, v, CFL, DT_MAX, MAX_BIN, rel=1e-4).astype(np.int32)
    lo = orc.limit_time_bins(p, h, np.maximum(b0 - edge, 0), scale=1 - 1e-4)
    hi = orc.limit_time_bins(p, h, np.minimum(b0 + edge, MAX_BIN), scale=1 + 1e-4)
    assert np.all(g >= lo) and np.all(g <= hi)
    exact = orc.limit_time_bins(p, h, b0)
    assert np.mean(g == exact) > 0.99
    if case == "fast_particle":
        assert g[17] == b0[17] and (g == b0[17] - 2).sum() > 30
    else:
        assert np.sum(exact > b0) > 50   # the limiter acted
