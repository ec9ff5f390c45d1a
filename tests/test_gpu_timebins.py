"""Time bins and the first time-step limiter (sph_time_bins) on the GPU
against the oracle: the CFL bins bit for bit (both decide in FP32), the
limited bins within the bins that the force-pair set with its radius moved by
1e-5 gives (pairs at the edge of max(H_i, H_j) may fall either way)."""
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


def test_uniform_speed_gives_one_bin(orc):
    p, h, v = _case(1, lambda r, n: np.full(n, 3.0))
    g = _gpu_bins(p, h, v)
    b0 = orc.time_bins(h, v, CFL, DT_MAX, MAX_BIN)
    assert np.array_equal(g, orc.limit_time_bins(p, h, b0))
    assert len(np.unique(b0)) <= 2


@pytest.mark.parametrize("seed", [2, 3])
def test_random_speeds_and_the_limiter(orc, seed):
    p, h, v = _case(seed, lambda r, n: np.exp(r.uniform(np.log(0.5), np.log(500.0), n)))
    g = _gpu_bins(p, h, v)
    b0 = orc.time_bins(h, v, CFL, DT_MAX, MAX_BIN)
    lo = orc.limit_time_bins(p, h, b0, scale=1 - 1e-5)
    hi = orc.limit_time_bins(p, h, b0, scale=1 + 1e-5)
    assert np.all(g >= lo) and np.all(g <= hi)
    assert np.mean(g == orc.limit_time_bins(p, h, b0)) > 0.99
    assert np.all(g >= b0) and np.sum(g > b0) > 50   # the limiter acted


def test_one_fast_particle_raises_its_neighbours(orc):
    p, h, v = _case(4, lambda r, n: np.full(n, 1.0))
    v[17] = 1e4
    g = _gpu_bins(p, h, v)
    b0 = orc.time_bins(h, v, CFL, DT_MAX, MAX_BIN)
    assert np.array_equal(g, orc.limit_time_bins(p, h, b0))
    assert g[17] == b0[17] and (g == b0[17] - 2).sum() > 30


def test_resting_particles_take_the_longest_bin(orc):
    p, h, v = _case(5, lambda r, n: np.zeros(n))
    assert np.all(_gpu_bins(p, h, v) == 0)
