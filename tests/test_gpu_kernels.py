"""The quartic spline and the Wendland C2 kernel (Sec. 3.1) on the GPU against
the oracle: density and force on lattice and clustered inputs, and a step,
with the kernel selected per context, on the uniform and the nested
grids."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

from gpu_common import as_f32, compare, run_gpu

pytestmark = pytest.mark.gpu

KERNELS = [(1, "quartic"), (2, "wendland_c2")]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


@pytest.mark.parametrize("k,name", KERNELS)
def test_density_force_lattice(orc, k, name):
    p = inputs.lattice(16, seed=11, sigma_v=0.05)
    q = as_f32(p)
    g = run_gpu(p, count_pairs=True, kernel=k)
    od, of = orc.density_force(q, q["h0"], orc.Physics(kernel=k))
    compare(g, od, of)
    # the neighbour count follows the kernel's support (pairs within rounding
    # of q = 1 may fall either way)
    assert abs(g["pairs"][0] - int(od["n_ngb"].sum())) <= 1e-5 * od["n_ngb"].sum()


@pytest.mark.parametrize("k,name", KERNELS)
def test_density_force_clustered(orc, k, name):
    p = inputs.clustered(6000, n_spheres=4, seed=9, a_min=0.03, a_max=0.06)
    q = as_f32(p)
    g = run_gpu(p, kernel=k)
    od, of = orc.density_force(q, q["h0"], orc.Physics(kernel=k))
    compare(g, od, of)


@pytest.mark.parametrize("k,name", KERNELS)
def test_step(orc, k, name):
    from paper_2305_13380_gb300 import sph
    from test_gpu_step import _pool
    phys = orc.Physics(kernel=k)
    p = inputs.lattice(12, seed=3, sigma_v=0.05)
    q = as_f32(p)
    d, f = orc.density_force(q, q["h0"], phys)
    s = {kk: q[kk].copy() for kk in ("x", "y", "z", "vx", "vy", "vz", "m", "u")}
    s.update(L=p["L"], h=d["h"].copy(), ax=f["ax"].copy(), ay=f["ay"].copy(), az=f["az"].copy(),
             du_dt=f["du_dt"].copy(), v_sig=f["v_sig"].copy())
    off, box, arr = _pool([s])
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC, kernel=k))
    sph.sph_step(ctx, sph.pool(off, box, arr))
    dt = orc.step(s, 0.1, phys)
    assert float(arr["dt"].cpu()[0]) == pytest.approx(dt, rel=1e-6)
    g = {kk: v.cpu().numpy() for kk, v in arr.items()}
    for kk in ("x", "y", "z"):
        diff = np.abs(g[kk] - s[kk])
        assert np.minimum(diff, 1.0 - diff).max() < 1e-6 / 12
    assert np.allclose(g["h"], s["h"], rtol=1e-5)
    assert np.allclose(g["rho"], s["rho"], rtol=1e-5)
    arms = np.sqrt(np.mean(s["ax"] ** 2 + s["ay"] ** 2 + s["az"] ** 2))
    for kk in ("ax", "ay", "az"):
        assert np.abs(g[kk] - s[kk]).max() < 1e-4 * arms


@pytest.mark.parametrize("k,name", KERNELS)
def test_nested_grids(orc, k, name):
    # clustered gas on the nested grids: the plain bounds, no precision floor
    p = inputs.clustered(6000, n_spheres=8, seed=5)
    q = as_f32(p)
    g = run_gpu(p, tree=True, kernel=k)
    od, of = orc.density_force(q, q["h0"], orc.Physics(kernel=k))
    compare(g, od, of)


@pytest.mark.parametrize("k,name", KERNELS)
def test_nested_grids_strongly_clustered(orc, k, name):
    # the densest configuration of the clustered workload (64 spheres)
    p = inputs.clustered(20000, n_spheres=64, seed=1)
    q = as_f32(p)
    g = run_gpu(p, tree=True, kernel=k)
    od, of = orc.density_force(q, q["h0"], orc.Physics(kernel=k))
    assert od["h"].max() / od["h"].min() > 50
    compare(g, od, of)


def test_unknown_kernel_rejected():
    from paper_2305_13380_gb300 import sph
    with pytest.raises(sph.SPHError) as e:
        sph.Context(sph.sph_default_params(kernel=3))
    assert e.value.code == sph.SPH_E_INVAL
