"""The symmetric force (SPH_FLAG_SYMMETRIC: each pair within reach evaluated
once, the partner's side grouped by receiver and added in source order)
against the FP64 oracle, against the gather form, and bitwise equal alone and
in a pool."""
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


def _sym():
    from paper_2305_13380_gb300 import sph
    return sph.SPH_FLAG_SYMMETRIC


def test_symmetric_lattice_4096(orc):
    p = inputs.lattice(16, sigma_v=0.1)
    q = as_f32(p)
    g = run_gpu(p, count_pairs=True, extra_flags=_sym())
    od, of = orc.density_force(q, q["h0"])
    compare(g, od, of)
    # every ordered pair is counted once for each of its two particles
    assert abs(g["pairs"][1] - of["n_pairs"].sum()) <= 1e-4 * of["n_pairs"].sum()


def test_symmetric_smallest_grid(orc):
    # 3 cells per side: every cell sees all 27 cells
    p = inputs.lattice(8, seed=7, sigma_v=0.05)
    q = as_f32(p)
    g = run_gpu(p, extra_flags=_sym())
    od, of = orc.density_force(q, q["h0"])
    compare(g, od, of)


def test_symmetric_clustered_with_overflowing_blocks(orc):
    # h over two decades on one uniform grid: dense blocks exceed the
    # staging buffer and take the in-place path over global memory
    p = inputs.clustered(6000, n_spheres=4, seed=9)
    q = as_f32(p)
    g = run_gpu(p, extra_flags=_sym())
    od, of = orc.density_force(q, q["h0"])
    from paper_2305_13380_gb300 import sph
    cell = p["L"] / sph.sph_cells_sync(g["_ctx"], g["_cells"])
    vmax = float(np.sqrt(q["vx"] ** 2 + q["vy"] ** 2 + q["vz"] ** 2).max())
    compare(g, od, of, cell=cell, vmax=vmax)


def test_symmetric_matches_gather_form(orc):
    p = inputs.lattice(20, seed=4, sigma_v=0.2)
    g0 = run_gpu(p)
    g1 = run_gpu(p, extra_flags=_sym())
    for k in ("h", "rho"):
        assert np.array_equal(g0[k], g1[k]), k       # the density is the same
    a0 = np.stack([g0[k] for k in ("ax", "ay", "az")], 1)
    a1 = np.stack([g1[k] for k in ("ax", "ay", "az")], 1)
    rms = np.sqrt(np.mean(np.sum(a0 ** 2, 1)))
    assert np.abs(a1 - a0).max() < 1e-5 * rms
    assert np.abs(g1["du_dt"] - g0["du_dt"]).max() < 1e-5 * np.sqrt(np.mean(g0["du_dt"] ** 2))
    assert np.allclose(g1["v_sig"], g0["v_sig"], rtol=1e-6)
    # one evaluation per pair: the momentum sum is antisymmetric up to the
    # FP32 rounding of the shared pair term
    m = np.asarray(p["m"], np.float64)
    P1 = (m[:, None] * a1.astype(np.float64)).sum(0)
    P0 = (m[:, None] * a0.astype(np.float64)).sum(0)
    scale = (m * np.sqrt((a0.astype(np.float64) ** 2).sum(1))).sum()
    assert np.all(np.abs(P1) <= np.abs(P0) + 1e-6 * scale)


def test_symmetric_step_pool_equals_alone(orc):
    """Each simulation's step is bitwise the same alone and inside a pool."""
    import torch
    from test_gpu_step import _oracle_state, _pool
    from paper_2305_13380_gb300 import sph
    sims = [inputs.lattice(10, seed=11), inputs.lattice(13, seed=12, sigma_v=0.1),
            inputs.two_spheres(5, n_max=4e3)]
    states = [_oracle_state(orc, p) for p in sims]
    off, box, arr = _pool(states)
    prm = lambda: sph.sph_default_params(flags=sph.SPH_FLAG_SYNC | sph.SPH_FLAG_SYMMETRIC)  # noqa: E731
    ctx = sph.Context(prm())
    for _ in range(3):
        sph.sph_step(ctx, sph.pool(off, box, arr))
    assert sph.sph_status(ctx) == 0
    mixed = {k: v.cpu().numpy() for k, v in arr.items()}
    offs = off.cpu().numpy()
    for i, st in enumerate(states):
        o1, b1, a1 = _pool([st])
        c1 = sph.Context(prm())
        for _ in range(3):
            sph.sph_step(c1, sph.pool(o1, b1, a1))
        alone = {k: v.cpu().numpy() for k, v in a1.items()}
        sl = slice(offs[i], offs[i + 1])
        for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "ax", "ay", "az", "du_dt", "v_sig"):
            assert np.array_equal(mixed[k][sl], alone[k]), (i, k)
    torch.cuda.synchronize()


def test_symmetric_step_matches_oracle(orc):
    from test_gpu_step import _oracle_state, _pool
    from paper_2305_13380_gb300 import sph
    p = inputs.lattice(12, seed=3, sigma_v=0.05)
    s = _oracle_state(orc, p)
    off, box, arr = _pool([s])
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC | sph.SPH_FLAG_SYMMETRIC))
    sph.sph_step(ctx, sph.pool(off, box, arr))
    orc.step(s, 0.1)
    g = {k: v.cpu().numpy() for k, v in arr.items()}
    arms = np.sqrt(np.mean(s["ax"] ** 2 + s["ay"] ** 2 + s["az"] ** 2))
    for k in ("ax", "ay", "az"):
        assert np.abs(g[k] - s[k]).max() < 1e-4 * arms
    assert np.allclose(g["rho"], s["rho"], rtol=1e-5)
