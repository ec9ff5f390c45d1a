"""Friends-of-friends groups on the GPU (sph_fof, Sec. 7.1) against the
FP64 oracle: the labels (smallest index of each group) are integers decided
by the FP64 predicate on both sides, so they must be equal bit for bit."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


def _gpu_fof(x, y, z, L, b, sync=True):
    import torch
    from paper_2305_13380_gb300 import sph
    ctx = sph.Context(sph.sph_default_params(box_size=float(L),
                                             flags=sph.SPH_FLAG_SYNC if sync else 0))
    t = [torch.as_tensor(np.asarray(v, dtype=np.float64), device="cuda") for v in (x, y, z)]
    g = sph.sph_fof(ctx, *t, b)
    torch.cuda.synchronize()
    out = g.cpu().numpy()
    ctx.close()
    return out


def _xyz(p):
    return tuple(np.asarray(p[k], dtype=np.float64) for k in "xyz")


CASES = {
    # uniform random points, b = 0.6 of the mean spacing: many small groups
    "uniform": lambda: (dict(zip("xyz", np.random.default_rng(3).random((3, 20000)))), 1.0,
                        0.6 * 20000 ** (-1 / 3)),
    # the clustered recipe with b = 0.2 of the mean spacing (the usual choice)
    "clustered6000": lambda: (inputs.clustered(6000, n_spheres=4, seed=9), 1.0, 0.2 * 6000 ** (-1 / 3)),
    "clustered20000": lambda: (inputs.clustered(20000, n_spheres=64, seed=1), 1.0, 0.2 * 20000 ** (-1 / 3)),
    # a jittered lattice with b at the spacing: pairs at the linking length,
    # where the FP32 distance cannot decide and the FP64 test does
    "lattice_edge": lambda: (inputs.lattice(20, seed=4), 1.0, 1.0 / 20),
    # b = L/3: three cells per side, every cell's neighbours wrap
    "three_cells": lambda: (inputs.clustered(3000, n_spheres=3, seed=5), 1.0, 1.0 / 3),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fof_equals_oracle(orc, case):
    p, L, b = CASES[case]()
    x, y, z = _xyz(p)
    got = _gpu_fof(x, y, z, L, b)
    ref = orc.fof(x, y, z, L, b)
    assert np.array_equal(got, ref)


def test_fof_periodic_and_tiny_inputs(orc):
    x = np.array([0.995, 0.5, 0.005, 0.5005])
    y = np.array([0.5, 0.5, 0.5, 0.5])
    z = np.array([0.5, 0.5, 0.5, 0.5])
    assert _gpu_fof(x, y, z, 1.0, 0.02).tolist() == [0, 1, 0, 1]
    assert _gpu_fof(x[:1], y[:1], z[:1], 1.0, 0.02).tolist() == [0]
    # a box of side 3: positions and b scale together
    assert _gpu_fof(3 * x, 3 * y, 3 * z, 3.0, 0.06).tolist() == [0, 1, 0, 1]


def test_fof_async_and_repeated_calls(orc):
    # without SPH_FLAG_SYNC, and twice on one context: the second call
    # rebuilds the cells and starts from singletons again
    import torch
    from paper_2305_13380_gb300 import sph
    p = inputs.clustered(6000, n_spheres=4, seed=9)
    x, y, z = _xyz(p)
    ctx = sph.Context(sph.sph_default_params(box_size=1.0))
    t = [torch.as_tensor(v, device="cuda") for v in (x, y, z)]
    b = 0.2 * 6000 ** (-1 / 3)
    g1 = sph.sph_fof(ctx, *t, b).cpu().numpy()
    g2 = sph.sph_fof(ctx, *t, 2 * b).cpu().numpy()
    torch.cuda.synchronize()
    assert sph.sph_status(ctx) == 0
    assert np.array_equal(g1, orc.fof(x, y, z, 1.0, b))
    assert np.array_equal(g2, orc.fof(x, y, z, 1.0, 2 * b))


def test_fof_rejects_bad_linking_lengths():
    import torch
    from paper_2305_13380_gb300 import sph
    ctx = sph.Context(sph.sph_default_params(box_size=1.0))
    t = [torch.zeros(4, dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(sph.SPHError) as e:
        sph.sph_fof(ctx, *t, 0.4)
    assert e.value.code == sph.SPH_E_BOX
    with pytest.raises(sph.SPHError) as e:
        sph.sph_fof(ctx, *t, 0.0)
    assert e.value.code == sph.SPH_E_INVAL


def test_fof_full_size_clustered_2M(orc):
    # the benchmark's workload: 2^21 particles in 64 Plummer spheres plus the
    # background, b = 0.2 of the mean spacing, every label against the oracle
    p = inputs.clustered(1 << 21, n_spheres=64, seed=0)
    x, y, z = _xyz(p)
    b = 0.2 * (1 << 21) ** (-1 / 3)
    got = _gpu_fof(x, y, z, 1.0, b)
    ref = orc.fof(x, y, z, 1.0, b)
    assert np.array_equal(got, ref)
