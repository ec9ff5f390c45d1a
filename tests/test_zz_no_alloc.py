"""The allocation-free cell build (sph_build_cells_static).

Callers that cannot allocate device memory (code inside another framework's
memory arena, loops whose allocator must not synchronise, plugins that are only
handed buffers) use this entry point; its scratch is a fixed array inside the
library.  It must give exactly the cell lists of sph_build_cells, and a second
call must not see anything left over from the first.  This file is collected
last on purpose."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

pytestmark = pytest.mark.gpu


def _reference(p, margin):
    import torch
    from paper_2305_13380_gb300 import sph
    ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), cell_margin=margin))
    t = sph.to_device(p)
    cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], t["h0"])
    cs, perm = sph.sph_cells_copy(ctx, cells)
    torch.cuda.synchronize()
    return cells.n_c, cs, perm


def _static(p, margin):
    import torch
    from paper_2305_13380_gb300 import build, sph
    build.build()
    t = sph.to_device(p)
    n = t["x"].shape[0]
    cell_start = torch.full((8 * n + 217,), -7, dtype=torch.int32, device="cuda")
    perm = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    nc = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    sph.sph_build_cells_static(t["x"], t["y"], t["z"], t["h0"], float(p["L"]), margin, cell_start,
                               perm, nc, status)
    torch.cuda.synchronize()
    k = int(nc.item())
    return k, cell_start[:k ** 3 + 1].cpu().numpy(), perm.cpu().numpy(), int(status.item())


def test_static_build_matches_and_repeats():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    # two calls in a row with different sizes and grids: the second must not
    # see the first one's counts
    for p, margin in ((inputs.lattice(24, seed=5), 0.05), (inputs.clustered(9000, 5, seed=8), 0.1)):
        nc, cs, perm, st = _static(p, margin)
        rnc, rcs, rperm = _reference(p, margin)
        assert st == 0
        assert nc == rnc
        assert np.array_equal(cs, rcs)
        assert np.array_equal(perm, rperm)


def test_static_build_rejects_oversize():
    import torch
    from paper_2305_13380_gb300 import sph
    n = sph.STATIC_MAX_N + 1
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    h = torch.ones(n, dtype=torch.float32, device="cuda")
    cs = torch.zeros(8 * n + 217, dtype=torch.int32, device="cuda")
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(sph.SPHError) as e:
        sph.sph_build_cells_static(x, x, x, h, 1.0, 0.05, cs, perm)
    assert e.value.code == sph.SPH_E_CAPACITY
    small = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(sph.SPHError) as e:
        sph.sph_build_cells_static(x[:100], x[:100], x[:100], h[:100], 1.0, 0.05, small, perm[:100])
    assert e.value.code == sph.SPH_E_INVAL


def test_static_build_at_capacity_and_empty():
    """n = STATIC_MAX_N fills every part of the fixed array (keys, slots, counts
    of 8 n + 216 cells, scan partials, histograms): an off-by-one in the layout
    would corrupt the next part.  n = 0 writes an empty grid."""
    import torch
    from paper_2305_13380_gb300 import sph
    p = inputs.clustered(sph.STATIC_MAX_N, 7, seed=12)
    assert len(p["x"]) == sph.STATIC_MAX_N
    for margin in (0.05, 0.0):
        nc, cs, perm, st = _static(p, margin)
        rnc, rcs, rperm = _reference(p, margin)
        assert st == 0 and nc == rnc
        assert np.array_equal(cs, rcs) and np.array_equal(perm, rperm)
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    he = torch.zeros(0, dtype=torch.float32, device="cuda")
    cs = torch.full((217,), -7, dtype=torch.int32, device="cuda")
    perm = torch.zeros(0, dtype=torch.int32, device="cuda")
    nc = torch.zeros(1, dtype=torch.int32, device="cuda")
    sph.sph_build_cells_static(e, e, e, he, 1.0, 0.05, cs, perm, nc)
    torch.cuda.synchronize()
    k = int(nc.item())
    assert 3 <= k <= 6
    assert np.all(cs[:k ** 3 + 1].cpu().numpy() == 0)
