"""Sub-steps of the time-step hierarchy (sph_hier_substep) on the GPU against
the oracle's: fixed bins over several sub-steps, and adaptive bins, on the
uniform grid and on the nested grids."""
import numpy as np
import pytest

from gpu_common import as_f32

from paper_2305_13380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


def _state(orc, seed, u_spread=False):
    p = inputs.lattice(12, seed=seed, sigma_v=0.05)
    if u_spread:
        # sound speeds over a decade: CFL steps over several bins
        p["u"] = 10.0 ** np.random.default_rng(seed).uniform(-1.0, 1.0, len(p["x"]))
    q = as_f32(p)
    d, f = orc.density_force(q, q["h0"])
    s = {k: q[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u")}
    s.update(L=float(p["L"]), h=d["h"].copy(), ax=f["ax"].copy(), ay=f["ay"].copy(), az=f["az"].copy(),
             du_dt=f["du_dt"].copy(), v_sig=f["v_sig"].copy())
    for k in ("rho", "f", "P", "c", "B", "div_v"):
        s[k] = d[k].copy()
    return s


def _start(s, bins, dt_max, max_bin):
    """Half kicks of the first steps, in FP32 as the GPU holds them."""
    dt_i = np.ldexp(dt_max, -max_bin) * 2.0 ** (max_bin - bins)
    for k in ("x", "y", "z"):
        s["v" + k] = (s["v" + k] + s["a" + k] * 0.5 * dt_i).astype(np.float32).astype(np.float64)
    s["u"] = (s["u"] + s["du_dt"] * 0.5 * dt_i).astype(np.float32).astype(np.float64)


def _pool(s):
    import torch
    from paper_2305_13380_gb300 import sph
    dev = "cuda"
    arr = {k: torch.tensor(s[k], dtype=torch.float64, device=dev) for k in ("x", "y", "z")}
    for k in ("vx", "vy", "vz", "u", "m", "h", "ax", "ay", "az", "du_dt", "v_sig", "rho", "f", "div_v", "P", "c"):
        arr[k] = torch.tensor(s[k], dtype=torch.float32, device=dev)
    arr["balsara"] = torch.tensor(s["B"], dtype=torch.float32, device=dev)
    arr["curl_v"] = torch.zeros_like(arr["h"])
    arr["dt"] = torch.zeros(1, dtype=torch.float64, device=dev)
    n = len(s["x"])
    off = torch.tensor([0, n], dtype=torch.int64, device=dev)
    box = torch.tensor([s["L"]], dtype=torch.float64, device=dev)
    return arr, sph.pool(off, box, arr)


def _compare(g, s, d, predict=False):
    if predict:
        # predicted (inactive) and re-evaluated (active) densities alike
        for k in ("rho", "P", "c"):
            assert np.allclose(g[k], s[k], rtol=1e-5), k
    for k in ("x", "y", "z"):
        diff = np.abs(g[k] - s[k])
        assert np.minimum(diff, 1.0 - diff).max() < 1e-6 * d, k
    vs = np.sqrt(np.mean(s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2))
    for k in ("vx", "vy", "vz"):
        assert np.abs(g[k] - s[k]).max() < 1e-4 * vs, k
    assert np.allclose(g["u"], s["u"], rtol=1e-5)
    assert np.allclose(g["h"], s["h"], rtol=1e-5)


def _flags(grid):
    from paper_2305_13380_gb300 import sph
    return sph.SPH_FLAG_TREE if grid == "nested" else 0


@pytest.mark.parametrize("predict,keep,grid", [(False, False, "uniform"), (True, False, "uniform"),
                                               (True, True, "uniform"), (False, False, "nested"),
                                               (True, False, "nested")])
def test_fixed_bins_over_four_substeps(orc, predict, keep, grid):
    import torch
    from paper_2305_13380_gb300 import sph
    s = _state(orc, 3)
    n = len(s["x"])
    max_bin = 2
    dt_max = 4.0 * float(np.min(0.1 * orc.GAMMA_K * s["h"] / s["v_sig"]))
    rng = np.random.default_rng(2)
    bins = rng.integers(0, max_bin + 1, n).astype(np.int32)
    _start(s, bins, dt_max, max_bin)
    arr, pool = _pool(s)
    gb = torch.tensor(bins, device="cuda")
    gt = torch.zeros(n, dtype=torch.int64, device="cuda")
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC | sph.SPH_FLAG_TIMING | _flags(grid)))
    tb = np.zeros(n, np.int64)
    t = tg = 0
    calls = 0
    while t < 4:
        tg = sph.sph_hier_substep(ctx, pool, gb, gt, dt_max, max_bin, tg, adapt=False, predict=predict,
                                  keep_cells=keep)
        t = orc.hier_substep(s, bins, tb, dt_max, max_bin, t, False, predict=predict)
        assert tg == t
        calls += 1
    assert np.array_equal(gt.cpu().numpy(), tb) and np.array_equal(gb.cpu().numpy(), bins)
    g = {k: v.cpu().numpy() for k, v in arr.items()}
    _compare(g, s, 1.0 / 12, predict)
    builds = sph.sph_kernel_times(ctx)["build"][1]
    # kept cells: the first sub-step builds, later ones keep its cells while
    # the drift leaves room in them
    assert (builds < calls) if keep else (builds == calls)


@pytest.mark.parametrize("predict,keep,grid", [(False, False, "uniform"), (True, False, "uniform"),
                                               (True, True, "uniform"), (False, False, "nested"),
                                               (True, False, "nested")])
def test_adaptive_bins(orc, predict, keep, grid):
    import torch
    from paper_2305_13380_gb300 import sph
    s = _state(orc, 5, u_spread=True)
    n = len(s["x"])
    max_bin = 4
    dt_max = 16.0 * float(np.min(0.1 * orc.GAMMA_K * s["h"] / s["v_sig"]))
    bins = orc.limit_time_bins(s, s["h"], orc.time_bins(s["h"], s["v_sig"], 0.1, dt_max, max_bin))
    _start(s, bins, dt_max, max_bin)
    arr, pool = _pool(s)
    gb = torch.tensor(bins, device="cuda")
    gt = torch.zeros(n, dtype=torch.int64, device="cuda")
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC | _flags(grid)))
    tb = np.zeros(n, np.int64)
    t = tg = 0
    for _ in range(3):
        tg = sph.sph_hier_substep(ctx, pool, gb, gt, dt_max, max_bin, tg, adapt=True, predict=predict,
                                  keep_cells=keep)
        t = orc.hier_substep(s, bins, tb, dt_max, max_bin, t, True, predict=predict)
        assert tg == t
        g_bins, g_tb = gb.cpu().numpy(), gt.cpu().numpy()
        # every step starts on a multiple of its length, and the tick is an end
        assert np.all(g_tb % (1 << (max_bin - g_bins)) == 0)
        assert np.mean(g_bins == bins) > 0.99
    assert len(np.unique(bins)) > 1   # at least two levels of the hierarchy
    if np.array_equal(gb.cpu().numpy(), bins):
        g = {k: v.cpu().numpy() for k, v in arr.items()}
        _compare(g, s, 1.0 / 12, predict)


def _heated(orc, seed, heat):
    """A lattice box on bins 2 and 3 (64- and 32-tick steps of max_bin 8) in
    which particle f is heated in the middle of its step (u x heat^2 and its
    signal speed x heat, as a source term would leave it) and flagged."""
    s = _state(orc, seed)
    n = len(s["x"])
    max_bin = 8
    dt_max = 3.0 * float(np.min(0.1 * orc.GAMMA_K * s["h"] / s["v_sig"]))
    bins = np.full(n, 2, np.int32)
    bins[::7] = 3
    _start(s, bins, dt_max, max_bin)
    f = 1
    s["u"][f] = float(np.float32(s["u"][f] * heat * heat))
    s["v_sig"][f] = float(np.float32(s["v_sig"][f] * heat))
    return s, bins, dt_max, max_bin, f


@pytest.mark.parametrize("adapt,grid", [(False, "uniform"), (True, "uniform"), (True, "nested")])
def test_sync_and_wakeup(orc, adapt, grid):
    """The synchronisation step and the wake-up limiter (Sec. 3.4) against the
    oracle over five sub-steps: the flagged particle ends its step at the
    first tick, and (adapt) its deep bin wakes its neighbours at its next end;
    without adapt the bins stay fixed and only the synchronisation acts (a
    mild heating, which the fixed steps can carry)."""
    import torch
    from paper_2305_13380_gb300 import sph
    s, bins, dt_max, max_bin, f = _heated(orc, 6, 10.0 if adapt else 1.2)
    n = len(s["x"])
    arr, pool = _pool(s)
    gb = torch.tensor(bins, device="cuda")
    gt = torch.zeros(n, dtype=torch.int64, device="cuda")
    sync_g = torch.zeros(n, dtype=torch.uint8, device="cuda")
    sync_g[f] = 1
    sync_o = np.zeros(n, bool)
    sync_o[f] = True
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC | _flags(grid)))
    tb = np.zeros(n, np.int64)
    t = tg = 0
    exact, woken = True, 0
    for k in range(5):
        end = tb + (1 << (max_bin - bins))
        tg = sph.sph_hier_substep(ctx, pool, gb, gt, dt_max, max_bin, tg, adapt=adapt, wakeup=True,
                                  sync=sync_g if k == 0 else None)
        t = orc.hier_substep(s, bins, tb, dt_max, max_bin, t, adapt, wakeup=True,
                             sync=sync_o if k == 0 else None)
        assert tg == t
        g_bins, g_tb = gb.cpu().numpy(), gt.cpu().numpy()
        assert np.all(g_tb % (1 << (max_bin - g_bins)) == 0)
        if k == 0:
            assert int(sync_g.sum()) == 0 and t == 32 and g_tb[f] == 32
            assert g_bins[f] == bins[f] and bins[f] >= (5 if adapt else 3)
        else:
            woken += int(np.count_nonzero((end != t) & (tb == t)))
        assert np.mean((g_bins == bins) & (g_tb == tb)) > 0.995
        if not (np.array_equal(g_bins, bins) and np.array_equal(g_tb, tb)):
            exact = False   # a CFL bin at an edge: the two timelines part
            break
    if adapt:
        assert woken > 20
    if exact:
        g = {k: v.cpu().numpy() for k, v in arr.items()}
        _compare(g, s, 1.0 / 12)


def test_kept_cells_across_the_periodic_boundary(orc):
    """Cells kept across sub-steps under a bulk flow along x: particles drift
    out of the cells they are filed in and across the periodic boundary
    (taken at the image nearest their cell), and the sub-steps still match the
    oracle's; the cells are rebuilt once the drift bound uses up the margin."""
    import torch
    from paper_2305_13380_gb300 import sph
    s = _state(orc, 7)
    s["vx"] = s["vx"] + 1.0          # Galilean: the same forces, a drift across x = L
    n = len(s["x"])
    max_bin = 1
    dt_max = 2.0 * float(np.min(0.1 * orc.GAMMA_K * s["h"] / s["v_sig"]))
    bins = np.where(np.arange(n) % 2 == 0, 1, 0).astype(np.int32)
    _start(s, bins, dt_max, max_bin)
    arr, pool = _pool(s)
    gb = torch.tensor(bins, device="cuda")
    gt = torch.zeros(n, dtype=torch.int64, device="cuda")
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC | sph.SPH_FLAG_TIMING, cell_margin=0.2))
    tb = np.zeros(n, np.int64)
    x0 = s["x"].copy()
    t = tg = 0
    calls = 0
    while t < 8:
        tg = sph.sph_hier_substep(ctx, pool, gb, gt, dt_max, max_bin, tg, adapt=False, keep_cells=True)
        t = orc.hier_substep(s, bins, tb, dt_max, max_bin, t, False)
        assert tg == t
        calls += 1
    builds = sph.sph_kernel_times(ctx)["build"][1]
    assert 1 <= builds < calls
    assert np.count_nonzero(s["x"] < x0 - 0.5) > 20     # wrapped across x = L
    assert np.array_equal(gt.cpu().numpy(), tb) and np.array_equal(gb.cpu().numpy(), bins)
    g = {k: v.cpu().numpy() for k, v in arr.items()}
    _compare(g, s, 1.0 / 12)


@pytest.mark.parametrize("grid", ["uniform", "nested"])
def test_graph_replayed_substeps_equal_the_host_calls(orc, grid):
    """sph_hier_substep_dev captured once in a CUDA graph and replayed: each
    replay one sub-step, the tick advanced on the device; five replays equal
    five host calls on an identical pool bit for bit (adaptive bins, wake-up
    and prediction on)."""
    import torch
    from paper_2305_13380_gb300 import sph
    s = _state(orc, 5, u_spread=True)
    n = len(s["x"])
    max_bin = 4
    dt_max = 16.0 * float(np.min(0.1 * orc.GAMMA_K * s["h"] / s["v_sig"]))
    bins = orc.limit_time_bins(s, s["h"], orc.time_bins(s["h"], s["v_sig"], 0.1, dt_max, max_bin))
    _start(s, bins, dt_max, max_bin)
    arr_a, pool_a = _pool(s)
    arr_b, pool_b = _pool(s)
    gb_a, gb_b = torch.tensor(bins, device="cuda"), torch.tensor(bins, device="cuda")
    gt_a, gt_b = torch.zeros(n, dtype=torch.int64, device="cuda"), torch.zeros(n, dtype=torch.int64, device="cuda")
    st = torch.cuda.Stream()
    ctx_a = sph.Context(sph.sph_default_params(flags=_flags(grid)), st)
    ctx_b = sph.Context(sph.sph_default_params(flags=_flags(grid)), st)
    tick = torch.zeros(1, dtype=torch.int64, device="cuda")
    kw = dict(adapt=True, wakeup=True, predict=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        t_a = sph.sph_hier_substep(ctx_a, pool_a, gb_a, gt_a, dt_max, max_bin, 0, **kw)
        sph.sph_hier_substep_dev(ctx_b, pool_b, gb_b, gt_b, dt_max, max_bin, tick, **kw)   # allocates
    st.synchronize()
    assert int(tick.item()) == t_a
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        sph.sph_hier_substep_dev(ctx_b, pool_b, gb_b, gt_b, dt_max, max_bin, tick, **kw)
    st.synchronize()
    assert int(tick.item()) == t_a          # capturing ran nothing
    ticks = []
    for _ in range(5):
        with torch.cuda.stream(st):
            t_a = sph.sph_hier_substep(ctx_a, pool_a, gb_a, gt_a, dt_max, max_bin, t_a, **kw)
            g.replay()
        st.synchronize()
        ticks.append(t_a)
        assert int(tick.item()) == t_a
    assert len(set(ticks)) == 5
    assert torch.equal(gb_a, gb_b) and torch.equal(gt_a, gt_b)
    for k in arr_a:
        assert torch.equal(arr_a[k], arr_b[k]), k


def test_kept_cells_refused_on_the_nested_grids(orc):
    """Kept cells are cells of the uniform grid: the option is refused on the
    nested grids (which rebuild every sub-step)."""
    import torch
    from paper_2305_13380_gb300 import sph
    s = _state(orc, 3)
    n = len(s["x"])
    bins = np.zeros(n, np.int32)
    arr, pool = _pool(s)
    gb = torch.tensor(bins, device="cuda")
    gt = torch.zeros(n, dtype=torch.int64, device="cuda")
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC | sph.SPH_FLAG_TREE))
    with pytest.raises(sph.SPHError) as e:
        sph.sph_hier_substep(ctx, pool, gb, gt, 1e-3, 2, 0, adapt=False, keep_cells=True)
    assert e.value.code == sph.SPH_E_INVAL
