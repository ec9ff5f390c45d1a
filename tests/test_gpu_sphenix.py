"""The SPHENIX flavour (Sec. 3.3) on the GPU against the oracle: the viscosity
update, the gradient pass (Laplacian of u, conduction parameter) and the
force with conduction, through the C ABI, on lattice and clustered inputs, on
the uniform grid and the nested grids; steps and pools on both; and the
reduction to the "Minimal" force."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

from gpu_common import GAMMA_K, as_f32, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


def _f32(a):
    return np.asarray(a, dtype=np.float32)


def _setup(orc, p, seed):
    """Seeded SPHENIX inputs of one evaluation.  The previous divergence is
    the oracle's divergence plus a seeded offset bounded away from zero, so
    that the rate of the divergence is set by the offset and not by the
    rounding of the divergence itself."""
    q = as_f32(p)
    od = orc.density(q, q["h0"])
    n = len(q["x"])
    rng = np.random.default_rng(seed)
    rms = np.sqrt(np.mean(od["div_v"] ** 2)) + 1e-30
    off = rng.choice([-1.0, 1.0], n) * rng.uniform(0.5, 1.5, n) * rms
    # alpha_V well below alpha_V,max keeps the conduction limiter open, so
    # that the Euler step of alpha_c is seen and not only the limits
    st = dict(alpha_v=_f32(rng.uniform(0.0, 0.5, n)), alpha_c=_f32(rng.uniform(0.0, 0.3, n)),
              div_v_prev=_f32(od["div_v"] + off),
              v_sig=_f32(od["c"] * rng.uniform(1.5, 3.0, n)))
    H = GAMMA_K * od["h"]
    dt = float(0.05 * np.min(H / st["v_sig"]))
    return q, od, st, dt


def _run_gpu(p, st, dt, tree=False):
    import torch
    from paper_2305_13380_gb300 import sph
    flags = sph.SPH_FLAG_SYNC | (sph.SPH_FLAG_TREE if tree else 0)
    ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), flags=flags))
    t = sph.to_device(p)
    n = int(t["x"].shape[0])
    part = sph.particles(t)
    d = sph.alloc_density(n)
    f = sph.alloc_force(n)
    h_in = t["h0"]
    for _ in range(8):
        cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], h_in)
        try:
            sph.sph_density(ctx, cells, part, h_in, sph.density_out(d))
            break
        except sph.SPHError as e:
            if e.code != sph.SPH_E_REBUILD:
                raise
            h_in = d["h"].clone()
    dev = {k: torch.tensor(v, device="cuda") for k, v in st.items()}
    lap = torch.zeros(n, dtype=torch.float32, device="cuda")
    x = sph.sph_sphenix_default_params()
    s = sph.sphenix_state(dev["alpha_v"], dev["alpha_c"], dev["div_v_prev"], dev["v_sig"], lap)
    sph.sph_sphenix_gradient(ctx, cells, part, sph.density_out(d), x, dt, s)
    sph.sph_force_sphenix(ctx, cells, part, sph.density_out(d), dev["alpha_v"], dev["alpha_c"],
                          sph.force_out(f))
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in d.items()}
    out.update({k: v.cpu().numpy() for k, v in f.items()})
    # the updated parameters (v_sig stays the force's output)
    out.update({k: v.cpu().numpy() for k, v in dev.items() if k != "v_sig"})
    out["lap_u"] = lap.cpu().numpy()
    out["_cell"] = float(p["L"]) / sph.sph_cells_sync(ctx, cells)
    return out


def _check(orc, p, seed, floor=False, tree=False):
    """floor: bounds include the rounding of the FP32 cell-relative
    coordinates (needed where cells are many supports wide); tree: on the
    nested grids (positions relative to each target's own level: the plain
    bounds)."""
    q, od0, st, dt = _setup(orc, p, seed)
    g = _run_gpu(p, st, dt, tree=tree)
    cell = g["_cell"] if floor else None
    vmax = float(np.sqrt(q["vx"] ** 2 + q["vy"] ** 2 + q["vz"] ** 2).max()) if floor else None
    X = orc.Sphenix()
    f64 = {k: v.astype(np.float64) for k, v in st.items()}
    od, av, og, of = orc.sphenix_evaluate(q, q["h0"], f64["alpha_v"], f64["alpha_c"],
                                          f64["div_v_prev"], f64["v_sig"], dt, X)
    # density and force against the SPHENIX oracle, with the plain bounds
    rep = compare(g, od, of, cell=cell, vmax=vmax)
    # the divergence of this evaluation is handed on
    assert np.array_equal(g["div_v_prev"], g["div_v"])
    # viscosity parameter: FP32 rounding plus the effect of the divergence's
    # own error, measured by re-running the oracle's update with the
    # divergence moved by twice that error
    e_div = 2.0 * np.abs(g["div_v"] - od["div_v"]) + 1e-30
    up = orc.sphenix_alpha_v(dt, od["h"], od["c"], od["div_v"] + e_div, f64["div_v_prev"], f64["v_sig"],
                             f64["alpha_v"], X)
    dn = orc.sphenix_alpha_v(dt, od["h"], od["c"], od["div_v"] - e_div, f64["div_v_prev"], f64["v_sig"],
                             f64["alpha_v"], X)
    lim = 4e-6 * X.alpha_v_max + np.maximum(np.abs(up - av), np.abs(dn - av))
    err = np.abs(g["alpha_v"] - av)
    assert (err / lim).max() <= 1.0, f"alpha_v: max error {err.max():.3e}"
    # Laplacian: a sum with cancellation, 1e-4 of its rms plus the h error
    # (the gradient terms scale as H^-5), plus, with the coordinate floor d_i,
    # d_i times the sum of the absolute terms, which is at most
    # max|u_i - u_j| / H_i^2 int_0^1 4 pi q |w'(q)| dq = 12 max|u_i - u_j| / H_i^2
    # for the cubic spline
    rms = np.sqrt(np.mean(og["lap_u"] ** 2))
    err = np.abs(g["lap_u"] - og["lap_u"])
    lim = 1e-4 * rms + 5e-5 * np.abs(og["lap_u"])
    if floor:
        from gpu_common import coord_floor
        Hh = GAMMA_K * od["h"]
        du = np.maximum(np.abs(q["u"] - q["u"].min()), np.abs(q["u"] - q["u"].max()))
        lim = lim + 2.0 * coord_floor(cell, od["h"]) * 12.0 * du / Hh ** 2
    assert (err / lim).max() <= 1.0, f"lap_u: max error / rms {err.max() / rms:.3e}"
    # conduction parameter: dt times the Laplacian and v_c errors, plus the
    # limiter's dependence on the neighbours' alpha_V
    H = GAMMA_K * od["h"]
    e_av = np.abs(g["alpha_v"] - av).max()
    e_vc = 1e-5 * og["v_c"] + np.sqrt(8e-5 * np.max(od["P"] / od["rho"]))
    lim = (dt * (X.beta_c * H * lim / np.sqrt(q["u"]) + f64["alpha_c"] * e_vc / H) +
           X.alpha_c_max * e_av / X.alpha_v_max + 2e-6)
    err = np.abs(g["alpha_c"] - og["alpha_c"])
    assert (err / lim).max() <= 1.0, f"alpha_c: max error {err.max():.3e}"
    # the run exercised every branch of the updates
    assert (av > f64["alpha_v"]).any() and (av < f64["alpha_v"]).any()
    assert (og["alpha_c"] != f64["alpha_c"]).mean() > 0.5
    cap = X.alpha_c_max * (1.0 - og["alpha_v_ngb"] / X.alpha_v_max)
    interior = (og["alpha_c"] > 1e-6) & (og["alpha_c"] < cap - 1e-6)
    assert interior.any() and (~interior).any()
    assert np.abs(of["du_cond"]).max() > 1e-3 * np.abs(of["du_dt"]).max()
    return rep


def test_sphenix_evaluation_lattice(orc):
    p = inputs.lattice(16, seed=7, sigma_v=0.05)
    _check(orc, p, seed=1)


def test_sphenix_evaluation_clustered(orc):
    p = inputs.clustered(6000, n_spheres=8, seed=5)
    _check(orc, p, seed=2, floor=True)


def test_sphenix_reduces_to_minimal_force():
    """alpha_V,i = alpha_V everywhere and alpha_c = 0: sph_force_sphenix returns
    what sph_force returns (same pairs, one more zero term per pair)."""
    import torch
    from paper_2305_13380_gb300 import sph
    p = inputs.lattice(14, seed=2, sigma_v=0.05)
    ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), flags=sph.SPH_FLAG_SYNC))
    t = sph.to_device(p)
    n = int(t["x"].shape[0])
    part = sph.particles(t)
    d = sph.alloc_density(n)
    cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], t["h0"])
    sph.sph_density(ctx, cells, part, t["h0"], sph.density_out(d))
    f0, f1 = sph.alloc_force(n), sph.alloc_force(n)
    sph.sph_force(ctx, cells, part, sph.density_out(d), sph.force_out(f0))
    av = torch.full((n,), float(ctx.params.alpha_v), dtype=torch.float32, device="cuda")
    ac = torch.zeros(n, dtype=torch.float32, device="cuda")
    sph.sph_force_sphenix(ctx, cells, part, sph.density_out(d), av, ac, sph.force_out(f1))
    for k in ("ax", "ay", "az", "du_dt", "v_sig"):
        a, b = f0[k].cpu().numpy(), f1[k].cpu().numpy()
        scale = np.abs(a).max()
        assert np.abs(a - b).max() <= 2e-6 * scale, k


def test_sphenix_evaluation_clustered_nested_grids(orc):
    # the clustered case on the nested grids: lists, reverse pairs and the
    # list-free path carry the fifth record
    p = inputs.clustered(6000, n_spheres=8, seed=5)
    _check(orc, p, seed=2, tree=True)


def test_sphenix_evaluation_strongly_clustered_nested_grids(orc):
    # h over more than 30x (four dense spheres)
    p = inputs.clustered(6000, n_spheres=4, seed=9)
    q = as_f32(p)
    assert q["h0"].max() / q["h0"].min() > 10
    _check(orc, p, seed=3, tree=True)


def test_sphenix_nested_grids_match_uniform_grid(orc):
    # the same evaluation on both grid modes agrees to the FP32 rounding
    p = inputs.lattice(14, seed=6, sigma_v=0.05)
    q, od, st, dt = _setup(orc, p, seed=5)
    gu = _run_gpu(p, st, dt, tree=False)
    gt = _run_gpu(p, st, dt, tree=True)
    for k in ("ax", "ay", "az", "du_dt"):
        scale = np.sqrt(np.mean(gu[k] ** 2)) + 1e-30
        assert np.abs(gt[k] - gu[k]).max() <= 2e-5 * scale, k
    for k in ("alpha_v", "alpha_c", "v_sig"):
        assert np.allclose(gt[k], gu[k], rtol=2e-5, atol=2e-6), k


@pytest.mark.parametrize("tree", [False, True])
def test_sphenix_step_matches_oracle(orc, tree):
    import torch
    from paper_2305_13380_gb300 import sph
    from test_gpu_step import _oracle_state, _pool
    p = inputs.lattice(12, seed=4, sigma_v=0.05)
    s = _oracle_state(orc, p)
    n = len(s["x"])
    rng = np.random.default_rng(9)
    q = as_f32(p)
    od = orc.density(q, q["h0"])
    s["alpha_v"] = _f32(rng.uniform(0.0, 2.0, n)).astype(np.float64)
    s["alpha_c"] = _f32(rng.uniform(0.0, 1.0, n)).astype(np.float64)
    rms = np.sqrt(np.mean(od["div_v"] ** 2))
    s["div_v"] = _f32(od["div_v"] + rng.choice([-1.0, 1.0], n) * rng.uniform(2.0, 4.0, n) * rms).astype(np.float64)
    off, box, arr = _pool([s])
    arr["div_v"] = torch.tensor(s["div_v"], dtype=torch.float32, device="cuda")
    av = torch.tensor(s["alpha_v"], dtype=torch.float32, device="cuda")
    ac = torch.tensor(s["alpha_c"], dtype=torch.float32, device="cuda")
    flags = sph.SPH_FLAG_SYNC | (sph.SPH_FLAG_TREE if tree else 0)
    ctx = sph.Context(sph.sph_default_params(flags=flags))
    pool = sph.pool(off, box, arr)
    sph.sph_step_sphenix(ctx, pool, sph.sph_sphenix_default_params(), av, ac)
    vsig_prev = s["v_sig"].copy()
    dt = orc.sphenix_step(s, 0.1)
    assert float(arr["dt"].cpu()[0]) == pytest.approx(dt, rel=1e-6)
    g = {k: v.cpu().numpy() for k, v in arr.items()}
    for k in ("x", "y", "z"):
        diff = np.abs(g[k] - s[k])
        assert np.minimum(diff, 1.0 - diff).max() < 1e-6 / 12
    vscale = np.sqrt(np.mean(s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2))
    for k in ("vx", "vy", "vz"):
        assert np.abs(g[k] - s[k]).max() < 1e-4 * vscale
    assert np.allclose(g["u"], s["u"], rtol=1e-6)
    arms = np.sqrt(np.mean(s["ax"] ** 2 + s["ay"] ** 2 + s["az"] ** 2))
    for k in ("ax", "ay", "az"):
        assert np.abs(g[k] - s[k]).max() < 1e-4 * arms
    durms = np.sqrt(np.mean(s["du_dt"] ** 2))
    assert np.abs(g["du_dt"] - s["du_dt"]).max() < 1e-4 * durms
    # alpha_V: FP32 rounding plus the divergence error through alpha_loc,
    # whose slope in the divergence is at most alpha_max H^2 / (dt v_sig^2)
    X = orc.Sphenix()
    H = GAMMA_K * s["h"]
    e_div = np.abs(g["div_v"] - s["div_v"])
    lim = 4e-6 * X.alpha_v_max + X.alpha_v_max * H * H / (dt * vsig_prev ** 2) * e_div
    err = np.abs(av.cpu().numpy() - s["alpha_v"])
    assert (err / lim).max() <= 1.0, f"alpha_v: max error {err.max():.3e}"
    # alpha_c: the limiter follows the neighbours' alpha_V
    err = np.abs(ac.cpu().numpy() - s["alpha_c"])
    assert err.max() <= 1e-5 + X.alpha_c_max * np.max(lim) / X.alpha_v_max, f"alpha_c: {err.max():.3e}"


@pytest.mark.parametrize("tree", [False, True])
def test_sphenix_pool_equals_alone(orc, tree):
    """Three simulations with their own time-steps: each one's SPHENIX steps
    are bitwise the same alone and inside a pool (the viscosity and
    conduction updates take each simulation's own dt), on both grid modes."""
    import torch
    from paper_2305_13380_gb300 import sph
    from test_gpu_step import _oracle_state, _pool
    sims = [inputs.lattice(10, seed=11), inputs.lattice(13, seed=12, sigma_v=0.1),
            inputs.two_spheres(5, n_max=4e3)]
    states = [_oracle_state(orc, p) for p in sims]
    rng = np.random.default_rng(3)
    for st in states:
        n = len(st["x"])
        st["alpha_v"] = _f32(rng.uniform(0.0, 0.5, n))
        st["alpha_c"] = _f32(rng.uniform(0.0, 0.3, n))
        st["div_v"] = _f32(rng.normal(0.0, 1.0, n))
    X = sph.sph_sphenix_default_params()

    def run(sts):
        off, box, arr = _pool(sts)
        arr["div_v"] = torch.tensor(np.concatenate([s["div_v"] for s in sts]), device="cuda")
        av = torch.tensor(np.concatenate([s["alpha_v"] for s in sts]), device="cuda")
        ac = torch.tensor(np.concatenate([s["alpha_c"] for s in sts]), device="cuda")
        flags = sph.SPH_FLAG_SYNC | (sph.SPH_FLAG_TREE if tree else 0)
        ctx = sph.Context(sph.sph_default_params(flags=flags))
        for _ in range(3):
            sph.sph_step_sphenix(ctx, sph.pool(off, box, arr), X, av, ac)
        out = {k: v.cpu().numpy() for k, v in arr.items()}
        out["alpha_v"], out["alpha_c"] = av.cpu().numpy(), ac.cpu().numpy()
        return off.cpu().numpy(), out

    offs, mixed = run(states)
    dts = set()
    for i, st in enumerate(states):
        _, alone = run([st])
        sl = slice(offs[i], offs[i + 1])
        for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "div_v", "ax", "ay", "az", "du_dt",
                  "v_sig", "alpha_v", "alpha_c"):
            assert np.array_equal(mixed[k][sl], alone[k]), (i, k)
        assert mixed["dt"][i] == alone["dt"][0]
        dts.add(float(alone["dt"][0]))
    assert len(dts) == 3


def test_sphenix_without_time_keeps_the_viscosity_parameters(orc):
    # dt = 0: alpha_V is unchanged bit for bit; alpha_c only meets its limits
    p = inputs.lattice(12, seed=5, sigma_v=0.05)
    q, od, st, _ = _setup(orc, p, seed=4)
    g = _run_gpu(p, st, 0.0)
    assert np.array_equal(g["alpha_v"], st["alpha_v"])
    inside = g["alpha_c"] > 0.0
    assert np.array_equal(g["alpha_c"][inside], st["alpha_c"][inside])


def test_sphenix_with_sorted_interactions_and_wendland(orc):
    """The SPHENIX loops read the density's lists, so they run unchanged on
    the axis-sorted filter's lists, and with another kernel."""
    import torch
    from paper_2305_13380_gb300 import sph
    p = inputs.lattice(14, seed=8, sigma_v=0.05)
    q, _, st, dt = _setup(orc, p, seed=6)
    for axis, kern in ((True, 0), (False, 2)):
        flags = sph.SPH_FLAG_SYNC | (sph.SPH_FLAG_AXIS_SORT if axis else 0)
        ctx = sph.Context(sph.sph_default_params(box_size=float(p["L"]), flags=flags, kernel=kern))
        t = sph.to_device(p)
        n = int(t["x"].shape[0])
        part = sph.particles(t)
        d, f = sph.alloc_density(n), sph.alloc_force(n)
        cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], t["h0"])
        sph.sph_density(ctx, cells, part, t["h0"], sph.density_out(d))
        dev = {k: torch.tensor(v, device="cuda") for k, v in st.items()}
        s = sph.sphenix_state(dev["alpha_v"], dev["alpha_c"], dev["div_v_prev"], dev["v_sig"])
        sph.sph_sphenix_gradient(ctx, cells, part, sph.density_out(d), sph.sph_sphenix_default_params(), dt, s)
        sph.sph_force_sphenix(ctx, cells, part, sph.density_out(d), dev["alpha_v"], dev["alpha_c"],
                              sph.force_out(f))
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in d.items()}
        g.update({k: v.cpu().numpy() for k, v in f.items()})
        X = orc.Sphenix()
        phys = orc.Physics(kernel=kern)
        f64 = {k: v.astype(np.float64) for k, v in st.items()}
        od, av, og, of = orc.sphenix_evaluate(q, q["h0"], f64["alpha_v"], f64["alpha_c"], f64["div_v_prev"],
                                              f64["v_sig"], dt, X, phys)
        compare(g, od, of)
        assert np.abs(dev["alpha_c"].cpu().numpy() - og["alpha_c"]).max() < 1e-4
