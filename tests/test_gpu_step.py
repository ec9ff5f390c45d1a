"""sph_step on the GPU: one simulation against the oracle's kick-drift-kick
step, and a pool of several simulations against each one alone."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

from gpu_common import as_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


def _oracle_state(orc, p):
    q = as_f32(p)
    d, f = orc.density_force(q, q["h0"])
    s = {k: q[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u")}
    s.update(L=p["L"], h=d["h"].copy(), ax=f["ax"].copy(), ay=f["ay"].copy(), az=f["az"].copy(),
             du_dt=f["du_dt"].copy(), v_sig=f["v_sig"].copy())
    return s


def _pool(states):
    """Device pool from a list of state dicts (float64 numpy)."""
    import torch
    from paper_2305_13380_gb300 import sph
    dev = "cuda"
    cat = lambda k: np.concatenate([s[k] for s in states])  # noqa: E731
    arrays = {}
    for k in ("x", "y", "z"):
        arrays[k] = torch.tensor(cat(k), dtype=torch.float64, device=dev)
    for k in ("vx", "vy", "vz", "u", "m", "h", "ax", "ay", "az", "du_dt", "v_sig"):
        arrays[k] = torch.tensor(cat(k), dtype=torch.float32, device=dev)
    n = arrays["x"].shape[0]
    for k in ("rho", "f", "div_v", "curl_v", "P", "c", "balsara"):
        arrays[k] = torch.zeros(n, dtype=torch.float32, device=dev)
    arrays["dt"] = torch.zeros(len(states), dtype=torch.float64, device=dev)
    off = np.concatenate([[0], np.cumsum([len(s["x"]) for s in states])])
    sim_offset = torch.tensor(off, dtype=torch.int64, device=dev)
    box = torch.tensor([s["L"] for s in states], dtype=torch.float64, device=dev)
    return sim_offset, box, arrays


def test_step_matches_oracle(orc):
    from paper_2305_13380_gb300 import sph
    p = inputs.lattice(12, seed=3, sigma_v=0.05)
    s = _oracle_state(orc, p)
    off, box, arr = _pool([s])
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC))
    pool = sph.pool(off, box, arr)
    sph.sph_step(ctx, pool)
    dt_gpu = float(arr["dt"].cpu()[0])
    dt = orc.step(s, 0.1)
    assert dt_gpu == pytest.approx(dt, rel=1e-6)
    g = {k: v.cpu().numpy() for k, v in arr.items()}
    d = 1.0 / 12
    for k in ("x", "y", "z"):
        diff = np.abs(g[k] - s[k])
        diff = np.minimum(diff, 1.0 - diff)
        assert diff.max() < 1e-6 * d
    vscale = np.sqrt(np.mean(s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2))
    for k in ("vx", "vy", "vz"):
        assert np.abs(g[k] - s[k]).max() < 1e-4 * vscale
    assert np.allclose(g["u"], s["u"], rtol=1e-6)
    assert np.allclose(g["h"], s["h"], rtol=1e-5)
    assert np.allclose(g["rho"], s["rho"], rtol=1e-5)
    arms = np.sqrt(np.mean(s["ax"] ** 2 + s["ay"] ** 2 + s["az"] ** 2))
    for k in ("ax", "ay", "az"):
        assert np.abs(g[k] - s[k]).max() < 1e-4 * arms
    # FP64 conservation sums on the device against the oracle's sums of its
    # own state (m, the final v, a and du/dt of the step), within what the
    # per-particle bounds on a (1e-4 rms), v and du/dt allow
    import torch
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    sph.sph_conservation(ctx, pool, out)
    c = out.cpu().numpy()
    m = s["m"]
    A = np.stack([s["ax"], s["ay"], s["az"]], 1)
    V = np.stack([s["vx"], s["vy"], s["vz"]], 1)
    mom = (m[:, None] * A).sum(0)
    en = (m * ((V * A).sum(1) + s["du_dt"])).sum()
    scale = (m * np.sqrt((A ** 2).sum(1))).sum()
    assert np.all(np.abs(mom) < 1e-13 * scale)      # the oracle: round-off
    assert np.all(np.abs(c[:3] - mom) <= 1e-4 * arms * m.sum())
    rms_du = np.sqrt(np.mean(s["du_dt"] ** 2))
    e_tol = (m * (np.sqrt((V ** 2).sum(1)) * 1e-4 * arms * np.sqrt(3.0)
                  + np.sqrt((A ** 2).sum(1)) * 1e-4 * vscale * np.sqrt(3.0) + 1e-4 * rms_du)).sum()
    assert abs(c[3] - en) <= e_tol
    # and the device's FP64 sums of the GPU's own arrays
    mg = g["m"].astype(np.float64)
    assert c[0] == pytest.approx((mg * g["ax"]).sum(), rel=1e-6, abs=1e-9 * scale)
    eg = (mg * (g["vx"].astype(np.float64) * g["ax"] + g["vy"].astype(np.float64) * g["ay"]
                + g["vz"].astype(np.float64) * g["az"] + g["du_dt"])).sum()
    assert c[3] == pytest.approx(eg, rel=1e-6, abs=1e-9 * abs(eg) + 1e-12)


def test_pool_equals_alone(orc):
    """Each simulation's step is bitwise the same alone and inside a pool."""
    from paper_2305_13380_gb300 import sph
    sims = [inputs.lattice(10, seed=11), inputs.lattice(13, seed=12, sigma_v=0.1),
            inputs.two_spheres(5, n_max=4e3)]
    states = [_oracle_state(orc, p) for p in sims]
    off, box, arr = _pool(states)
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC))
    for _ in range(3):
        sph.sph_step(ctx, sph.pool(off, box, arr))
    mixed = {k: v.cpu().numpy() for k, v in arr.items()}
    offs = off.cpu().numpy()
    for i, st in enumerate(states):
        o1, b1, a1 = _pool([st])
        c1 = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC))
        for _ in range(3):
            sph.sph_step(c1, sph.pool(o1, b1, a1))
        alone = {k: v.cpu().numpy() for k, v in a1.items()}
        sl = slice(offs[i], offs[i + 1])
        for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "ax", "ay", "az", "du_dt",
                  "v_sig"):
            assert np.array_equal(mixed[k][sl], alone[k]), (i, k)
        assert mixed["dt"][i] == alone["dt"][0]


def test_conservation_after_a_force_evaluation(orc):
    """Right after density and force (velocities as the force saw them), the
    momentum and energy sums vanish up to round-off: the oracle's to FP64
    round-off, the device's (of the GPU's FP32 pair sums, each side of a pair
    computed by its own target) to the FP32 level."""
    import torch
    from gpu_common import run_gpu
    from paper_2305_13380_gb300 import sph
    p = inputs.lattice(14, seed=6, sigma_v=0.2)
    q = as_f32(p)
    od, of = orc.density_force(q, q["h0"])
    g = run_gpu(p)
    dev = "cuda"
    arr = {k: torch.tensor(np.asarray(p[k], dtype=np.float64), device=dev) for k in ("x", "y", "z")}
    for k in ("vx", "vy", "vz", "m", "u"):
        arr[k] = torch.tensor(np.asarray(p[k], dtype=np.float32), device=dev)
    for k in ("h", "rho", "f", "div_v", "curl_v", "P", "c", "balsara", "ax", "ay", "az", "du_dt", "v_sig"):
        arr[k] = torch.tensor(g[k], device=dev)
    arr["dt"] = torch.zeros(1, dtype=torch.float64, device=dev)
    n = len(p["x"])
    pl = sph.pool(torch.tensor([0, n], dtype=torch.int64, device=dev),
                  torch.tensor([p["L"]], dtype=torch.float64, device=dev), arr)
    ctx = sph.Context(sph.sph_default_params(flags=sph.SPH_FLAG_SYNC))
    out = torch.zeros(4, dtype=torch.float64, device=dev)
    sph.sph_conservation(ctx, pl, out)
    c = out.cpu().numpy()
    m = q["m"]
    A = np.stack([of["ax"], of["ay"], of["az"]], 1)
    V = np.stack([q["vx"], q["vy"], q["vz"]], 1)
    s_mom = (m * np.sqrt((A ** 2).sum(1))).sum()
    s_en = (m * (np.abs(V * A).sum(1) + np.abs(of["du_dt"]))).sum()
    mom = (m[:, None] * A).sum(0)
    en = (m * ((V * A).sum(1) + of["du_dt"])).sum()
    assert np.all(np.abs(mom) < 1e-13 * s_mom) and abs(en) < 1e-13 * s_en
    assert np.all(np.abs(c[:3] - mom) < 1e-5 * s_mom)
    assert abs(c[3] - en) < 1e-5 * s_en
