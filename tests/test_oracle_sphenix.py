"""Pins of the oracle's SPHENIX flavour (Sec. 3.3) against facts that do not
come from the oracle itself: limits and special cases of the viscosity
update, the composition law of its decay, the Laplacian of fields whose
Laplacian is known, the conservation of energy and momentum by the
symmetric pair terms, the direction of heat flow, and the reduction to the
"Minimal" force when every viscosity parameter equals alpha_V."""
import numpy as np
import pytest

import oracle
from paper_2305_13380_gb300 import inputs

X = oracle.Sphenix()


def _f64(p):
    return {k: (float(v) if k == "L" else np.asarray(v, dtype=np.float64).copy()) for k, v in p.items()}


def _perfect_lattice(n_side=12):
    p = _f64(inputs.lattice(n_side, jitter=0.0))
    for k in ("vx", "vy", "vz"):
        p[k][:] = 0.0
    return p


def _interior(p, frac=0.15):
    c0 = 0.5 * p["L"]
    r = np.sqrt((p["x"] - c0) ** 2 + (p["y"] - c0) ** 2 + (p["z"] - c0) ** 2)
    return np.where(r < frac * p["L"])[0]


# ---- viscosity parameter (eqs. "sphenix_visc1"-"sphenix_visc4") ------------

def _av(dt, alpha, div, div_prev, vsig=1.0, c=1.0, h=0.1):
    one = np.ones(1)
    return oracle.sphenix_alpha_v(dt, h * one, c * one, div * one, div_prev * one, vsig * one,
                                  alpha * one, X)[0]


def test_alpha_v_unchanged_without_time():
    # dt = 0: no rate of divergence, no decay
    for a in (0.0, 0.3, 1.7):
        assert _av(0.0, a, div=-5.0, div_prev=3.0) == a


def test_alpha_v_local_value_limits():
    # alpha_loc = alpha_max S / (v_sig^2 + S): half of alpha_max where S = v_sig^2,
    # alpha_max in the limit of a strong convergence, 0 for an expanding flow
    h, vsig, dt = 0.1, 2.0, 1e-3
    H = oracle.GAMMA_K * h
    rate = -(vsig / H) ** 2          # S = H^2 (-rate) = v_sig^2
    assert _av(dt, 0.0, div=rate * dt, div_prev=0.0, vsig=vsig, h=h) == pytest.approx(X.alpha_v_max / 2, rel=1e-12)
    assert _av(dt, 0.0, div=-1e12, div_prev=0.0, vsig=vsig, h=h) == pytest.approx(X.alpha_v_max, rel=1e-9)
    assert _av(dt, 0.0, div=+5.0, div_prev=0.0, vsig=vsig, h=h) == 0.0


def test_alpha_v_rises_to_local_value_and_decays_towards_it():
    h, vsig, dt = 0.1, 2.0, 1e-3
    H = oracle.GAMMA_K * h
    rate = -(vsig / H) ** 2
    # below alpha_loc = 1: jumps to it; above: decays towards it, never below
    assert _av(dt, 0.2, div=rate * dt, div_prev=0.0, vsig=vsig, h=h) == pytest.approx(1.0, rel=1e-12)
    up = _av(dt, 1.8, div=rate * dt, div_prev=0.0, vsig=vsig, h=h)
    assert 1.0 < up < 1.8


def test_alpha_v_decay_composes():
    # away from shocks (S = 0) the decay is exponential in time: two steps of
    # dt/2 equal one step of dt, and the time for a factor 1/2 is
    # ln 2 H / (ell c)
    h, c = 0.1, 3.0
    H = oracle.GAMMA_K * h
    dt = 0.4 * H / (X.ell * c)
    one = _av(dt, 1.5, div=0.0, div_prev=0.0, c=c, h=h)
    half = _av(dt / 2, _av(dt / 2, 1.5, div=0.0, div_prev=0.0, c=c, h=h), div=0.0, div_prev=0.0, c=c, h=h)
    assert one == pytest.approx(half, rel=1e-14)
    t_half = np.log(2.0) * H / (X.ell * c)
    assert _av(t_half, 1.5, div=0.0, div_prev=0.0, c=c, h=h) == pytest.approx(0.75, rel=1e-13)


# ---- gradient pass: Laplacian of u -----------------------------------------

def _lap(p, u, targets):
    q = dict(p)
    q["u"] = u
    d = oracle.density(q, p["h0"])
    n = len(u)
    return oracle.sphenix_gradient(q, d, np.zeros(n), np.zeros(n), 0.0, targets, X)["lap_u"]


def test_laplacian_of_known_fields():
    p = _perfect_lattice()
    tg = _interior(p)
    assert len(tg) > 20
    c0 = 0.5 * p["L"]
    x, y, z = p["x"] - c0, p["y"] - c0, p["z"] - c0
    scale = np.abs(x[tg]).max() ** 2
    # constant, linear and harmonic (xy) fields have zero Laplacian
    assert np.all(_lap(p, np.full(len(x), 2.0), tg) == 0.0)
    assert np.abs(_lap(p, 1.0 + 0.3 * x - 0.2 * y + 0.1 * z, tg)).max() < 1e-10
    assert np.abs(_lap(p, 1.0 + x * y, tg)).max() < 1e-10 / scale
    # |x|^2 has Laplacian 6, x^2 has 2: the estimate is exact for quadratics
    # up to the lattice quadrature of the kernel's second moment (~1 %), and
    # isotropic on a cubic lattice (the ratio is 3)
    quad = _lap(p, 1.0 + x * x + y * y + z * z, tg)
    x2 = _lap(p, 1.0 + x * x, tg)
    assert np.allclose(quad, 6.0, rtol=0.02)
    assert np.allclose(quad / x2, 3.0, rtol=1e-10)
    # the sign: a hot spot (local maximum of u) has a negative Laplacian
    assert np.all(_lap(p, 2.0 - (x * x + y * y + z * z), tg) < 0)


def test_gradient_pass_grid_equals_brute_force():
    p = _f64(inputs.clustered(1500, n_spheres=6, seed=3))
    n = len(p["x"])
    rng = np.random.default_rng(5)
    d = oracle.density(p, p["h0"])
    av = rng.uniform(0.0, 2.0, n)
    ac = rng.uniform(0.0, 1.0, n)
    g1 = oracle.sphenix_gradient(p, d, av, ac, 1e-3, None, X)
    g2 = oracle.sphenix_gradient(p, d, av, ac, 1e-3, None, X, brute=True)
    for k in g1:
        assert np.allclose(g1[k], g2[k], rtol=1e-12, atol=0.0), k


# ---- conduction parameter (eqs. "artconddt", "condshocklimiter", "conductionlimiter")

def test_conduction_parameter_limits():
    p = _perfect_lattice(10)
    n = len(p["x"])
    p["u"][:] = 1.0
    d = oracle.density(p, p["h0"])
    ac = np.full(n, 0.6)
    # uniform u at rest: no source and no decay (v_c = 0 but for the square
    # root of the rounding of P), alpha_c kept
    g = oracle.sphenix_gradient(p, d, np.zeros(n), ac, 0.1, None, X)
    assert np.all(g["v_c"] < 1e-6)
    assert np.all(g["lap_u"] == 0.0)
    assert np.allclose(g["alpha_c"], 0.6, rtol=0, atol=1e-6)
    # a neighbour at the largest viscosity shuts conduction off
    av = np.zeros(n)
    av[0] = X.alpha_v_max
    g = oracle.sphenix_gradient(p, d, av, ac, 0.1, None, X)
    nb = g["alpha_v_ngb"] == X.alpha_v_max
    assert nb.sum() > 30 and np.all(g["alpha_c"][nb] == 0.0)
    # half of the largest viscosity halves the bound
    av[0] = 0.5 * X.alpha_v_max
    g = oracle.sphenix_gradient(p, d, av, ac, 0.1, None, X)
    nb = g["alpha_v_ngb"] == 0.5 * X.alpha_v_max
    assert np.allclose(g["alpha_c"][nb], 0.5 * X.alpha_c_max, rtol=1e-15)


def test_conduction_parameter_grows_on_curved_u_and_decays_with_flow():
    p = _perfect_lattice(10)
    n = len(p["x"])
    c0 = 0.5 * p["L"]
    x = p["x"] - c0
    tg = _interior(p, 0.2)
    ac0 = np.full(n, 0.2)
    # u with positive curvature, no flow: alpha_c rises by dt beta_c H lap/sqrt(u)
    p["u"] = 1.0 + 5.0 * x * x
    d = oracle.density(p, p["h0"])
    g = oracle.sphenix_gradient(p, d, np.zeros(n), ac0, 1e-3, tg, X)
    assert np.all(g["alpha_c"] > 0.2) and np.all(g["lap_u"] > 0)
    # uniform u, converging flow: v_c > 0 and alpha_c decays towards alpha_c,min
    p["u"][:] = 1.0
    p["vx"] = -x
    d = oracle.density(p, p["h0"])
    g = oracle.sphenix_gradient(p, d, np.zeros(n), ac0, 1e-3, tg, X)
    assert np.all(g["v_c"] > 0) and np.all(g["alpha_c"] < 0.2) and np.all(g["alpha_c"] >= 0.0)


# ---- force loop -------------------------------------------------------------

def _state(seed=2, n=1200):
    p = _f64(inputs.clustered(n, n_spheres=5, seed=seed))
    n = len(p["x"])
    rng = np.random.default_rng(seed)
    p["u"] = rng.uniform(0.5, 2.0, n)
    p["vx"] = rng.normal(0, 0.3, n)
    p["vy"] = rng.normal(0, 0.3, n)
    p["vz"] = rng.normal(0, 0.3, n)
    d = oracle.density(p, p["h0"])
    return p, d, rng


def test_force_reduces_to_minimal():
    # alpha_V,i = alpha_V everywhere and no conduction: the "Minimal" force
    p, d, _ = _state()
    n = len(p["x"])
    phys = oracle.Physics()
    f0 = oracle.force(p, d, None, phys)
    f1 = oracle.sphenix_force(p, d, np.full(n, phys.alpha_v), np.zeros(n), None, phys)
    for k in ("ax", "ay", "az", "du_dt", "v_sig"):
        scale = np.abs(f0[k]).max()
        assert np.abs(f1[k] - f0[k]).max() <= 1e-13 * scale, k
    assert np.array_equal(f0["n_pairs"], f1["n_pairs"])
    assert np.all(f1["du_cond"] == 0.0)


def test_sphenix_pair_terms_conserve_energy_and_momentum():
    p, d, rng = _state(seed=4)
    n = len(p["x"])
    av = rng.uniform(0.0, 2.0, n)
    ac = rng.uniform(0.0, 1.0, n)
    f = oracle.sphenix_force(p, d, av, ac)
    m = p["m"]
    cond = m * f["du_cond"]
    assert abs(cond.sum()) <= 1e-12 * np.abs(cond).sum()
    assert np.abs(cond).sum() > 0
    for k in ("ax", "ay", "az"):
        assert abs((m * f[k]).sum()) <= 1e-12 * np.abs(m * f[k]).sum()
    power = m * (p["vx"] * f["ax"] + p["vy"] * f["ay"] + p["vz"] * f["az"] + f["du_dt"])
    work = np.abs(m * f["du_dt"]).sum()
    assert abs(power.sum()) <= 1e-11 * work


def test_conduction_moves_heat_from_hot_to_cold():
    p = _perfect_lattice(10)
    n = len(p["x"])
    p["u"][:] = 1.0
    hot = _interior(p, 0.1)[0]
    p["u"][hot] = 3.0
    d = oracle.density(p, p["h0"])
    f = oracle.sphenix_force(p, d, np.zeros(n), np.full(n, 0.5))
    dc = f["du_cond"]
    assert dc[hot] < 0
    others = np.delete(np.arange(n), hot)
    assert np.all(dc[others] >= 0) and (dc[others] > 0).sum() > 30
    assert abs((p["m"] * dc).sum()) <= 1e-12 * np.abs(p["m"] * dc).sum()


def test_sphenix_step_matches_minimal_step_without_new_terms():
    # every alpha_V at alpha_V,max with no decay (ell = 0) stays there, and
    # alpha_c = 0 with beta_c = 0 keeps conduction off: the step is then the
    # "Minimal" step with alpha_V = alpha_V,max
    p, _, _ = _state(seed=6, n=800)
    n = len(p["x"])
    phys = oracle.Physics()
    d, f = oracle.density_force(p, p["h0"], phys)
    s0 = dict(p)
    s0.update(h=d["h"], ax=f["ax"], ay=f["ay"], az=f["az"], du_dt=f["du_dt"], v_sig=f["v_sig"])
    s1 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s0.items()}
    s1.update(alpha_v=np.full(n, X.alpha_v_max), alpha_c=np.zeros(n), div_v=d["div_v"])
    Xs = oracle.Sphenix(ell=0.0, beta_c=0.0)
    phys2 = oracle.Physics(alpha_v=X.alpha_v_max)
    dt0 = oracle.step(s0, 0.1, phys2)
    dt1 = oracle.sphenix_step(s1, 0.1, Xs, phys2)
    assert dt0 == dt1
    assert np.all(s1["alpha_v"] == X.alpha_v_max)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h"):
        assert np.allclose(s0[k], s1[k], rtol=1e-12, atol=1e-15), k
