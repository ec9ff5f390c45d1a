"""Pins of the oracle's force loop (Sec. 3.2, eqs. "densityenergy",
"basicartvisc", "alpha", "nuij", "balsara") and its kick-drift-kick step
(Sec. 2.4 with the Sec. 5.4 operators at a = 1)."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs


def _sums(p, f):
    m = p["m"]
    mom = np.array([(m * f["ax"]).sum(), (m * f["ay"]).sum(), (m * f["az"]).sum()])
    scale_m = (m * np.sqrt(f["ax"] ** 2 + f["ay"] ** 2 + f["az"] ** 2)).sum()
    e = (m * (p["vx"] * f["ax"] + p["vy"] * f["ay"] + p["vz"] * f["az"] + f["du_dt"])).sum()
    scale_e = (m * (np.abs(p["vx"] * f["ax"]) + np.abs(p["vy"] * f["ay"]) +
                    np.abs(p["vz"] * f["az"]) + np.abs(f["du_dt"]))).sum()
    return mom, scale_m, e, scale_e


@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_momentum_and_energy_conserved(orc, kind):
    # pair antisymmetry of the symmetrised equations of motion (Sec. 2.2, 3.2)
    if kind == "lattice":
        p = inputs.lattice(12, seed=1, sigma_v=0.2)
    else:
        p = inputs.clustered(1500, n_spheres=3, seed=11, sigma_v=0.3)
    d, f = orc.density_force(p, p["h0"])
    mom, sm, e, se = _sums(p, f)
    assert np.all(np.abs(mom) < 1e-13 * sm)
    assert abs(e) < 1e-13 * se
    # the viscosity is active in this input
    assert np.any(d["B"] > 0.1)


def test_lattice_at_rest_has_no_force(orc):
    p = inputs.lattice(10, jitter=0.0, sigma_v=0.0, u_noise=0.0)
    d, f = orc.density_force(p, p["h0"])
    # scale: one pressure pair term
    one = p["m"][0] * 2 * d["P"][0] / d["rho"][0] ** 2 * 10.0 / (orc.GAMMA_K * d["h"][0]) ** 4
    for k in ("ax", "ay", "az", "du_dt"):
        assert np.all(np.abs(f[k]) < 1e-13 * one)
    assert np.allclose(f["v_sig"], 2 * d["c"], rtol=1e-14)


def test_galilean_invariance(orc):
    p = inputs.lattice(10, seed=3, sigma_v=0.1)
    d, f = orc.density_force(p, p["h0"])
    q = dict(p)
    q["vx"] = p["vx"] - 2.0
    q["vz"] = p["vz"] + 0.7
    d2, f2 = orc.density_force(q, p["h0"])
    for k in ("ax", "ay", "az", "du_dt", "v_sig"):
        assert np.allclose(f[k], f2[k], rtol=1e-8, atol=1e-9 * np.abs(f[k]).max()), k


def _pair(orc, dx, dv, alpha=0.8):
    """Two particles in a large box with a given density state."""
    L = 10.0
    p = dict(L=L, x=np.array([5.0, 5.0 + dx]), y=np.array([5.0, 5.0]), z=np.array([5.0, 5.0]),
             vx=np.array([0.0, dv]), vy=np.zeros(2), vz=np.zeros(2), m=np.array([1.0, 2.0]),
             u=np.array([1.0, 1.5]))
    state = dict(h=np.array([0.6, 0.4]), rho=np.array([1.2, 1.6]), f=np.array([0.95, 1.05]),
                 P=np.array([0.8, 1.6]), c=np.array([1.0, 1.2]), B=np.array([0.5, 0.9]))
    phys = orc.Physics(alpha_v=alpha)
    return p, orc.force(p, state, phys=phys)


def test_pair_antisymmetry_and_switches(orc):
    H = orc.GAMMA_K * np.array([0.6, 0.4])
    # approaching pair (particle 2 moves toward 1): viscosity on
    p, f = _pair(orc, 0.5, -0.7)
    m = p["m"]
    assert m[0] * f["ax"][0] == pytest.approx(-m[1] * f["ax"][1], rel=1e-14)
    assert f["ay"][0] == 0.0 and f["az"][0] == 0.0
    e = (m * (p["vx"] * f["ax"] + f["du_dt"])).sum()
    assert abs(e) < 1e-14 * np.abs(m * f["du_dt"]).sum()
    _, f0 = _pair(orc, 0.5, -0.7, alpha=0.0)
    assert abs(f["ax"][0] - f0["ax"][0]) > 1e-3 * abs(f0["ax"][0])
    # v_sig grows with the approach speed: c_i + c_j - beta mu, mu = -0.7
    assert f["v_sig"][0] == pytest.approx(1.0 + 1.2 + 3 * 0.7, rel=1e-14)
    # receding pair: no viscosity at all
    _, fr = _pair(orc, 0.5, +0.7)
    _, fr0 = _pair(orc, 0.5, +0.7, alpha=0.0)
    assert fr["ax"][0] == fr0["ax"][0] and fr["du_dt"][1] == fr0["du_dt"][1]
    assert fr["v_sig"][0] == pytest.approx(2.2, rel=1e-14)
    # pressure pushes the pair apart: particle 1 (left) accelerates to -x
    assert fr0["ax"][0] < 0 < fr0["ax"][1]
    # the pair interacts while r < max(H_i, H_j) even though r > H_j
    assert H[1] < 0.9 < H[0]
    _, fm = _pair(orc, 0.9, 0.0)
    assert fm["ax"][0] != 0.0 and fm["n_pairs"][0] == 1
    # beyond both supports: nothing
    _, ff = _pair(orc, 1.1 * H[0], -0.5)
    assert ff["ax"][0] == 0.0 and ff["du_dt"][0] == 0.0 and ff["n_pairs"][0] == 0


def test_grid_equals_brute_force(orc):
    p = inputs.clustered(1200, n_spheres=2, seed=5)
    d = orc.density(p, p["h0"])
    a = orc.force(p, d, brute=False)
    b = orc.force(p, d, brute=True)
    for k in ("ax", "ay", "az", "du_dt", "v_sig"):
        assert np.allclose(a[k], b[k], rtol=1e-11, atol=1e-11 * np.abs(b[k]).max()), k
    assert np.array_equal(a["n_pairs"], b["n_pairs"])


def _initial_state(orc, p):
    d, f = orc.density_force(p, p["h0"])
    s = {k: np.array(p[k], dtype=np.float64) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u")}
    s.update(L=p["L"], h=d["h"].copy(), ax=f["ax"].copy(), ay=f["ay"].copy(), az=f["az"].copy(),
             du_dt=f["du_dt"].copy(), v_sig=f["v_sig"].copy())
    return s


def test_step_keeps_lattice_at_rest(orc):
    p = inputs.lattice(6, jitter=0.0, sigma_v=0.0, u_noise=0.0)
    s = _initial_state(orc, p)
    x0, u0 = s["x"].copy(), s["u"].copy()
    dt = orc.step(s, 0.1)
    assert dt > 0
    assert np.allclose(s["x"], x0, atol=1e-15)
    assert np.all(np.abs(s["vx"]) < 1e-14) and np.allclose(s["u"], u0, rtol=1e-14)


def test_step_conserves_momentum_and_converges(orc):
    p = inputs.lattice(6, seed=2, sigma_v=0.3)
    errs = []
    for cfl in (0.2, 0.1, 0.05):
        s = _initial_state(orc, p)
        m = s["m"]
        P0 = np.array([(m * s[k]).sum() for k in ("vx", "vy", "vz")])
        E0 = (m * (0.5 * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2) + s["u"])).sum()
        T = 0.0
        while T < 0.02:
            T += orc.step(s, cfl)
        P1 = np.array([(m * s[k]).sum() for k in ("vx", "vy", "vz")])
        E1 = (m * (0.5 * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2) + s["u"])).sum()
        assert np.all(np.abs(P1 - P0) < 1e-14)
        errs.append(abs(E1 - E0) / E0)
    # the leapfrog energy error shrinks as the time-step shrinks
    assert errs[2] < errs[0]
    assert errs[0] < 1e-4
