"""Magnitude pins of the oracle's force loop and kick-drift-kick step (Sec. 3.2,
eqs. "densityenergy", "basicartvisc", "alpha", "nuij", "balsara"; Sec. 2.4
leapfrog), evaluated here by hand from the equations, independently of the
oracle's code:

- the kernel gradient grad_i W(|x_i - x_j|, h) is differentiated by sympy from
  the cubic spline w(q) of Sec. 3.1 (not the oracle's hand-coded w'(q));
- two particles: a, du/dt and v_sig of each from the printed pair equations
  (with the readings of the equations taken where the paper is garbled);
- a perfect lattice with a linear pressure field: a = -f tau (gamma - 1) grad u,
  tau a lattice sum;
- at alpha_V = 0 the force loop's du_i/dt equals -f_i P_i div_v_i / rho_i, with
  div_v_i from the density loop (the pressure term ties the two loops);
- one kick-drift-kick step of two particles, every stage by hand (smoothing
  length from scipy's brentq on the partition condition).

Each of these fails when the pressure term reads P/rho instead of P/rho^2, when
nu/2 becomes nu in both a and du/dt, or when f is dropped: errors that pair
antisymmetry and energy conservation cannot see."""
import math

import numpy as np
import pytest

sp = pytest.importorskip("sympy")
from scipy.optimize import brentq  # noqa: E402

from paper_2305_13380_gb300 import inputs  # noqa: E402

GAMMA_K = 1.825742


class Spline:
    """The cubic spline of Sec. 3.1 in the H-normalised convention, W(r, h) =
    w(r/H)/H^3, H = gamma_K h, and its derivatives by symbolic differentiation."""

    def __init__(self):
        xi, yi, zi, xj, yj, zj, h, r = sp.symbols("xi yi zi xj yj zj h r", real=True)
        q = sp.Symbol("q", nonnegative=True)
        w = sp.Piecewise((16 / sp.pi * ((1 - q) ** 3 - 4 * (sp.Rational(1, 2) - q) ** 3),
                          q < sp.Rational(1, 2)),
                         (16 / sp.pi * (1 - q) ** 3, q < 1), (0, True))
        H = GAMMA_K * h
        Wr = w.subs(q, r / H) / H ** 3
        dist = sp.sqrt((xi - xj) ** 2 + (yi - yj) ** 2 + (zi - zj) ** 2)
        Wx = Wr.subs(r, dist)
        args = (xi, yi, zi, xj, yj, zj, h)
        self._W = sp.lambdify((r, h), Wr, "math")
        self._dWdh = sp.lambdify((r, h), sp.diff(Wr, h), "math")
        self._grad = [sp.lambdify(args, sp.diff(Wx, v), "math") for v in (xi, yi, zi)]

    def W(self, r, h):
        return float(self._W(r, h))

    def dWdh(self, r, h):
        return float(self._dWdh(r, h))

    def grad(self, xi, xj, h):
        """grad with respect to x_i of W(|x_i - x_j|, h)."""
        if np.array_equal(xi, xj):
            return np.zeros(3)
        a = tuple(float(v) for v in (*xi, *xj, h))
        return np.array([float(g(*a)) for g in self._grad])


@pytest.fixture(scope="module")
def K():
    return Spline()


def _pair_terms(K, i, j, X, V, m, st, alpha_v, beta_v=3.0):
    """Contribution of source j to a_i and du_i/dt, and v_sig,ij: the
    "Minimal" equation of motion and energy equation with the artificial
    viscosity of eqs. "basicartvisc"-"nuij" (viscosity symmetrised in B and
    with the mean density, as read for the oracle)."""
    xij = X[i] - X[j]
    vij = V[i] - V[j]
    r = float(np.sqrt(xij @ xij))
    Hi, Hj = GAMMA_K * st["h"][i], GAMMA_K * st["h"][j]
    if not r < max(Hi, Hj):
        return np.zeros(3), 0.0, None
    gi = K.grad(X[i], X[j], st["h"][i])   # grad_i W_ij(h_i)
    gj = K.grad(X[i], X[j], st["h"][j])   # grad_i W_ij(h_j)
    mu = min(vij @ xij, 0.0) / r
    vsig = st["c"][i] + st["c"][j] - beta_v * mu
    alpha = alpha_v * 0.5 * (st["B"][i] + st["B"][j])
    nu = -alpha * mu * vsig / (0.5 * (st["rho"][i] + st["rho"][j]))
    Pi = st["f"][i] * st["P"][i] / st["rho"][i] ** 2
    Pj = st["f"][j] * st["P"][j] / st["rho"][j] ** 2
    visc = st["f"][i] * gi + st["f"][j] * gj
    a = -m[j] * (Pi * gi + Pj * gj + 0.5 * nu * visc)
    du = m[j] * (Pi * (vij @ gi) + 0.25 * nu * (vij @ visc))
    return a, du, vsig


def _force_by_hand(K, X, V, m, st, alpha_v):
    n = len(m)
    a = np.zeros((n, 3))
    du = np.zeros(n)
    vs = np.zeros(n)
    for i in range(n):
        for j in range(n):
            if j == i:
                continue
            ai, di, si = _pair_terms(K, i, j, X, V, m, st, alpha_v)
            a[i] += ai
            du[i] += di
            if si is not None:
                vs[i] = max(vs[i], si)
    return a, du, vs


def _pair_input(dx, dy, dvx, dvy):
    L = 10.0
    p = dict(L=L, x=np.array([5.0, 5.0 + dx]), y=np.array([5.0, 5.0 + dy]), z=np.array([5.0, 5.0]),
             vx=np.array([0.1, 0.1 + dvx]), vy=np.array([0.0, dvy]), vz=np.zeros(2),
             m=np.array([1.0, 2.0]), u=np.array([1.0, 1.5]))
    st = dict(h=np.array([0.6, 0.4]), rho=np.array([1.2, 1.6]), f=np.array([0.95, 1.05]),
              P=np.array([0.8, 1.6]), c=np.array([1.0, 1.2]), B=np.array([0.5, 0.9]))
    return p, st


def _xv(p):
    X = np.stack([p["x"], p["y"], p["z"]], 1)
    V = np.stack([p["vx"], p["vy"], p["vz"]], 1)
    return X, V


@pytest.mark.parametrize("case", [
    (0.5, 0.0, -0.7, 0.0),    # approaching head on: viscosity on
    (0.5, 0.0, +0.7, 0.0),    # receding: pressure only
    (0.3, 0.25, -0.4, 0.3),   # oblique approach, r < H_j < H_i
    (0.9, 0.0, -0.5, 0.0),    # H_j < r < H_i: only h_i's kernel reaches
])
@pytest.mark.parametrize("alpha_v", [0.8, 0.0])
def test_pair_force_by_hand(orc, K, case, alpha_v):
    p, st = _pair_input(*case)
    X, V = _xv(p)
    a, du, vs = _force_by_hand(K, X, V, p["m"], st, alpha_v)
    f = orc.force(p, st, phys=orc.Physics(alpha_v=alpha_v))
    got = np.stack([f["ax"], f["ay"], f["az"]], 1)
    scale = np.abs(a).max()
    assert scale > 0
    assert np.allclose(got, a, rtol=1e-12, atol=1e-13 * scale)
    assert np.allclose(f["du_dt"], du, rtol=1e-12, atol=1e-13 * np.abs(du).max())
    assert np.allclose(f["v_sig"], vs, rtol=1e-14)


def test_pair_by_hand_values(K):
    """The head-on approaching case written out as numbers, so that the hand
    evaluation itself is pinned: with r = 0.5, H_i = 1.0954452, H_j = 0.7302968,
    q_i = 0.4564355, q_j = 0.6846532."""
    p, st = _pair_input(0.5, 0.0, -0.7, 0.0)
    X, V = _xv(p)
    # w'(q) of the cubic spline: (16/pi)(-3 (1-q)^2 + 12 (1/2-q)^2) below 1/2,
    # (16/pi)(-3 (1-q)^2) above
    qi, qj = 0.5 / (GAMMA_K * 0.6), 0.5 / (GAMMA_K * 0.4)
    wpi = 16 / math.pi * (-3 * (1 - qi) ** 2 + 12 * (0.5 - qi) ** 2)
    wpj = 16 / math.pi * (-3 * (1 - qj) ** 2)
    dWi = wpi / (GAMMA_K * 0.6) ** 4
    dWj = wpj / (GAMMA_K * 0.4) ** 4
    # x_12 = -0.5 along x: grad_1 W = dW/dr * (-1, 0, 0)
    assert K.grad(X[0], X[1], 0.6)[0] == pytest.approx(-dWi, rel=1e-13)
    assert K.grad(X[0], X[1], 0.4)[0] == pytest.approx(-dWj, rel=1e-13)
    # mu = v_12 . x_12 / r = (0.7 * -0.5) / 0.5 = -0.7; v_sig = 1 + 1.2 + 3 * 0.7;
    # alpha = 0.8 (0.5 + 0.9)/2 = 0.56; nu = -alpha mu v_sig / ((1.2 + 1.6)/2) = 1.204
    mu, vsig = -0.7, 4.3
    nu = -0.56 * mu * vsig / 1.4
    assert nu == pytest.approx(1.204, rel=1e-14)
    a1 = -2.0 * (0.95 * 0.8 / 1.44 * (-dWi) + 1.05 * 1.6 / 2.56 * (-dWj)
                 + 0.5 * nu * (0.95 * (-dWi) + 1.05 * (-dWj)))
    a, du, vs = _force_by_hand(K, X, V, p["m"], st, 0.8)
    assert a[0, 0] == pytest.approx(a1, rel=1e-13)
    # v_12 = +0.7 along x, so v_12 . grad_1 W_12(h) = 0.7 * (-dW/dr(h)) > 0
    du1 = 2.0 * (0.95 * 0.8 / 1.44 * 0.7 * (-dWi) + 0.25 * nu * 0.7 * (0.95 * (-dWi) + 1.05 * (-dWj)))
    assert du[0] == pytest.approx(du1, rel=1e-13)
    assert vs[0] == pytest.approx(vsig, rel=1e-15)
    # the numbers themselves (pressure pushes particle 1 to -x; the approach heats it)
    assert a1 == pytest.approx(-20.4814044755, rel=1e-10)
    assert du1 == pytest.approx(5.8431301973, rel=1e-10)


def test_linear_pressure_on_a_lattice(orc, K):
    """Perfect lattice at rest, u = u0 + g x: with h, rho and f uniform,
    a_x = -(f/rho^2) sum_j m_j (P_j - P_i) dW/dx_i = -f tau (gamma - 1) g, with
    the lattice sum tau = -(1/rho) sum_j m_j dx_j^2 W'(r_j)/r_j, and a_y = a_z =
    du/dt = 0 (particles farther than H from the jump of u at the box edge)."""
    n = 12
    p = inputs.lattice(n, jitter=0.0, sigma_v=0.0, u_noise=0.0)
    N = n ** 3
    p["m"] = np.full(N, 3.0 / N)          # rho ~ 3: P/rho^2 and P/rho differ
    g = 0.8
    p["u"] = 1.0 + g * np.asarray(p["x"])
    phys = orc.Physics()
    d = orc.density(p, p["h0"], phys=phys)
    h = float(d["h"][0])
    assert np.allclose(d["h"], h, rtol=1e-12)
    # lattice sums by hand at that h
    dsp = 1.0 / n
    k = np.arange(-4, 5)
    Kv = np.array(np.meshgrid(k, k, k, indexing="ij")).reshape(3, -1).T * dsp
    m = 3.0 / N
    rho = sum(m * K.W(float(np.sqrt(v @ v)), h) for v in Kv)
    drho = sum(m * K.dWdh(float(np.sqrt(v @ v)), h) for v in Kv)
    f = 1.0 / (1.0 + h / (3.0 * rho) * drho)
    # grad_i W_ij with x_i = 0, x_j = v is -W'(r) v / r, so tau = sum m v_x grad_x / rho
    tau = sum(m * v[0] * K.grad(np.zeros(3), v, h)[0] for v in Kv) / rho
    assert rho == pytest.approx(float(d["rho"][0]), rel=1e-12)
    assert f == pytest.approx(float(d["f"][0]), rel=1e-11)
    assert abs(tau - 1.0) < 0.05 and abs(f - 1.0) > 1e-4
    gam = phys.gamma
    ax = -f * tau * (gam - 1.0) * g
    F = orc.force(p, d, phys=phys)
    x = np.asarray(p["x"])
    mid = (x > 0.25) & (x < 0.75)
    assert np.allclose(F["ax"][mid], ax, rtol=1e-10)
    for key in ("ay", "az", "du_dt"):
        assert np.all(np.abs(F[key][mid]) < 1e-10 * abs(ax)), key


@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_energy_equation_is_the_density_divergence(orc, kind):
    """At alpha_V = 0, du_i/dt = sum_j m_j f_i P_i/rho_i^2 v_ij . grad_i W_ij(h_i)
    and rho_i div_v_i = -sum_j m_j v_ij . grad_i W_ij(h_i), so du_i/dt =
    -f_i P_i div_v_i / rho_i: the force loop's pressure term against the density
    loop's velocity divergence."""
    if kind == "lattice":
        p = inputs.lattice(10, seed=7, sigma_v=0.3)
    else:
        p = inputs.clustered(1500, n_spheres=3, seed=13, sigma_v=0.3)
    phys = orc.Physics(alpha_v=0.0)
    d = orc.density(p, p["h0"], phys=phys)
    F = orc.force(p, d, phys=phys)
    want = -d["f"] * d["P"] * d["div_v"] / d["rho"]
    scale = np.abs(want).max()
    assert scale > 0
    assert np.allclose(F["du_dt"], want, rtol=1e-10, atol=1e-12 * scale)


def _solve_h(K, i, X, m, eta):
    """The unique root of n_hat_i(h) h^3 = eta^3, n_hat_i = sum_j W(r_ij, h)
    (self included), by brentq."""
    r = [float(np.sqrt((X[i] - X[j]) @ (X[i] - X[j]))) for j in range(len(m))]

    def F(h):
        return sum(K.W(rj, h) for rj in r) * h ** 3 - eta ** 3
    return brentq(F, 1e-3, 5.0, xtol=1e-15, rtol=1e-15)


def _density_by_hand(K, X, V, m, u, eta, gam=5.0 / 3.0, eps=1e-4):
    n = len(m)
    st = {k: np.zeros(n) for k in ("h", "rho", "f", "P", "c", "B", "div")}
    for i in range(n):
        h = _solve_h(K, i, X, m, eta)
        rho = drho = 0.0
        div = np.zeros(1)[0]
        curl = np.zeros(3)
        for j in range(n):
            r = float(np.sqrt((X[i] - X[j]) @ (X[i] - X[j])))
            rho += m[j] * K.W(r, h)
            drho += m[j] * K.dWdh(r, h)
            gw = K.grad(X[i], X[j], h)
            div += m[j] * (V[j] - V[i]) @ gw
            curl += m[j] * np.cross(V[j] - V[i], gw)
        div /= rho
        curl /= rho
        P = (gam - 1.0) * u[i] * rho
        c = math.sqrt(gam * P / rho)
        st["h"][i], st["rho"][i], st["div"][i] = h, rho, div
        st["f"][i] = 1.0 / (1.0 + h / (3.0 * rho) * drho)
        st["P"][i], st["c"][i] = P, c
        st["B"][i] = abs(div) / (abs(div) + float(np.sqrt(curl @ curl)) + eps * c / h)
    return st


def test_two_particle_step_by_hand(orc, K):
    """One kick-drift-kick step of two particles (eta = 0.9, so that a pair
    satisfies the partition condition): dt from the previous v_sig, half kick,
    drift, prediction, density and force at the predicted state, half kick."""
    # a small CFL factor: the pair's viscous kick must not reverse the approach
    eta, cfl = 0.9, 0.01
    X = np.array([[5.0, 5.0, 5.0], [5.45, 5.1, 5.0]])
    V = np.array([[1.5, 0.0, 0.05], [-1.2, 0.4, 0.0]])
    m = np.array([1.0, 1.5])
    u = np.array([1.0, 2.0])
    phys = orc.Physics(eta=eta)
    # the previous force evaluation, by hand
    st0 = _density_by_hand(K, X, V, m, u, eta)
    a0, du0, vs0 = _force_by_hand(K, X, V, m, st0, phys.alpha_v)
    # the step by hand
    dt = min(cfl * GAMMA_K * st0["h"] / vs0)
    Vh = V + 0.5 * dt * a0
    uh = u + 0.5 * dt * du0
    X1 = X + Vh * dt
    Vp = Vh + 0.5 * dt * a0
    up = uh + 0.5 * dt * du0
    st1 = _density_by_hand(K, X1, Vp, m, up, eta)
    a1, du1, vs1 = _force_by_hand(K, X1, Vp, m, st1, phys.alpha_v)
    V1 = Vh + 0.5 * dt * a1
    u1 = uh + 0.5 * dt * du1
    # the oracle's step from the same state
    s = dict(L=10.0, x=X[:, 0].copy(), y=X[:, 1].copy(), z=X[:, 2].copy(),
             vx=V[:, 0].copy(), vy=V[:, 1].copy(), vz=V[:, 2].copy(), m=m.copy(), u=u.copy(),
             h=st0["h"].copy(), ax=a0[:, 0].copy(), ay=a0[:, 1].copy(), az=a0[:, 2].copy(),
             du_dt=du0.copy(), v_sig=vs0.copy())
    got_dt = orc.step(s, cfl, phys=phys)
    assert got_dt == pytest.approx(dt, rel=1e-14)
    assert np.allclose(np.stack([s["x"], s["y"], s["z"]], 1), X1, rtol=0, atol=1e-14)
    assert np.allclose(np.stack([s["vx"], s["vy"], s["vz"]], 1), V1, rtol=1e-11,
                       atol=1e-12 * np.abs(V1).max())
    assert np.allclose(s["u"], u1, rtol=1e-12)
    assert np.allclose(s["h"], st1["h"], rtol=1e-12)
    assert np.allclose(s["rho"], st1["rho"], rtol=1e-12)
    assert np.allclose(np.stack([s["ax"], s["ay"], s["az"]], 1), a1, rtol=1e-10,
                       atol=1e-12 * np.abs(a1).max())
    assert np.allclose(s["du_dt"], du1, rtol=1e-10, atol=1e-12 * np.abs(du1).max())
    assert np.allclose(s["v_sig"], vs1, rtol=1e-13)
    # the pair still approaches at the predicted state, so the viscosity acts
    assert (Vp[0] - Vp[1]) @ (X1[0] - X1[1]) < 0 and np.all(st1["B"] > 0.1)
    a1_inviscid = _force_by_hand(K, X1, Vp, m, st1, 0.0)[0]
    assert np.abs(a1 - a1_inviscid).max() > 0.5 * np.abs(a1_inviscid).max()


@pytest.mark.parametrize("case", [
    (0.5, 0.0, -0.7, 0.0),    # approaching: |v.x|/r adds to the conduction speed
    (0.3, 0.25, -0.4, 0.3),   # oblique, r < H_j < H_i
    (0.9, 0.0, -0.5, 0.0),    # H_j < r < H_i: only h_i's kernel reaches
])
def test_conduction_by_hand(orc, K, case):
    """SPHENIX artificial conduction (Sec. 3.3, eq. "art_cond"), two particles:
    du_i/dt|cond = alpha_c,ij v_c,ij m_j (u_i - u_j) [f_i grad_i W(h_i) +
    f_j grad_i W(h_j)] . x_ij / r / (rho_i + rho_j), with the pressure-weighted
    alpha_c,ij and v_c,ij = |v_ij . x_ij| / r + sqrt(2 |P_i - P_j| /
    (rho_i + rho_j)) (the readings of the garbled terms), against the oracle's
    conduction part of du/dt.  A dropped 1/2-weighting, a wrong density sum or
    a swapped sign of (u_i - u_j) changes these values."""
    p, st = _pair_input(*case)
    X, V = _xv(p)
    alpha_c = np.array([0.3, 0.9])
    alpha_v = np.array([0.5, 1.0])
    out = orc.sphenix_force(p, st, alpha_v, alpha_c)
    for i, j in ((0, 1), (1, 0)):
        xij = X[i] - X[j]
        vij = V[i] - V[j]
        r = float(np.sqrt(xij @ xij))
        gi = K.grad(X[i], X[j], st["h"][i]) @ xij / r
        gj = K.grad(X[i], X[j], st["h"][j]) @ xij / r
        a_c = (st["P"][i] * alpha_c[i] + st["P"][j] * alpha_c[j]) / (st["P"][i] + st["P"][j])
        rs = st["rho"][i] + st["rho"][j]
        v_c = abs(vij @ xij) / r + math.sqrt(2.0 * abs(st["P"][i] - st["P"][j]) / rs)
        du = a_c * v_c * p["m"][j] * (p["u"][i] - p["u"][j]) * (st["f"][i] * gi + st["f"][j] * gj) / rs
        assert out["du_cond"][i] == pytest.approx(du, rel=1e-10, abs=1e-14)
    # heat flows from the hotter particle (u = 1.5) to the colder one
    assert out["du_cond"][1] < 0.0 < out["du_cond"][0]
    # energy: m_i du_i + m_j du_j = 0
    assert p["m"] @ out["du_cond"] == pytest.approx(0.0, abs=1e-12)


def test_sphenix_viscosity_by_hand(orc, K):
    """SPHENIX viscosity (Sec. 3.3, eq. "av_ij"): the pair's alpha is the mean
    of the two particles' alpha_V times the mean Balsara switch; with the
    conduction off (equal u) the SPHENIX a and du/dt of two approaching
    particles are the hand-evaluated Minimal pair terms with that alpha."""
    p, st = _pair_input(0.3, 0.25, -0.4, 0.3)
    p["u"] = np.array([1.2, 1.2])                 # no conduction
    X, V = _xv(p)
    alpha_v = np.array([0.4, 1.6])
    out = orc.sphenix_force(p, st, alpha_v, np.zeros(2))
    for i, j in ((0, 1), (1, 0)):
        B = st["B"]
        # _pair_terms takes alpha_V (B_i + B_j)/2: pass the mean alpha_V
        a, du, _ = _pair_terms(K, i, j, X, V, p["m"], st, 0.5 * (alpha_v[i] + alpha_v[j]))
        for k, ax in enumerate(("ax", "ay", "az")):
            assert out[ax][i] == pytest.approx(a[k], rel=1e-10, abs=1e-13)
        assert out["du_dt"][i] == pytest.approx(du, rel=1e-10, abs=1e-13)
        assert B[i] != B[j]
    # a single alpha_V (either particle's) gives other values
    a0, _, _ = _pair_terms(K, 0, 1, X, V, p["m"], st, alpha_v[0])
    assert abs(out["ax"][0] - a0[0]) > 1e-6 * abs(a0[0])
