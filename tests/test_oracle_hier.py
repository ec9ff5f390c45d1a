"""Pins of the oracle's time-step hierarchy sub-step (Sec. 2.4): with every
particle in one bin it is the global kick-drift-kick step (itself pinned),
and with two bins the long-step particles only drift until their step ends."""
import numpy as np

import oracle
from paper_2305_13380_gb300 import inputs


def _state(n_side=8, seed=3):
    p = inputs.lattice(n_side, seed=seed, sigma_v=0.05)
    q = {k: (float(v) if k == "L" else np.asarray(v, dtype=np.float64).copy()) for k, v in p.items()}
    d, f = oracle.density_force(q, q["h0"])
    s = {k: q[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u")}
    s.update(L=q["L"], h=d["h"].copy(), ax=f["ax"].copy(), ay=f["ay"].copy(), az=f["az"].copy(),
             du_dt=f["du_dt"].copy(), v_sig=f["v_sig"].copy())
    for k in ("rho", "f", "P", "c", "B", "div_v"):
        s[k] = d[k].copy()
    return s


def _half_kicked(s, dt_i):
    h = {k: s[k].copy() if isinstance(s[k], np.ndarray) else s[k] for k in s}
    for k in ("x", "y", "z"):
        h["v" + k] = s["v" + k] + s["a" + k] * 0.5 * dt_i
    h["u"] = s["u"] + s["du_dt"] * 0.5 * dt_i
    return h


def test_one_bin_is_the_global_step():
    s = _state()
    n = len(s["x"])
    dt = float(np.min(0.1 * oracle.GAMMA_K * s["h"] / s["v_sig"]))
    g = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    dt_g = oracle.step(g, 0.1)
    assert dt_g == dt
    hs = _half_kicked(s, dt)
    bins = np.zeros(n, np.int32)
    tb = np.zeros(n, np.int64)
    t = oracle.hier_substep(hs, bins, tb, dt, 0, 0, False)
    assert t == 1 and np.all(tb == 1)
    for k in ("x", "y", "z"):
        dd = np.abs(hs[k] - g[k])
        assert np.minimum(dd, 1.0 - dd).max() < 1e-14
    for k in ("vx", "vy", "vz"):
        assert np.allclose(hs[k] - hs["a" + k[-1]] * 0.5 * dt, g[k], rtol=0, atol=1e-13)
    assert np.allclose(hs["u"] - hs["du_dt"] * 0.5 * dt, g["u"], rtol=1e-13)


def test_long_steps_only_drift_until_they_end():
    s = _state()
    n = len(s["x"])
    dt_max = 2.0 * float(np.min(0.1 * oracle.GAMMA_K * s["h"] / s["v_sig"]))
    bins = np.where(np.arange(n) % 2 == 0, 1, 0).astype(np.int32)   # steps of 1 and 2 ticks
    step = 2.0 ** (1 - bins) * 0.5 * dt_max
    hs = _half_kicked(s, step)
    tb = np.zeros(n, np.int64)
    v0 = hs["vx"].copy()
    t = oracle.hier_substep(hs, bins, tb, dt_max, 1, 0, False)
    assert t == 1
    short = bins == 1
    assert np.all(tb[short] == 1) and np.all(tb[~short] == 0)
    assert np.array_equal(hs["vx"][~short], v0[~short])          # no kick on the long steps
    assert not np.array_equal(hs["vx"][short], v0[short])
    t = oracle.hier_substep(hs, bins, tb, dt_max, 1, t, False)
    assert t == 2 and np.all(tb == 2)


def test_limiter_takes_the_bins_that_inactive_neighbours_hold():
    """Adaptive bins: an active particle's new bin is limited against the bin an
    inactive neighbour holds for its current step, not against a CFL bin
    recomputed from that neighbour's last h and v_sig.  Particle b steps 16
    ticks (bin 0) with a stale signal speed whose CFL bin would be the deepest;
    the others step 8 ticks (bin 1) and end their step first."""
    s = _state()
    n = len(s["x"])
    max_bin = 4
    dt_cfl = 0.1 * oracle.GAMMA_K * s["h"] / s["v_sig"]
    dt_max = 0.5 * float(np.min(dt_cfl))        # every fresh CFL bin is 0
    b = 0
    s["v_sig"][b] *= 1e6                          # stale: its CFL bin would be 4
    assert oracle.time_bins(s["h"], s["v_sig"], 0.1, dt_max, max_bin)[b] == max_bin
    bins = np.ones(n, np.int32)
    bins[b] = 0
    tb = np.zeros(n, np.int64)
    hs = _half_kicked(s, 2.0 ** (max_bin - bins) * np.ldexp(dt_max, -max_bin))
    t = oracle.hier_substep(hs, bins, tb, dt_max, max_bin, 0, True)
    assert t == 8 and tb[b] == 0 and bins[b] == 0
    d = [(np.asarray(s[k]) - s[k][b] + 0.5) % 1.0 - 0.5 for k in "xyz"]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    H = oracle.GAMMA_K * s["h"]
    near = (r < np.maximum(H, H[b])) & (np.arange(n) != b)
    assert near.sum() > 20
    # held bin 0 limits nothing: the step of 8 ticks stays (aligned at tick 8);
    # a limiter fed with b's recomputed CFL bin (4) would force bin 2
    assert np.all(bins[near] == 1)
    assert np.all(bins[np.arange(n) != b] == 1)
