"""Pins of the oracle's time bins and first time-step limiter (Sec. 2.4 and
the time-step limiter of the SPH section): power-of-two steps below the CFL
step, one bin per factor of two, and neighbours at most two bins apart after
the limiter."""
import numpy as np

import oracle


def test_bins_are_the_largest_power_of_two_step_below_cfl():
    rng = np.random.default_rng(1)
    h = rng.uniform(0.5, 2.0, 500).astype(np.float32)
    v = rng.uniform(0.5, 50.0, 500).astype(np.float32)
    b = oracle.time_bins(h, v, 0.1, 1.0, 20)
    dt = 0.1 * oracle.GAMMA_K * h.astype(np.float64) / v
    step = 2.0 ** -b.astype(np.float64)
    assert np.all(step <= dt * (1 + 1e-6)) and np.all(2 * step > dt * (1 - 1e-6))


def test_bins_follow_h_and_v_by_factors_of_two():
    h = np.full(8, 1.0, np.float32)
    v = np.float32(1.0) * 2.0 ** np.arange(8, dtype=np.float32)
    b = oracle.time_bins(h, v, 0.1, 1.0, 30)
    assert np.all(np.diff(b) == 1)            # twice the speed: half the step
    assert np.array_equal(oracle.time_bins(2 * h, 2 * v, 0.1, 1.0, 30), b)
    assert np.all(oracle.time_bins(h, v, 0.1, 1e9, 3) == 3)   # capped at max_bin
    assert np.all(oracle.time_bins(h, np.zeros(8, np.float32), 0.1, 1.0, 5) == 0)


def test_limiter_keeps_neighbours_within_two_bins():
    from paper_2305_13380_gb300 import inputs
    p = inputs.lattice(8, seed=2)
    n = len(p["x"])
    h = np.asarray(p["h0"], np.float64)
    bins = np.zeros(n, np.int32)
    bins[0] = 9                                   # one particle on a short step
    out = oracle.limit_time_bins(p, h, bins)
    d = [(np.asarray(p[k]) - p[k][0] + 0.5) % 1.0 - 0.5 for k in "xyz"]
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    H = oracle.GAMMA_K * h
    near = (r < H) & (np.arange(n) != 0)
    assert out[0] == 9
    assert np.all(out[near] == 7) and np.all(out[~near & (np.arange(n) != 0)] == 0)
    # applied once: a second pass spreads the short step one shell further
    out2 = oracle.limit_time_bins(p, h, out)
    assert out2.max() == 9 and (out2 == 5).sum() > 0
