"""Pins of the oracle's kernel (Sec. 3.1, eq. "kernel") against properties
the paper and the textbook cubic spline fix, not against its own formula."""
import math

import numpy as np
import pytest
from scipy import integrate


def test_normalised(orc):
    # The kernel must be normalised (Sec. 3.1): 4 pi int_0^1 q^2 w(q) dq = 1.
    val, err = integrate.quad(lambda q: 4.0 * math.pi * q * q * orc.w(q), 0.0, 1.0,
                              points=[0.5], epsabs=1e-13, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-12


def test_textbook_values(orc):
    # M4 cubic spline with compact support H: sigma = 8/pi, w(1/2) = sigma/4.
    assert orc.w(0.0) == pytest.approx(8.0 / math.pi, rel=1e-15)
    assert orc.w(0.5) == pytest.approx(2.0 / math.pi, rel=1e-15)
    assert orc.w(1.0) == 0.0
    assert orc.w(1.3) == 0.0
    assert orc.dw_dq(1.0) == 0.0


def test_zero_central_gradient(orc):
    # "must have a central gradient of zero" (Sec. 3.1)
    assert orc.dw_dq(0.0) == 0.0


def test_derivative_matches_finite_difference(orc):
    for q in np.linspace(0.01, 0.99, 57):
        if abs(q - 0.5) < 1e-3:
            continue
        d = 1e-6
        fd = (orc.w(q + d) - orc.w(q - d)) / (2 * d)
        assert orc.dw_dq(q) == pytest.approx(fd, rel=1e-7, abs=1e-8)


def test_smooth_at_half_and_edge(orc):
    # cubic spline: w, w', w'' continuous at q = 1/2; w, w' vanish at q = 1
    e = 1e-9
    assert orc.w(0.5 - e) == pytest.approx(orc.w(0.5 + e), abs=1e-7)
    assert orc.dw_dq(0.5 - e) == pytest.approx(orc.dw_dq(0.5 + e), abs=1e-7)
    d = 1e-5
    w2_lo = (orc.dw_dq(0.5 - d) - orc.dw_dq(0.5 - 2 * d)) / d
    w2_hi = (orc.dw_dq(0.5 + 2 * d) - orc.dw_dq(0.5 + d)) / d
    assert w2_lo == pytest.approx(w2_hi, rel=1e-3)
    assert orc.w(1.0 - 1e-6) < 1e-16
    assert abs(orc.dw_dq(1.0 - 1e-6)) < 1e-10


def test_monotone_decreasing(orc):
    qs = np.linspace(0.0, 1.0, 1001)
    w = np.array([orc.w(q) for q in qs])
    assert np.all(np.diff(w) <= 0.0)


def test_gamma_k_gives_about_48_neighbours(orc):
    # eta = 1.2348 corresponds to ~48 neighbours, N_ngb = 4 pi/3 (gamma_K eta)^3
    nngb = 4.0 * math.pi / 3.0 * (orc.GAMMA_K * 1.2348) ** 3
    assert abs(nngb - 48.0) < 0.01
    assert orc.lib().oracle_gamma_k() == orc.GAMMA_K
