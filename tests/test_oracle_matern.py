"""Pins for the oracle's Matern covariance and its partials (CPU only): closed forms at
nu = 1/2, 3/2, 5/2, the value at h = 0, and extended-precision derivatives of an independent
mpmath restatement of C(h; theta)."""
import math

import numpy as np
import pytest

from oracle import matern
from paper_2601_11437_gb300 import inputs


def test_closed_forms_half_integer_nu():
    h = np.array([1e-5, 0.01, 0.05, 0.2, 0.6, 1.3])
    alpha, s2 = 0.07, 1.7
    x = h / alpha
    for nu, poly in ((0.5, 1.0), (1.5, 1.0 + x), (2.5, 1.0 + x + x * x / 3.0)):
        R, _, _ = matern.correlation_parts(x, alpha, nu, partials=False)
        np.testing.assert_allclose(s2 * R, s2 * poly * np.exp(-x), rtol=1e-13)


def test_value_and_partials_at_zero_distance():
    R, dRa, dRn = matern.correlation_parts(np.zeros(3), 0.1, 0.8)
    assert np.all(R == 1.0) and np.all(dRa == 0.0) and np.all(dRn == 0.0)


def test_dalpha_closed_form_nu_half():
    # nu = 1/2: C = s2 exp(-h/alpha), dC/dalpha = s2 h / alpha^2 exp(-h/alpha)
    h = np.array([0.003, 0.05, 0.4, 1.2])
    alpha, s2 = 0.11, 0.9
    _, dRa, _ = matern.correlation_parts(h / alpha, alpha, 0.5)
    np.testing.assert_allclose(s2 * dRa, s2 * h / alpha ** 2 * np.exp(-h / alpha), rtol=1e-13)


def _mp_matern(mpmath, h, s2, alpha, nu):
    x = h / alpha
    return s2 * x ** nu * mpmath.besselk(nu, x) / (2 ** (nu - 1) * mpmath.gamma(nu))


@pytest.mark.parametrize("nu", [0.13, 0.5, 0.8, 1.0, 1.2, 1.5, 2.3])
def test_partials_against_mpmath_derivatives(nu):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    s2, alpha = 1.3, 0.08
    h = np.array([1e-4, 0.004, 0.03, 0.1, 0.35, 0.68, 1.1, 2.5])
    x = h / alpha
    R, dRa, dRn = matern.correlation_parts(x, alpha, nu)
    for i, hh in enumerate(h):
        c = float(_mp_matern(mpmath, mpmath.mpf(hh), s2, mpmath.mpf(alpha), mpmath.mpf(nu)))
        da = float(mpmath.diff(lambda a: _mp_matern(mpmath, mpmath.mpf(hh), s2, a, mpmath.mpf(nu)), alpha))
        dn = float(mpmath.diff(lambda v: _mp_matern(mpmath, mpmath.mpf(hh), s2, mpmath.mpf(alpha), v), nu))
        assert s2 * R[i] == pytest.approx(c, rel=1e-13, abs=1e-300)
        assert s2 * dRa[i] == pytest.approx(da, rel=1e-12, abs=1e-300)
        assert s2 * dRn[i] == pytest.approx(dn, rel=1e-11, abs=1e-14 * s2)


def test_paper_mode_matrices_close_to_exact():
    locs = inputs.uniform_locations(120, 3)
    for theta in ((1.0, 0.1, 0.8), (2.0, 0.05, 1.7), (0.7, 0.3, 0.35)):
        ex = matern.covariance(locs, theta, dnu="exact")
        pa = matern.covariance(locs, theta, dnu="paper")
        np.testing.assert_array_equal(ex["S"], pa["S"])
        err = np.max(np.abs(ex["S_nu"] - pa["S_nu"])) / np.max(np.abs(ex["S_nu"]))
        # the paper's truncated series are good to about 1e-8 relative near x = 8.5 (cases 2-3)
        assert err < 1e-8


def test_covariance_structure_and_jitter_modes():
    locs = inputs.uniform_locations(50, 11)
    th = (1.7, 0.2, 1.3)
    m0 = matern.covariance(locs, th, jitter=1e-8, mode=0)
    m1 = matern.covariance(locs, th, jitter=1e-8, mode=1)
    for M in (m0["S"], m0["S_alpha"], m0["S_nu"]):
        np.testing.assert_array_equal(M, M.T)
    np.testing.assert_allclose(np.diag(m0["S"]), th[0] * (1 + 1e-8), rtol=1e-15)
    np.testing.assert_allclose(np.diag(m1["S"]), th[0] + 1e-8, rtol=1e-15)
    assert np.all(np.diag(m0["S_alpha"]) == 0) and np.all(np.diag(m0["S_nu"]) == 0)
    np.testing.assert_allclose(m0["S_sigma2"], m0["S"] / th[0], rtol=1e-15)
    np.testing.assert_allclose(m1["S_sigma2"] * th[0] + 1e-8 * np.eye(50), m1["S"], rtol=1e-14, atol=1e-22)
    # Sigma_alpha and Sigma_nu do not depend on the jitter
    np.testing.assert_array_equal(m0["S_alpha"], m1["S_alpha"])
    np.testing.assert_array_equal(m0["S_nu"], m1["S_nu"])
