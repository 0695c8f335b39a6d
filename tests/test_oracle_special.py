"""Pins for the oracle's K_nu, dK_nu/dnu and digamma against closed forms, recurrences,
extended-precision library routines and special cases (CPU only)."""
import math

import numpy as np
import pytest

from oracle import special

XS = np.array([1e-8, 1e-4, 0.013, 0.2, 0.7, 1.0, 2.5, 6.0, 8.49, 8.5, 14.0, 15.0, 29.9, 30.0,
               57.0, 120.0, 400.0, 700.0])


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b)))


def test_k_half_integer_closed_forms():
    # DLMF 10.39.2 and the recurrence: K_1/2, K_3/2, K_5/2 are elementary
    x = XS[XS < 700]
    base = np.sqrt(math.pi / (2 * x)) * np.exp(-x)
    assert rel(special.bessel_k(0.5, x), base) < 1e-13
    assert rel(special.bessel_k(1.5, x), base * (1 + 1 / x)) < 1e-13
    assert rel(special.bessel_k(2.5, x), base * (1 + 3 / x + 3 / x ** 2)) < 1e-13
    assert rel(special.bessel_k(-0.5, x), base) < 1e-13          # K is even in its order


@pytest.mark.parametrize("nu", [0.05, 0.3, 0.8, 1.0, 1.2, 1.7, 2.5, 3.3])
def test_k_recurrence(nu):
    # DLMF 10.29.1: K_(nu+1) - K_(nu-1) = (2 nu / x) K_nu
    x = XS[(XS > 1e-3) & (XS < 500)]
    kp, km = special.bessel_k(nu + 1, x), special.bessel_k(nu - 1, x)
    rhs = 2 * nu / x * special.bessel_k(nu, x)
    # the difference cancels for small nu or large x: bound the error by the operands' size
    assert np.all(np.abs((kp - km) - rhs) <= 5e-14 * (kp + km))


@pytest.mark.parametrize("nu", [0.0, 0.1, 0.37, 0.5, 0.999999, 1.0, 1.2, 2.0, 2.71])
def test_k_against_mpmath(nu):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    x = XS[XS < 700]
    ref = np.array([float(mpmath.besselk(nu, xx)) for xx in x])
    assert rel(special.bessel_k(nu, x), ref) < 2e-14


def test_k_against_scipy():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(7)
    nu = rng.uniform(0, 4, 40)
    for v in nu:
        x = rng.uniform(1e-3, 60, 25)
        assert rel(special.bessel_k(v, x), sp.kv(v, x)) < 2e-13   # scipy (Amos) is good to ~1e-14


@pytest.mark.parametrize("nu", [0.05, 0.5, 1.2, 2.5, 3.7])
def test_k_wronskian_with_i(nu):
    # DLMF 10.28.2: I_nu(x) K_(nu+1)(x) + I_(nu+1)(x) K_nu(x) = 1 / x.  I_nu comes from scipy, an
    # independent routine; scaled forms (ive e^x, K e^-x cancel) keep large x in range
    sp = pytest.importorskip("scipy.special")
    x = XS[(XS >= 1e-4) & (XS <= 400)]
    lhs = (sp.ive(nu, x) * special.bessel_k(nu + 1, x) + sp.ive(nu + 1, x) * special.bessel_k(nu, x)) * np.exp(x)
    assert rel(lhs, 1 / x) < 1e-13


def test_dnu_at_zero_order_vanishes():
    # K_nu is even in nu, so dK/dnu = 0 at nu = 0
    assert np.all(special.bessel_k_dnu(0.0, XS) == 0.0)


def test_dnu_half_closed_form():
    # DLMF 10.38.7: dK_nu/dnu at nu = 1/2 equals sqrt(pi/(2x)) E_1(2x) e^x
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    x = XS[(XS > 1e-6) & (XS < 300)]
    ref = np.array([float(mpmath.sqrt(mpmath.pi / (2 * xx)) * mpmath.e1(2 * xx) * mpmath.exp(xx)) for xx in x])
    assert rel(special.bessel_k_dnu(0.5, x), ref) < 2e-14


def test_dnu_integer_order_one():
    # DLMF 10.38.5 at n = 1: dK_nu/dnu at nu = 1 equals K_0(x) / x
    x = XS[XS < 700]
    assert rel(special.bessel_k_dnu(1.0, x), special.bessel_k(0.0, x) / x) < 1e-13


@pytest.mark.parametrize("nu", [0.13, 0.5, 0.8, 1.0, 1.2, 1.5, 2.4])
def test_dnu_against_mpmath_derivative(nu):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    x = XS[(XS > 1e-6) & (XS < 300)]
    ref = np.array([float(mpmath.diff(lambda v: mpmath.besselk(v, xx), nu)) for xx in x])
    assert rel(special.bessel_k_dnu(nu, x), ref) < 5e-14


def test_digamma_closed_forms():
    g = special.EULER_GAMMA
    assert abs(special.digamma(1.0) + g) < 1e-15
    assert abs(special.digamma(0.5) + g + 2 * math.log(2)) < 1e-15          # DLMF 5.4.13
    for x in (0.07, 0.6, 1.3, 4.4, 17.0):
        assert abs(special.digamma(x + 1) - special.digamma(x) - 1 / x) < 2e-14 * max(1, 1 / x)


def test_digamma_against_mpmath_including_negative_arguments():
    mpmath = pytest.importorskip("mpmath")
    for x in (0.05, 0.3, 0.8, 1.2, 2.5, 9.9, 33.0, -0.3, -0.8, -1.2, -2.5):
        assert abs(special.digamma(x) - float(mpmath.digamma(x))) < 1e-13 * max(1.0, abs(float(mpmath.digamma(x))))
    with pytest.raises(ValueError):
        special.digamma(-2.0)
