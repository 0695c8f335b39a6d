"""Cross-check of the oracle's K_nu (an integral representation, summed by the trapezoid rule)
against independent methods: Temme's series for x <= 2 and a three-term recurrence of the
confluent hypergeometric function for x >= 2.

N. M. Temme, "On the numerical evaluation of the modified Bessel function of the third kind",
J. Comput. Phys. 19 (1975) 324-337, writes K_mu and K_(mu+1) for |mu| <= 1/2 and x <= 2 as
    K_mu(x)     = sum_k c_k f_k,        K_(mu+1)(x) = (2 / x) sum_k c_k (p_k - k f_k),
    c_k = (x^2 / 4)^k / k!,
    f_k = (k f_(k-1) + p_(k-1) + q_(k-1)) / (k^2 - mu^2),
    p_k = p_(k-1) / (k - mu),           q_k = q_(k-1) / (k + mu),
    p_0 = (x / 2)^(-mu) Gamma(1 + mu) / 2,   q_0 = (x / 2)^mu Gamma(1 - mu) / 2,
    f_0 = (pi mu / sin(pi mu)) [cosh(s) G1(mu) + ln(2 / x) (sinh(s) / s) G2(mu)],  s = mu ln(2 / x),
    G1(mu) = (1 / Gamma(1 - mu) - 1 / Gamma(1 + mu)) / (2 mu),
    G2(mu) = (1 / Gamma(1 - mu) + 1 / Gamma(1 + mu)) / 2.
Orders above 3/2 follow from the upward recurrence K_(v+1) = K_(v-1) + (2 v / x) K_v (DLMF
10.29.1), which is stable for K.  Every term of these sums is positive for x <= 2, so the series is
accurate to a few units of rounding.  This is the small-argument region, where the integrand of
the integral representation decays slowest.  G1 and G2 are evaluated with mpmath at 40 digits
(their two reciprocal gammas cancel for small mu); the rest is FP64.

For x >= 2 the check goes through the confluent hypergeometric function,
K_nu(x) = sqrt(pi) (2x)^nu e^-x U(nu + 1/2, 2 nu + 1, 2x).  With
V_k = Gamma(nu + 1/2 + k) U(nu + 1/2 + k, 2 nu + 1, 2x)
    = int_0^inf e^(-2xt) t^(nu-1/2) (1+t)^(nu-1/2) (t / (1+t))^k dt,
the contiguous relation of U (DLMF 13.3.7) becomes
    (k + nu - 1/2) V_(k-1) - 2 (k + x) V_k + (k + 1/2 - nu) V_(k+1) = 0,
whose decaying solution is found by backward recurrence from a large k (Miller's algorithm), and
expanding (1 - t/(1+t))^(nu - 1/2) under the integral gives the normalisation
    sum_k ((1/2 - nu)_k / k!) V_k = Gamma(nu + 1/2) (2x)^(-nu-1/2),
so that K_nu(x) = sqrt(pi / (2x)) e^-x v_0 / sum_k ((1/2 - nu)_k / k!) v_k for the unnormalised
values v_k of the recurrence.  This is written here from those identities, for any nu >= 0.
"""
import math

import numpy as np
import pytest

from oracle import special

mpmath = pytest.importorskip("mpmath")


def temme_k_pair(mu, x):
    """(K_mu(x), K_(mu+1)(x)) for |mu| <= 1/2, 0 < x <= 2, by Temme's series."""
    assert abs(mu) <= 0.5 and 0.0 < x <= 2.0
    with mpmath.workdps(40):
        m = mpmath.mpf(mu)
        r1, r2 = mpmath.rgamma(1 - m), mpmath.rgamma(1 + m)
        g1 = float(-mpmath.euler) if mu == 0 else float((r1 - r2) / (2 * m))
        g2 = float((r1 + r2) / 2)
    lx = math.log(2.0 / x)
    s = mu * lx
    pm = 1.0 if mu == 0 else math.pi * mu / math.sin(math.pi * mu)
    sh = 1.0 if s == 0 else math.sinh(s) / s
    f = pm * (math.cosh(s) * g1 + lx * sh * g2)
    p = 0.5 * math.exp(s) * math.gamma(1.0 + mu)      # (x/2)^(-mu) = exp(mu ln(2/x))
    q = 0.5 * math.exp(-s) * math.gamma(1.0 - mu)
    c = 1.0
    k_mu = c * f
    k_mu1 = c * p                                        # h_0 = p_0 - 0 f_0
    y = 0.25 * x * x
    for k in range(1, 200):
        f = (k * f + p + q) / (k * k - mu * mu)
        c *= y / k
        p /= k - mu
        q /= k + mu
        t_mu, t_mu1 = c * f, c * (p - k * f)
        k_mu += t_mu
        k_mu1 += t_mu1
        if abs(t_mu) < 1e-18 * abs(k_mu) and abs(t_mu1) < 1e-18 * abs(k_mu1):
            break
    return k_mu, 2.0 / x * k_mu1


def temme_k(nu, x):
    """K_nu(x) for nu >= 0, 0 < x <= 2: the series at mu = nu - round(nu), then the recurrence."""
    m = int(math.floor(nu + 0.5))
    mu = nu - m
    k0, k1 = temme_k_pair(mu, x)
    v = mu + 1.0
    for _ in range(m - 1):
        k0, k1 = k1, k0 + 2.0 * v / x * k1
        v += 1.0
    return k0 if m == 0 else k1


def test_temme_series_itself_against_mpmath():
    # the test's own series, before it is used as a pin
    for nu in (0.0, 0.05, 0.5, 1.0, 1.3, 4.0):
        for x in (1e-3, 0.3, 2.0):
            ref = float(mpmath.besselk(nu, x))
            assert abs(temme_k(nu, x) - ref) <= 3e-15 * ref


NUS = [0.05, 0.1, 0.3, 0.5, 0.8, 1.0, 1.3, 1.5, 2.0, 2.5, 3.7, 4.0]
XS = [1e-6, 1e-3, 0.01, 0.1, 0.37, 0.5, 1.0, 1.5, 1.999, 2.0]


@pytest.mark.parametrize("nu", NUS)
def test_oracle_k_agrees_with_temme_series(nu):
    xs = np.array(XS)
    got = special.bessel_k(nu, xs)
    ref = np.array([temme_k(nu, x) for x in XS])
    assert np.all(np.abs(got - ref) <= 1e-14 * ref)


def miller_k(nu, x, N=400):
    """K_nu(x) for nu >= 0, x >= 2, by backward recurrence of V_k and its normalising sum."""
    assert nu >= 0 and x >= 2.0
    v = [0.0] * (N + 2)
    v[N] = 1e-30
    for k in range(N, 0, -1):
        v[k - 1] = (2.0 * (k + x) * v[k] - (k + 0.5 - nu) * v[k + 1]) / (k + nu - 0.5)
        if abs(v[k - 1]) > 1e250:                        # keep the growing values finite
            v = [t * 1e-250 for t in v]
    s, w = 0.0, 1.0
    for k in range(N + 1):
        if k > 0:
            w *= (k - 0.5 - nu) / k                      # (1/2 - nu)_k / k!
        s += w * v[k]
    return math.sqrt(math.pi / (2.0 * x)) * math.exp(-x) * v[0] / s


def test_miller_recurrence_itself_against_mpmath():
    for nu in (0.0, 0.05, 0.5, 1.3, 4.0):
        for x in (2.0, 8.49, 57.0, 600.0):
            ref = float(mpmath.besselk(nu, x))
            assert abs(miller_k(nu, x) - ref) <= 5e-15 * ref


XL = [2.0, 2.5, 5.0, 8.49, 8.5, 14.99, 15.0, 29.99, 30.0, 57.0, 120.0, 400.0, 600.0]


@pytest.mark.parametrize("nu", NUS)
def test_oracle_k_agrees_with_the_recurrence_for_large_x(nu):
    xs = np.array(XL)
    got = special.bessel_k(nu, xs)
    ref = np.array([miller_k(nu, x) for x in XL])
    assert np.all(np.abs(got - ref) <= 1e-14 * ref)
