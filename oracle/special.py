"""Special functions for the oracle: K_nu, dK_nu/dnu and the digamma function, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper needs K_nu for the Matern covariance (Sec. 2.1) and for dC/dalpha, which uses K_{nu-1}
(Sec. 2.2), and d/dnu[x^nu K_nu(x)] for Sigma_nu (Supp. A).  The paper does not say which routine
evaluates K_nu itself; the oracle takes the exact function from its integral representation
    K_nu(x)        = int_0^inf exp(-x cosh t) cosh(nu t) dt            (DLMF 10.32.9)
    dK_nu/dnu (x)  = int_0^inf t sinh(nu t) exp(-x cosh t) dt          (its nu-derivative)
by the trapezoid rule, which converges geometrically for these analytic, doubly-exponentially
decaying integrands.  The step h depends on x so that the discretisation error, about
exp(-2 pi^2 / (h^2 x)) for large x and exp(-2 pi d / h) for small x, stays below 1e-30:
h = 0.1 for x <= 25 and h = 0.1 / 2^l for 25*4^(l-1) < x <= 25*4^l.  The sum runs until the
integrand is 50 e-folds below its peak.
"""
from __future__ import annotations

import math

import numpy as np

LOG2 = math.log(2.0)
EULER_GAMMA = 0.57721566490153286060651209008240243


def _logcosh(u: np.ndarray) -> np.ndarray:
    a = np.abs(u)
    return a + np.log1p(np.exp(-2.0 * a)) - LOG2


def _t_log_sinh(t: np.ndarray, mu: float) -> tuple:
    """log|t sinh(mu t)| and its sign, for t >= 0 (value -inf at t = 0 or mu = 0)."""
    a = abs(mu) * t
    with np.errstate(divide="ignore"):
        small = a < 20.0
        ls = np.where(small, np.log(np.where(small, np.sinh(a), 1.0)),
                      a + np.log1p(-np.exp(-2.0 * a)) - LOG2)
        ls = ls + np.log(t)
    return ls, (1.0 if mu >= 0 else -1.0)


_LEVEL_EDGES = [(0.0, 25.0)] + [(25.0 * 4 ** (l - 1), 25.0 * 4 ** l) for l in range(1, 4)]
_X_UNDERFLOW = 1600.0       # K_nu(x) < 1e-690 beyond this for the orders used here: exactly 0 in FP64


def _quadrature(x: np.ndarray, nu: float, kind: str) -> np.ndarray:
    """Trapezoid sums for K_nu (kind='k') or dK_nu/dnu (kind='dnu') at every x > 0."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    grow = abs(nu) + 1.0                       # exponential growth rate of the integrand's factor
    for level, (lo, hi) in enumerate(_LEVEL_EDGES):
        sel = (x > lo) & (x <= hi)
        if not np.any(sel):
            continue
        xs = x[sel]
        h = 0.1 / 2 ** level
        xmin = float(xs.min())
        tpk = math.asinh(grow / xmin)
        gpk = -xmin * math.cosh(tpk) + grow * tpk
        T = tpk
        while -xmin * math.cosh(T) + grow * T > gpk - 50.0:
            T += 0.25
        t = np.arange(int(math.ceil(T / h)) + 1) * h
        w = np.full(t.shape, h)
        w[0] = 0.5 * h                          # trapezoid rule on [0, inf) of an even integrand
        if kind == "k":
            logf, sign = _logcosh(nu * t), 1.0
        else:
            logf, sign = _t_log_sinh(t, nu)
        # x cosh t = x + 2 x sinh^2(t/2): factoring exp(-x) out keeps the exponent small near
        # the peak, so a large x does not cost relative accuracy in the exponential
        st2 = 2.0 * np.sinh(0.5 * t) ** 2
        res = np.empty_like(xs)
        step = max(1, 4_000_000 // len(t))
        for s in range(0, len(xs), step):
            xc = xs[s:s + step, None]
            res[s:s + step] = np.exp(-xc * st2[None, :] + logf[None, :]) @ w
        out[sel] = sign * res * np.exp(-xs)
    return out


def bessel_k(nu: float, x) -> np.ndarray:
    """Modified Bessel function of the second kind K_nu(x), x > 0 (array), any real nu."""
    x = np.asarray(x, dtype=np.float64)
    if np.any(x <= 0):
        raise ValueError("K_nu(x) needs x > 0")
    return _quadrature(x, float(nu), "k")


def bessel_k_dnu(nu: float, x) -> np.ndarray:
    """Partial derivative dK_nu(x)/dnu, x > 0 (array)."""
    x = np.asarray(x, dtype=np.float64)
    if np.any(x <= 0):
        raise ValueError("dK_nu/dnu(x) needs x > 0")
    return _quadrature(x, float(nu), "dnu")


# Bernoulli numbers B_2 .. B_14 (exact rationals) for the digamma asymptotic series
_BERNOULLI_2K = [1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0, 5.0 / 66.0, -691.0 / 2730.0, 7.0 / 6.0]


def digamma(x: float) -> float:
    """psi(x) = Gamma'(x)/Gamma(x) for real x not a non-positive integer.

    psi(x) = psi(x+1) - 1/x shifts x to >= 10, then
    psi(x) ~ ln x - 1/(2x) - sum_k B_2k / (2k x^2k)      (DLMF 5.11.2)
    and psi(x) = psi(1-x) - pi cot(pi x) reflects negative arguments (DLMF 5.5.4).
    """
    x = float(x)
    if x <= 0.0 and x == math.floor(x):
        raise ValueError("digamma has poles at non-positive integers")
    if x < 0.0:
        return digamma(1.0 - x) - math.pi / math.tan(math.pi * x)
    acc = 0.0
    while x < 10.0:
        acc -= 1.0 / x
        x += 1.0
    inv2 = 1.0 / (x * x)
    p = inv2
    s = 0.0
    for k, b in enumerate(_BERNOULLI_2K, start=1):
        s += b / (2 * k) * p
        p *= inv2
    return acc + math.log(x) - 0.5 / x - s


def gamma(x: float) -> float:
    """Gamma function (the library routine math.gamma)."""
    return math.gamma(x)
