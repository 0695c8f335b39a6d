"""The paper's own evaluation of d/dnu [x^nu K_nu(x)] (Supplementary A), in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Supplementary A dispatches on x = h/alpha and nu:
  case 1  x = 0                                   -> derivative zero
  case 2  0 < x < 8.5, |nu - [nu]| > 1e-6          -> small-x series with g_k, d_k, digamma
  case 3  8.5 <= x < 30                            -> Debye uniform expansion of K_nu(nu z)
                                                      with the U_k polynomial recursion
  case 4  x >= 30, |(nu + 0.5) - [nu + 0.5]| > 1e-6 -> Hankel large-x expansion, a_k and b_k
  case 5  otherwise                                -> difference quotient with lag 1e-9
"up to the N-th term" is read as the inclusive partial sum k = 0..N.  Case 5's difference
quotient only reaches about 1e-7 relative accuracy; the oracle's exact route (matern.py,
dnu='exact') replaces it, and this module keeps the literal quotient for comparison.  [nu] is
the nearest integer, ties rounded half away from zero.
"""
from __future__ import annotations

import math

import numpy as np

from . import special

CASE2_TERMS = 20                 # "partial sum up to the 20th term"
CASE3_TERMS_NEAR = 12            # 8.5 <= x < 15
CASE3_TERMS_FAR = 8              # 15 <= x < 30
CASE4_TERMS = 5
NEAR_INT = 1e-6
FD_LAG = 1e-9


def nearest_int(v: float) -> float:
    return math.floor(abs(v) + 0.5) * (1.0 if v >= 0 else -1.0)


def g_k(nu: float, k: int) -> float:
    """g_k(nu) = Gamma(1+nu)/Gamma(1+k+nu) = prod_{j=1..k} (nu+j)^-1."""
    g = 1.0
    for j in range(1, k + 1):
        g /= (nu + j)
    return g


def d_k(nu: float, k: int) -> float:
    """d_k(nu) = d/dnu log g_k(nu) = -sum_{j=1..k} (nu+j)^-1."""
    return -sum(1.0 / (nu + j) for j in range(1, k + 1))


def case2(nu: float, x: np.ndarray, terms: int = CASE2_TERMS) -> np.ndarray:
    """Small-x series for d/dnu[x^nu K_nu(x)], nu not an integer (Supp. A, case 2)."""
    x = np.asarray(x, dtype=np.float64)
    psi_p, psi_m = special.digamma(nu), special.digamma(-nu)
    gam_p, gam_m = math.gamma(nu), math.gamma(-nu)
    lx = np.log(x)
    x2nu = np.exp(2.0 * nu * lx)
    acc = np.zeros_like(x)
    for k in range(terms + 1):
        pref = (x / 2.0) ** (2 * k) / (2.0 * math.factorial(k))
        first = 2.0 ** nu * (special.LOG2 + psi_p - d_k(-nu, k)) * gam_p * g_k(-nu, k)
        second = 2.0 ** (-nu) * x2nu * (-special.LOG2 + 2.0 * lx - psi_m + d_k(nu, k)) * gam_m * g_k(nu, k)
        acc += pref * (first + second)
    return acc


def case2_k(nu: float, x: np.ndarray, terms: int = CASE2_TERMS) -> np.ndarray:
    """The series for K_nu(x) that case 2 differentiates (the first display of Supp. A)."""
    x = np.asarray(x, dtype=np.float64)
    acc = np.zeros_like(x)
    for k in range(terms + 1):
        pref = (x / 2.0) ** (2 * k) / (2.0 * math.factorial(k))
        acc += pref * (math.gamma(nu) * (x / 2.0) ** (-nu) * g_k(-nu, k)
                       + math.gamma(-nu) * (x / 2.0) ** nu * g_k(nu, k))
    return acc


def debye_u_coefficients(kmax: int) -> list:
    """Coefficients c_j^(k), j = 0..3k, of the Debye polynomials U_k(p), k = 0..kmax.

    U_0 = 1 and U_{k+1}(p) = p^2 (1 - p^2) U_k'(p) / 2 + (1/8) int_0^p (1 - 5 t^2) U_k(t) dt,
    whose coefficients obey c_0 = 0 and
    c_j^(k+1) = (j - 1 + 1/(4j)) c_{j-1}^(k) / 2 - (j - 3 + 5/(4j)) c_{j-3}^(k) / 2
    (with c_i^(k) = 0 outside 0..3k), which gives the paper's special cases j = 1, 2, 3 and
    j in {3k+2, 3k+3}.
    """
    coeffs = [[1.0]]
    for k in range(kmax):
        prev = coeffs[-1]
        nxt = [0.0] * (3 * (k + 1) + 1)

        def c(i, prev=prev):
            return prev[i] if 0 <= i < len(prev) else 0.0

        for j in range(1, 3 * (k + 1) + 1):
            nxt[j] = 0.5 * (j - 1 + 1.0 / (4 * j)) * c(j - 1) - 0.5 * (j - 3 + 5.0 / (4 * j)) * c(j - 3)
        coeffs.append(nxt)
    return coeffs


def _poly(c: list, p: np.ndarray) -> np.ndarray:
    acc = np.zeros_like(p)
    for cj in reversed(c):
        acc = acc * p + cj
    return acc


def _dpoly(c: list, p: np.ndarray) -> np.ndarray:
    acc = np.zeros_like(p)
    for j in range(len(c) - 1, 0, -1):
        acc = acc * p + j * c[j]
    return acc


def case3(nu: float, x: np.ndarray) -> np.ndarray:
    """Debye-expansion value of d/dnu[x^nu K_nu(x)] for 8.5 <= x < 30 (Supp. A, case 3)."""
    x = np.asarray(x, dtype=np.float64)
    U = debye_u_coefficients(CASE3_TERMS_NEAR)
    z = x / nu
    s = np.sqrt(1.0 + z * z)
    p = 1.0 / s
    eta = s + np.log(z / (1.0 + s))
    gnu = x ** nu * np.sqrt(math.pi / (2.0 * nu)) * np.exp(-nu * eta) / (1.0 + z * z) ** 0.25
    out = np.empty_like(x)
    for kmax, mask in ((CASE3_TERMS_NEAR, x < 15.0), (CASE3_TERMS_FAR, x >= 15.0)):
        if not np.any(mask):
            continue
        pm = p[mask]
        s0 = np.zeros_like(pm)
        s1 = np.zeros_like(pm)
        s2 = np.zeros_like(pm)
        for k in range(kmax + 1):
            sgn = (-1.0) ** k
            uk = _poly(U[k], pm)
            s0 += sgn * nu ** (-k) * uk
            s1 += sgn * k * nu ** (-k - 1) * uk
            s2 += sgn * nu ** (-k) * _dpoly(U[k], pm)
        zm = z[mask]
        bracket = math.log(nu) + np.log(1.0 + np.sqrt(1.0 + zm * zm)) - 1.0 / (2.0 * nu * (1.0 + zm * zm))
        xm = x[mask]
        out[mask] = gnu[mask] * (bracket * s0 - s1 + xm * xm / nu ** 3 * (1.0 + zm * zm) ** -1.5 * s2)
    return out


def hankel_a(nu: float, k: int) -> float:
    """a_k(nu) = prod_{j=1..k} (4 nu^2 - (2j-1)^2) / (8^k k!)."""
    a = 1.0
    for j in range(1, k + 1):
        a *= (4.0 * nu * nu - (2 * j - 1) ** 2)
    return a / (8.0 ** k * math.factorial(k))


def hankel_b(nu: float, k: int) -> float:
    """b_k(nu) = sum_{j=1..k} 8 nu / (4 nu^2 - (2j-1)^2)  (= d/dnu log a_k)."""
    return sum(8.0 * nu / (4.0 * nu * nu - (2 * j - 1) ** 2) for j in range(1, k + 1))


def case4(nu: float, x: np.ndarray) -> np.ndarray:
    """Hankel-expansion value of d/dnu[x^nu K_nu(x)] for x >= 30 (Supp. A, case 4)."""
    x = np.asarray(x, dtype=np.float64)
    acc = np.zeros_like(x)
    lx = np.log(x)
    for k in range(CASE4_TERMS + 1):
        acc += x ** (-k) * (lx + hankel_b(nu, k)) * hankel_a(nu, k)
    return math.sqrt(math.pi / 2.0) * x ** (nu - 0.5) * np.exp(-x) * acc


def case5(nu: float, x: np.ndarray) -> np.ndarray:
    """The literal difference quotient with lag 1e-9 (Supp. A, case 5), on the exact K_nu."""
    x = np.asarray(x, dtype=np.float64)
    f1 = x ** (nu + FD_LAG) * special.bessel_k(nu + FD_LAG, x)
    f0 = x ** nu * special.bessel_k(nu, x)
    return (f1 - f0) / FD_LAG


def classify(nu: float, x: np.ndarray) -> np.ndarray:
    """Case number 1..5 of Supp. A for each x."""
    x = np.asarray(x, dtype=np.float64)
    near_int = abs(nu - nearest_int(nu)) <= NEAR_INT
    near_half = abs((nu + 0.5) - nearest_int(nu + 0.5)) <= NEAR_INT
    case = np.full(x.shape, 5, dtype=np.int64)
    case[(x >= 30.0) & (not near_half)] = 4
    case[(x >= 8.5) & (x < 30.0)] = 3
    case[(x > 0) & (x < 8.5) & (not near_int)] = 2
    case[x == 0] = 1
    return case


def dnu_xnu_k(nu: float, x) -> np.ndarray:
    """d/dnu [x^nu K_nu(x)] following Supp. A's five cases in their order."""
    x = np.asarray(x, dtype=np.float64)
    case = classify(nu, x)
    out = np.zeros_like(x)
    for c, fn in ((2, case2), (3, case3), (4, case4), (5, case5)):
        m = case == c
        if np.any(m):
            out[m] = fn(nu, x[m])
    return out
