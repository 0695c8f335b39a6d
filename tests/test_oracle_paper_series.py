"""Pins for the oracle's restatement of Supplementary A (the paper's five-case evaluation of
d/dnu [x^nu K_nu(x)]): its building blocks against their definitions and published closed forms,
and each case against the exact derivative within that case's truncation error (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import paper_series as ps, special

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "algorithm_constants.txt")


def _constants():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def test_constants_match_supplement_a():
    c = _constants()
    assert ps.CASE2_TERMS == c["supp_a_case2_terms"]
    assert ps.CASE3_TERMS_NEAR == c["supp_a_case3_near"]
    assert ps.CASE3_TERMS_FAR == c["supp_a_case3_far"]
    assert ps.CASE4_TERMS == c["supp_a_case4_terms"]
    assert ps.NEAR_INT == c["supp_a_near_int"]
    assert ps.FD_LAG == c["supp_a_fd_lag"]


def exact_dnu(nu, x):
    x = np.asarray(x, float)
    return x ** nu * (np.log(x) * special.bessel_k(nu, x) + special.bessel_k_dnu(nu, x))


def test_debye_u1_u2_closed_forms():
    # DLMF 10.41.10: u_1 = (3p - 5p^3)/24, u_2 = (81p^2 - 462p^4 + 385p^6)/1152
    c = ps.debye_u_coefficients(2)
    assert c[0] == [1.0]
    np.testing.assert_allclose(c[1], [0, 3 / 24, 0, -5 / 24], rtol=0, atol=1e-17)
    np.testing.assert_allclose(c[2], [0, 0, 81 / 1152, 0, -462 / 1152, 0, 385 / 1152], rtol=0, atol=1e-17)


def test_debye_recursion_reproduces_defining_relation():
    # U_(k+1)(p) = p^2 (1-p^2) U_k'(p) / 2 + (1/8) int_0^p (1 - 5 t^2) U_k(t) dt, evaluated with
    # numpy's polynomial calculus (independent of the coefficient recursion)
    from numpy.polynomial import polynomial as P
    c = ps.debye_u_coefficients(8)
    for k in range(8):
        uk = np.array(c[k])
        term1 = P.polymul([0, 0, 0.5, 0, -0.5], P.polyder(uk)) if len(uk) > 1 else np.zeros(1)
        integrand = P.polymul([1, 0, -5], uk)
        term2 = P.polyint(integrand) / 8.0
        rhs = P.polyadd(term1, term2)
        lhs = np.array(c[k + 1])
        m = max(len(lhs), len(rhs))
        np.testing.assert_allclose(np.pad(lhs, (0, m - len(lhs))), np.pad(rhs, (0, m - len(rhs))),
                                   rtol=1e-13, atol=1e-13 * np.max(np.abs(lhs)))


def test_gk_dk_definitions():
    mpmath = pytest.importorskip("mpmath")
    for nu in (0.3, -0.7, 1.25, -1.4):
        for k in (0, 1, 5, 20):
            assert ps.g_k(nu, k) == pytest.approx(math.gamma(1 + nu) / math.gamma(1 + k + nu), rel=1e-13)
            ref = float(mpmath.diff(lambda v: mpmath.log(abs(mpmath.gamma(1 + v) / mpmath.gamma(1 + k + v))), nu))
            assert ps.d_k(nu, k) == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_hankel_b_is_log_derivative_of_a():
    mpmath = pytest.importorskip("mpmath")
    for nu in (0.3, 0.8, 1.7):
        for k in range(1, 6):
            ref = float(mpmath.diff(lambda v: mpmath.log(abs(
                mpmath.fprod([4 * v * v - (2 * j - 1) ** 2 for j in range(1, k + 1)]))), nu))
            assert ps.hankel_b(nu, k) == pytest.approx(ref, rel=1e-12)
            assert ps.hankel_a(nu, k) == pytest.approx(
                math.prod(4 * nu * nu - (2 * j - 1) ** 2 for j in range(1, k + 1)) / (8 ** k * math.factorial(k)),
                rel=1e-14)


def test_small_x_series_for_k_matches_exact():
    for nu in (0.3, 0.8, 1.4, 2.2):
        x = np.array([0.01, 0.3, 1.0, 3.0])
        np.testing.assert_allclose(ps.case2_k(nu, x), special.bessel_k(nu, x), rtol=1e-12)


def test_case_classification_boundaries():
    x = np.array([0.0, 1e-9, 8.4999999, 8.5, 14.999, 15.0, 29.999, 30.0, 1e3])
    assert list(ps.classify(0.8, x)) == [1, 2, 2, 3, 3, 3, 3, 4, 4]
    assert list(ps.classify(1.0, x)) == [1, 5, 5, 3, 3, 3, 3, 4, 4]
    assert list(ps.classify(1.0 + 5e-7, x)) == [1, 5, 5, 3, 3, 3, 3, 4, 4]
    assert list(ps.classify(1.0 + 2e-6, x)) == [1, 2, 2, 3, 3, 3, 3, 4, 4]
    assert list(ps.classify(1.5, x)) == [1, 2, 2, 3, 3, 3, 3, 5, 5]
    assert list(ps.classify(2.5 - 1e-7, x)) == [1, 2, 2, 3, 3, 3, 3, 5, 5]


# (case, x values, relative tolerance): the truncation / cancellation error of each case, measured
# against the exact derivative; a dropped term or sign in any case moves it by orders of magnitude.
CASES = [
    (2, [1e-6, 0.01, 0.4, 2.0], 1e-11),
    (2, [5.0, 7.0, 8.4], 1e-6),
    (3, [8.5, 10.0, 14.9], 1e-7),
    (3, [15.0, 20.0, 29.9], 1e-9),
    (4, [30.0, 45.0, 100.0, 300.0], 1e-8),
]


@pytest.mark.parametrize("nu", [0.13, 0.3, 0.8, 1.2, 1.7, 2.2])
@pytest.mark.parametrize("case,xs,tol", CASES)
def test_paper_cases_against_exact_derivative(nu, case, xs, tol):
    x = np.array(xs)
    assert np.all(ps.classify(nu, x) == case)
    got = {2: ps.case2, 3: ps.case3, 4: ps.case4}[case](nu, x)
    np.testing.assert_allclose(got, exact_dnu(nu, x), rtol=tol)


def test_case5_difference_quotient_is_only_approximate():
    # nu = 1 exactly: every 0 < x < 8.5 falls into case 5; the lag-1e-9 quotient is accurate
    # to roughly 1e-6 relative, far from FP64 (why the oracle's exact route replaces it)
    x = np.array([0.05, 0.5, 2.0, 6.0])
    err = np.abs(ps.case5(1.0, x) / exact_dnu(1.0, x) - 1)
    assert np.all(err < 1e-4) and np.max(err) > 1e-12
