"""Pins for the oracle's Algorithm 1 (CPU only): Table 1, the constants of Sec. 2.1, the relaxed
Armijo test, the 3x3 Fisher solve, and the iteration's behaviour on fake evaluators with known
answers (one-step convergence on a quadratic, halving, the 60/20 shift rule, singular Fisher,
infeasible steps), plus a full run on a small field."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import fisher_bt as fb, likelihood, fields
from paper_2601_11437_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_l9_design_matches_table_1():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "l9_table1.txt")) if l.strip() and not l.startswith("#")]
    W = np.array([[float(Fraction(v)) for v in r[1:]] for r in rows])
    np.testing.assert_array_equal(W, np.asarray(fb.L9_LOWER_WEIGHTS))
    lo, hi = np.array([0.01, 0.01, 0.01]), np.array([5.0, 5.0, 2.0])
    cands = fb.l9_design(lo, hi)
    np.testing.assert_allclose(cands[0], (lo + hi) / 2)
    np.testing.assert_allclose(cands[4], [5 / 6 * lo[0] + hi[0] / 6, 5 / 6 * lo[1] + hi[1] / 6, lo[2] / 6 + 5 / 6 * hi[2]])
    # an L9(3^3) orthogonal array: every pair of columns shows all nine level pairs once
    for a in range(3):
        for b in range(a + 1, 3):
            assert len({(r[a], r[b]) for r in map(tuple, W)}) == 9


def test_constants_match_section_2_1():
    c = {}
    for line in open(os.path.join(GOLDEN, "algorithm_constants.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            c[k] = float(v)
    assert (fb.ARMIJO_C, fb.RHO, fb.ARMIJO_SLACK, fb.GRAD_TOL) == (c["armijo_c"], c["armijo_rho"], c["armijo_slack"], c["grad_tol"])
    assert (fb.MAX_LL_CALLS, fb.MAX_GRAD_CALLS, fb.NM_FTOL) == (c["max_ll_calls"], c["max_grad_calls"], c["nm_ftol"])


def test_relaxed_armijo():
    g, phi = np.array([1.0, 2.0, 0.0]), np.array([0.5, 0.25, 3.0])     # g.phi = 1
    assert fb.armijo_relaxed(10.0 + 0.001 - 0.001, 10.0, g, phi)        # equality counts
    assert not fb.armijo_relaxed(10.0 - 1e-9, 10.0, g, phi)
    assert fb.armijo_relaxed(10.0 - 0.0005, 10.0, np.zeros(3), phi)     # within the slack
    assert not fb.armijo_relaxed(-math.inf, 10.0, g, phi)
    assert not fb.armijo_relaxed(float("nan"), 10.0, g, phi)


def test_fisher_direction():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 3))
    I = A @ A.T + np.eye(3)
    g = rng.standard_normal(3)
    np.testing.assert_allclose(fb.fisher_direction(g, I), np.linalg.solve(I, g), rtol=1e-12)
    assert fb.fisher_direction(g, np.diag([1.0, -1.0, 1.0])) is None


class Quadratic:
    """l(theta) = -1/2 (theta - t*)^T H (theta - t*): score -H (theta - t*), Fisher H."""

    def __init__(self, tstar, H, shift=0.0):
        self.t, self.H, self.calls = np.asarray(tstar, float), np.asarray(H, float), []

    def loglik(self, th):
        self.calls.append(("ll", tuple(th)))
        d = np.asarray(th) - self.t
        if np.any(np.asarray(th) <= 0):
            return -math.inf
        return -0.5 * d @ self.H @ d

    def evaluate(self, th):
        self.calls.append(("eval", tuple(th)))
        d = np.asarray(th) - self.t
        return -0.5 * d @ self.H @ d, -self.H @ d, self.H


def test_quadratic_converges_in_one_step():
    H = np.array([[2.0, 0.3, 0.0], [0.3, 1.0, 0.1], [0.0, 0.1, 0.5]])
    ev = Quadratic([1.0, 0.1, 0.8], H)
    st = fb.run(ev, theta0=(0.5, 0.05, 0.6))
    assert st.state == fb.CONVERGED and st.iter == 1
    np.testing.assert_allclose(st.theta, [1.0, 0.1, 0.8], atol=1e-14)
    assert (st.n_ll, st.n_grad) == (3, 2)          # eval(theta0), ll(candidate), eval(theta1)


def test_l9_start_picks_best_candidate_and_counts_calls():
    H = np.eye(3)
    lo, hi = np.array([0.01, 0.01, 0.01]), np.array([5.0, 5.0, 2.0])
    cands = fb.l9_design(lo, hi)
    best = cands[6]
    ev = Quadratic(best + np.array([0.01, 0.0, 0.0]), H)
    st = fb.start(ev, theta_lo=lo, theta_hi=hi)
    np.testing.assert_allclose(st.theta, best)
    assert st.n_ll == 10 and st.n_grad == 1


class Overshoot(Quadratic):
    """Fisher = H / 8, so the full step overshoots 8x and needs three halvings."""

    def evaluate(self, th):
        ll, g, H = super().evaluate(th)
        return ll, g, H / 8.0


def test_backtracking_halves_until_relaxed_armijo_holds():
    ev = Overshoot([1.0, 1.0, 1.0], np.diag([100.0, 100.0, 100.0]))
    st = fb.start(ev, theta0=(2.0, 2.0, 2.0))
    np.testing.assert_allclose(st.phi, [-8.0, -8.0, -8.0])
    fb.step(ev, st)
    # candidates at phi, phi/2, phi/4 are infeasible (non-positive); phi/8 lands on the optimum
    lls = [c for c in ev.calls if c[0] == "ll"]
    assert len(lls) == 4
    np.testing.assert_allclose(st.theta, [1.0, 1.0, 1.0])
    assert st.state == fb.CONVERGED


class NeverConverges:
    """Constant unit gradient; l increases along the Fisher step, so every step is accepted."""

    def loglik(self, th):
        return float(np.sum(th))

    def evaluate(self, th):
        return float(np.sum(th)), np.ones(3), np.eye(3) * 1e3


def test_gradient_call_limit_shifts_to_nelder_mead():
    st = fb.start(NeverConverges(), theta0=(1.0, 1.0, 1.0))
    while st.state == fb.RUNNING:
        fb.step(NeverConverges(), st)
    assert st.state == fb.SHIFT
    assert st.n_grad == 21 and st.n_ll == 41       # shift once more than 20 gradient calls


def test_singular_fisher_shifts_immediately():
    class Singular(NeverConverges):
        def evaluate(self, th):
            return 0.0, np.ones(3), np.zeros((3, 3))
    st = fb.start(Singular(), theta0=(1.0, 1.0, 1.0))
    assert st.state == fb.SHIFT


def test_nelder_mead_minimises_a_smooth_function():
    f = lambda x: (x[0] - 1) ** 2 + 10 * (x[1] - 2) ** 2 + 0.5 * (x[2] - 0.3) ** 2  # noqa: E731
    x, fx, calls = fb.nelder_mead(f, np.array([1.5, 1.5, 0.5]), ftol=1e-14, max_calls=4000)
    np.testing.assert_allclose(x, [1, 2, 0.3], atol=1e-5)
    assert calls <= 4000


def test_full_run_on_small_field_converges():
    n = 150
    locs = inputs.uniform_locations(n, 8)
    th_true = (1.0, 0.1, 0.5)
    z = fields.sample_field(locs, inputs.standard_normal(n, 8), th_true)
    ev = likelihood.DenseEvaluator(locs, z)
    st = fb.run(ev, theta0=(0.5, 0.05, 1.0))
    assert st.state in (fb.CONVERGED, fb.DONE_NM)
    if st.state == fb.CONVERGED:
        assert np.linalg.norm(st.score) <= 1e-3
    # the estimate beats the start and the truth in likelihood
    assert st.loglik >= ev.loglik(th_true) - 1e-9
    assert st.loglik >= ev.loglik((0.5, 0.05, 1.0))
