"""Algorithm 1 (Fisher-BT) with the L9 start (Table 1) and the Nelder-Mead fallback (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2.1 fixes: Armijo constant c = 0.001 and halving rho = 0.5; the relaxed condition
    l(theta + phi) >= l(theta) + 0.001 grad l(theta) . phi - 0.001            (Eq. 5, relaxed)
the stopping rule ||grad l(theta)||_2 <= 0.001; the shift to Nelder-Mead once l has been evaluated
more than 60 times (the L9 start included) or the gradient more than 20 times; Nelder-Mead stops
when a step changes l by less than 1e-9 and is followed by one Fisher information evaluation.

Readings where the paper is silent (shared with the CUDA library's host driver):
  * every Algorithm 2 or Algorithm 3 call counts as an l call; every Algorithm 3 call counts as a
    gradient call; a candidate with a non-positive parameter or a non-PD Sigma counts as a call
    and has l = -inf, so Armijo fails and phi is halved;
  * the call-count shift rule is checked where Algorithm 1 checks its while condition (after each
    Fisher iteration); the line search itself halves until Armijo holds, which the -0.001 slack
    guarantees for a finite l(theta), with a cap of 64 halvings as a guard;
  * a Fisher matrix whose 3x3 Cholesky fails shifts to Nelder-Mead at once;
  * Nelder-Mead uses reflection 1, expansion 2, contraction 1/2, shrink 1/2, an initial simplex of
    theta and theta + 0.05 theta_i e_i, and stops when the spread of l over the simplex is below
    1e-9 (the absolute function tolerance of a Nelder-Mead step), or after 1000 l calls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ARMIJO_C = 0.001
ARMIJO_SLACK = 0.001
RHO = 0.5
GRAD_TOL = 1e-3
MAX_LL_CALLS = 60
MAX_GRAD_CALLS = 20
NM_FTOL = 1e-9
NM_MAX_CALLS = 1000
MAX_HALVINGS = 64

RUNNING, CONVERGED, SHIFT, DONE_NM, FAILED = 0, 1, 2, 3, -1

# Table 1: the weight on the lower corner theta^(l) for each of the three parameters.
# M = 1/2 (midpoint), L = 5/6 (near the lower corner), U = 1/6 (near the upper corner).
_M, _L, _U = 0.5, 5.0 / 6.0, 1.0 / 6.0
L9_LOWER_WEIGHTS = (
    (_M, _M, _M), (_M, _L, _L), (_M, _U, _U),
    (_L, _M, _L), (_L, _L, _U), (_L, _U, _M),
    (_U, _M, _U), (_U, _L, _M), (_U, _U, _L),
)


def l9_design(theta_lo, theta_hi) -> np.ndarray:
    """The nine initial candidates of Table 1: w * theta^(l) + (1 - w) * theta^(u) per parameter."""
    lo = np.asarray(theta_lo, dtype=np.float64)
    hi = np.asarray(theta_hi, dtype=np.float64)
    W = np.asarray(L9_LOWER_WEIGHTS)
    return W * lo[None, :] + (1.0 - W) * hi[None, :]


def armijo_relaxed(ll_new: float, ll: float, score, phi) -> bool:
    """Relaxed Armijo test of Sec. 2.1: LHS minus RHS of Eq. 5 (c = 0.001, s = 1) >= -0.001."""
    if not math.isfinite(ll_new):
        return False
    return ll_new - (ll + ARMIJO_C * float(np.dot(score, phi))) >= -ARMIJO_SLACK


def fisher_direction(score, fisher):
    """phi = I^-1 grad l by a 3x3 Cholesky; None when I is not positive definite."""
    I = np.asarray(fisher, dtype=np.float64)
    L = np.zeros((3, 3))
    for j in range(3):
        d = I[j, j] - sum(L[j, k] ** 2 for k in range(j))
        if not (d > 0.0 and math.isfinite(d)):
            return None
        L[j, j] = math.sqrt(d)
        for i in range(j + 1, 3):
            L[i, j] = (I[i, j] - sum(L[i, k] * L[j, k] for k in range(j))) / L[j, j]
    g = np.asarray(score, dtype=np.float64)
    y = np.zeros(3)
    for i in range(3):
        y[i] = (g[i] - sum(L[i, k] * y[k] for k in range(i))) / L[i, i]
    x = np.zeros(3)
    for i in (2, 1, 0):
        x[i] = (y[i] - sum(L[k, i] * x[k] for k in range(i + 1, 3))) / L[i, i]
    return x


@dataclass
class State:
    theta: np.ndarray
    phi: np.ndarray = field(default_factory=lambda: np.zeros(3))
    loglik: float = -math.inf
    score: np.ndarray = field(default_factory=lambda: np.zeros(3))
    fisher: np.ndarray = field(default_factory=lambda: np.zeros((3, 3)))
    n_ll: int = 0
    n_grad: int = 0
    iter: int = 0
    state: int = RUNNING
    history: list = field(default_factory=list)


def _fisher_iteration(ev, st: State) -> None:
    """One "Fisher scoring iteration" of Algorithm 1: l, grad l, I at theta, then phi = I^-1 grad l."""
    ll, g, I = ev.evaluate(tuple(st.theta))
    st.n_ll += 1
    st.n_grad += 1
    st.loglik, st.score, st.fisher = ll, np.asarray(g, float), np.asarray(I, float)
    st.history.append((st.theta.copy(), ll))
    if float(np.linalg.norm(st.score)) <= GRAD_TOL:
        st.state = CONVERGED
        return
    phi = fisher_direction(st.score, st.fisher)
    if phi is None:
        st.state = SHIFT
        return
    st.phi = phi
    if st.n_ll > MAX_LL_CALLS or st.n_grad > MAX_GRAD_CALLS:
        st.state = SHIFT


def start(ev, theta0=None, theta_lo=None, theta_hi=None) -> State:
    """Pick theta^(0) (given, or the best of the L9 design) and run the first Fisher iteration."""
    n_ll = 0
    if theta0 is None:
        cands = l9_design(theta_lo, theta_hi)
        lls = []
        for c in cands:
            lls.append(ev.loglik(tuple(c)))
            n_ll += 1
        theta0 = cands[int(np.argmax(lls))]
    st = State(theta=np.asarray(theta0, dtype=np.float64).copy(), n_ll=n_ll)
    _fisher_iteration(ev, st)
    return st


def step(ev, st: State) -> State:
    """One accepted Fisher-BT step: backtracking on phi, theta <- theta + phi, Fisher iteration."""
    if st.state != RUNNING:
        return st
    for _ in range(MAX_HALVINGS + 1):
        cand = st.theta + st.phi
        ll_new = ev.loglik(tuple(cand))
        st.n_ll += 1
        if armijo_relaxed(ll_new, st.loglik, st.score, st.phi):
            break
        st.phi = st.phi * RHO
    else:
        st.state = FAILED
        return st
    st.theta = cand
    st.iter += 1
    _fisher_iteration(ev, st)
    return st


def nelder_mead(f, x0, ftol: float = NM_FTOL, max_calls: int = NM_MAX_CALLS):
    """Minimise f from x0 (reflection 1, expansion 2, contraction 1/2, shrink 1/2)."""
    x0 = np.asarray(x0, dtype=np.float64)
    d = x0.shape[0]
    simplex = [x0.copy()]
    for i in range(d):
        v = x0.copy()
        v[i] += 0.05 * (x0[i] if x0[i] != 0 else 1.0)
        simplex.append(v)
    fs = [f(v) for v in simplex]
    calls = len(fs)
    while calls < max_calls:
        order = np.argsort(fs, kind="stable")
        simplex = [simplex[i] for i in order]
        fs = [fs[i] for i in order]
        if math.isfinite(fs[-1]) and fs[-1] - fs[0] < ftol:
            break
        c = np.mean(simplex[:-1], axis=0)
        xr = c + (c - simplex[-1])
        fr = f(xr)
        calls += 1
        if fr < fs[0]:
            xe = c + 2.0 * (c - simplex[-1])
            fe = f(xe)
            calls += 1
            simplex[-1], fs[-1] = (xe, fe) if fe < fr else (xr, fr)
        elif fr < fs[-2]:
            simplex[-1], fs[-1] = xr, fr
        else:
            if fr < fs[-1]:
                xc = c + 0.5 * (xr - c)
                fc = f(xc)
                calls += 1
                ok = fc <= fr
            else:
                xc = c + 0.5 * (simplex[-1] - c)
                fc = f(xc)
                calls += 1
                ok = fc < fs[-1]
            if ok:
                simplex[-1], fs[-1] = xc, fc
            else:
                for i in range(1, d + 1):
                    simplex[i] = simplex[0] + 0.5 * (simplex[i] - simplex[0])
                    fs[i] = f(simplex[i])
                    calls += 1
    best = int(np.argmin(fs))
    return simplex[best], fs[best], calls


def run(ev, theta0=None, theta_lo=None, theta_hi=None, max_steps: int = 200) -> State:
    """Algorithm 1 end to end: start, Fisher-BT steps until stop or shift, Nelder-Mead fallback."""
    st = start(ev, theta0, theta_lo, theta_hi)
    for _ in range(max_steps):
        if st.state != RUNNING:
            break
        step(ev, st)
    if st.state == SHIFT:
        def negll(th):
            if np.any(np.asarray(th) <= 0):
                return math.inf
            v = ev.loglik(tuple(th))
            return -v if math.isfinite(v) else math.inf
        theta, _, calls = nelder_mead(negll, st.theta)
        st.n_ll += calls
        st.theta = np.asarray(theta, dtype=np.float64)
        ll, g, I = ev.evaluate(tuple(st.theta))
        st.n_ll += 1
        st.n_grad += 1
        st.loglik, st.score, st.fisher = ll, np.asarray(g, float), np.asarray(I, float)
        st.state = DONE_NM
    return st
