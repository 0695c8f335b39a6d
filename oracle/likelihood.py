"""Algorithm 2 (log-likelihood) and Algorithm 3 (log-likelihood, score, Fisher) in FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Eq. 1:  l(theta) = -n/2 log(2 pi) - 1/2 log det Sigma - 1/2 Z^T Sigma^-1 Z
Eq. 2:  l_i = -1/2 tr(Sigma^-1 Sigma_i) + 1/2 Z^T Sigma^-1 Sigma_i Sigma^-1 Z
Eq. 3:  I_ij = 1/2 tr(Sigma^-1 Sigma_i Sigma^-1 Sigma_j)
Algorithm 3 computes these in four steps: Step 1 is Algorithm 2; Step 2 the closed forms
l_1 = (Z^T Sigma^-1 Z - n) / (2 sigma^2) and I_11 = n / (2 sigma^4) (exact when Sigma_sigma2 =
Sigma / sigma^2, jitter mode 0); Steps 3 and 4 form A_i = Sigma^-1 Sigma_i, its trace,
w = Sigma^-1 Z, v = Sigma_i w, w^T v and the trace products.  The oracle forms A_i by column solves
with the Cholesky factor and tr(A_i A_j) by its definition (the direct double sum); Eq. 4 is
available as linalg.trace_product_eq4 and pinned against the direct sum in the tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import matern, linalg

LOG_2PI = math.log(2.0 * math.pi)


@dataclass
class Evaluation:
    loglik: float
    score: np.ndarray          # (3,)
    fisher: np.ndarray         # (3, 3)
    logdet: float
    quad: float                # Z^T Sigma^-1 Z
    # the two terms of each score component (Eq. 2), l_i = -1/2 trace[i] + 1/2 qform[i]:
    # trace[i] = tr(Sigma^-1 Sigma_i), qform[i] = w^T Sigma_i w with w = Sigma^-1 Z
    trace: np.ndarray = None
    qform: np.ndarray = None


def check_theta(theta) -> None:
    if len(theta) != 3 or not all(math.isfinite(t) and t > 0 for t in theta):
        raise ValueError(f"theta must be three positive finite numbers, got {theta}")


def loglik(locs, z, theta, jitter: float = 1e-8, mode: int = 0) -> float:
    """Algorithm 2.  Raises linalg.NotPositiveDefinite when Sigma(theta) is not PD."""
    check_theta(theta)
    z = np.asarray(z, dtype=np.float64)
    n = z.shape[0]
    S = matern.covariance(locs, theta, jitter=jitter, mode=mode, partials=False)["S"]
    L = linalg.cholesky(S)
    logdet = linalg.logdet_from_cholesky(L)
    Y = linalg.solve_lower(L, z)
    quad = float(Y @ Y)
    return -0.5 * n * LOG_2PI - 0.5 * logdet - 0.5 * quad


def loglik_score_fisher(locs, z, theta, jitter: float = 1e-8, mode: int = 0,
                        dnu: str = "exact") -> Evaluation:
    """Algorithm 3: (l, grad l, I) at theta."""
    check_theta(theta)
    sigma2 = float(theta[0])
    z = np.asarray(z, dtype=np.float64)
    n = z.shape[0]
    mats = matern.covariance(locs, theta, jitter=jitter, mode=mode, partials=True, dnu=dnu)
    # Step 1
    L = linalg.cholesky(mats["S"])
    logdet = linalg.logdet_from_cholesky(L)
    Y = linalg.solve_lower(L, z)
    quad = float(Y @ Y)
    ll = -0.5 * n * LOG_2PI - 0.5 * logdet - 0.5 * quad
    w = linalg.solve_lower_t(L, Y)                        # w = Sigma^-1 Z

    def sigma_inv_times(M):
        return linalg.solve_lower_t(L, linalg.solve_lower(L, M))

    score = np.zeros(3)
    fisher = np.zeros((3, 3))
    traces, qforms = np.zeros(3), np.zeros(3)
    A = [None, None, None]
    # Step 2 (closed forms, valid in jitter mode 0); mode 1 uses Eq. 2 / Eq. 3 directly
    if mode == 0:
        score[0] = (quad - n) / (2.0 * sigma2)
        fisher[0, 0] = n / (2.0 * sigma2 ** 2)
        traces[0], qforms[0] = n / sigma2, quad / sigma2
    else:
        A[0] = sigma_inv_times(mats["S_sigma2"])
        traces[0], qforms[0] = float(np.trace(A[0])), float(w @ (mats["S_sigma2"] @ w))
        score[0] = -0.5 * traces[0] + 0.5 * qforms[0]
        fisher[0, 0] = 0.5 * linalg.trace_product(A[0], A[0])
    # Steps 3 and 4
    for i, key in ((1, "S_alpha"), (2, "S_nu")):
        Si = mats[key]
        A[i] = sigma_inv_times(Si)
        tr = float(np.trace(A[i]))
        v = Si @ w
        traces[i], qforms[i] = tr, float(w @ v)
        score[i] = -0.5 * tr + 0.5 * qforms[i]
        if mode == 0:
            fisher[0, i] = fisher[i, 0] = tr / (2.0 * sigma2)
        else:
            fisher[0, i] = fisher[i, 0] = 0.5 * linalg.trace_product(A[0], A[i])
        for j in range(1, i + 1):
            fisher[i, j] = fisher[j, i] = 0.5 * linalg.trace_product(A[i], A[j])
    return Evaluation(ll, score, fisher, logdet, quad, traces, qforms)


class DenseEvaluator:
    """Evaluator over fixed (locs, z) with the interface Algorithm 1 needs."""

    def __init__(self, locs, z, jitter: float = 1e-8, mode: int = 0, dnu: str = "exact"):
        self.locs = np.asarray(locs, dtype=np.float64)
        self.z = np.asarray(z, dtype=np.float64)
        self.jitter, self.mode, self.dnu = jitter, mode, dnu

    def loglik(self, theta) -> float:
        try:
            return loglik(self.locs, self.z, theta, self.jitter, self.mode)
        except (ValueError, linalg.NotPositiveDefinite):
            return -math.inf

    def evaluate(self, theta):
        e = loglik_score_fisher(self.locs, self.z, theta, self.jitter, self.mode, self.dnu)
        return e.loglik, e.score, e.fisher
