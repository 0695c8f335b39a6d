"""Seeded synthetic Gaussian fields z = L_true e, L_true the oracle's Cholesky of Sigma(theta_true).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The standard normal vector e and the
locations come from the caller (the shared seeded generators); this module only applies the
oracle's own covariance and Cholesky factor to them.
"""
from __future__ import annotations

import numpy as np

from . import matern, linalg


def sample_field(locs, e, theta_true, jitter: float = 1e-8, mode: int = 0) -> np.ndarray:
    """z = L e with Sigma(theta_true) = L L^T, so z ~ N(0, Sigma(theta_true)) when e ~ N(0, I)."""
    S = matern.covariance(locs, theta_true, jitter=jitter, mode=mode, partials=False)["S"]
    L = linalg.cholesky(S, nb=256)
    return L @ np.asarray(e, dtype=np.float64)
