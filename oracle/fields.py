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


def covariance_blocked(locs, theta, jitter: float = 1e-8, block: int = 2048,
                       lower_only: bool = False) -> np.ndarray:
    """Sigma (mode 0) built one block of columns at a time, for sizes where the dense
    intermediate arrays of matern.covariance would not fit in host memory; entries are the same
    correlation_parts values.  lower_only: rows from the block's first column down only (the
    rest of the array is left unset), for a Cholesky that reads the lower triangle only."""
    sigma2, alpha, nu = (float(t) for t in theta)
    locs = np.asarray(locs, dtype=np.float64)
    n = locs.shape[0]
    S = np.empty((n, n))
    for c0 in range(0, n, block):
        c1 = min(n, c0 + block)
        r0 = c0 if lower_only else 0
        dx = locs[r0:, 0][:, None] - locs[c0:c1, 0][None, :]
        dy = locs[r0:, 1][:, None] - locs[c0:c1, 1][None, :]
        x = np.sqrt(dx * dx + dy * dy) / alpha
        del dx, dy
        R, _, _ = matern.correlation_parts(x.ravel(), alpha, nu, partials=False)
        S[r0:, c0:c1] = sigma2 * R.reshape(x.shape)
        del x, R
    S[np.diag_indices(n)] = sigma2 * (1.0 + jitter)
    return S


def sample_field_blocked(locs, e, theta_true, jitter: float = 1e-8) -> np.ndarray:
    """z = L e as sample_field, with Sigma from covariance_blocked and the factor in place."""
    S = covariance_blocked(locs, theta_true, jitter=jitter, lower_only=True)   # the in-place
    L = linalg.cholesky(S, nb=512, overwrite=True)                             # factor reads the lower part
    return L @ np.asarray(e, dtype=np.float64)
