"""Matern covariance and its parameter partials, dense, in FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2.1:  C(h; theta) = sigma^2 / (2^(nu-1) Gamma(nu)) (h/alpha)^nu K_nu(h/alpha),
           theta = (sigma^2, alpha, nu), Sigma_ij = C(||s_i - s_j||; theta).
Sec. 2.2:  Sigma_sigma2 = Sigma / sigma^2,
           dC/dalpha = sigma^2 / (2^(nu-1) Gamma(nu) alpha) (h/alpha)^(nu+1) K_(nu-1)(h/alpha),
           Sigma_nu from d/dnu [x^nu K_nu(x)] (Supp. A).
With x = h/alpha and R = C/sigma^2 the correlation,
           dR/dnu = ( d/dnu[x^nu K_nu] - (log 2 + psi(nu)) x^nu K_nu ) / (2^(nu-1) Gamma(nu)),
the second term being the nu-derivative of the normalising constant.  At x = 0, R = 1 for every
theta, so both partials of R vanish there (Supp. A case 1, read as dC/dnu(0) = 0).

Jitter (the paper has none; the workloads add delta = 1e-8 to the diagonal):
  mode 0: Sigma = sigma^2 (R + delta I)   -> Sigma_sigma2 = Sigma / sigma^2 stays exact, so the
          closed forms of Algorithm 3, Step 2 hold;
  mode 1: Sigma = sigma^2 R + delta I     -> Sigma_sigma2 = R.
"""
from __future__ import annotations

import math

import numpy as np

from . import special, paper_series


def distances(locs: np.ndarray) -> np.ndarray:
    """Euclidean distance matrix of n x 2 locations, written out coordinate by coordinate."""
    locs = np.asarray(locs, dtype=np.float64)
    dx = locs[:, 0][:, None] - locs[:, 0][None, :]
    dy = locs[:, 1][:, None] - locs[:, 1][None, :]
    return np.sqrt(dx * dx + dy * dy)


def correlation_parts(x, alpha: float, nu: float, dnu: str = "exact", partials: bool = True):
    """R(x), dR/dalpha, dR/dnu at x = h/alpha >= 0 (arrays of the shape of x).

    dnu='exact' uses the quadrature dK_nu/dnu; dnu='paper' uses Supp. A's five cases.
    """
    x = np.asarray(x, dtype=np.float64)
    R = np.ones_like(x)
    dRa = np.zeros_like(x)
    dRn = np.zeros_like(x)
    pos = x > 0
    if not np.any(pos):
        return R, dRa, dRn
    xp = x[pos]
    norm = 2.0 ** (nu - 1.0) * math.gamma(nu)
    lx = np.log(xp)
    knu = special.bessel_k(nu, xp)
    xnuk = np.exp(nu * lx) * knu                       # x^nu K_nu(x)
    R[pos] = xnuk / norm
    if partials:
        knum1 = special.bessel_k(nu - 1.0, xp)         # K_(nu-1) = K_(1-nu)
        dRa[pos] = np.exp((nu + 1.0) * lx) * knum1 / (norm * alpha)
        if dnu == "exact":
            d_xnuk = np.exp(nu * lx) * (lx * knu + special.bessel_k_dnu(nu, xp))
        elif dnu == "paper":
            d_xnuk = paper_series.dnu_xnu_k(nu, xp)
        else:
            raise ValueError(dnu)
        dRn[pos] = (d_xnuk - (special.LOG2 + special.digamma(nu)) * xnuk) / norm
    return R, dRa, dRn


def covariance(locs, theta, jitter: float = 1e-8, mode: int = 0, partials: bool = True,
               dnu: str = "exact") -> dict:
    """Dense Sigma and, if asked, Sigma_sigma2, Sigma_alpha, Sigma_nu (all n x n, symmetric)."""
    sigma2, alpha, nu = (float(t) for t in theta)
    locs = np.asarray(locs, dtype=np.float64)
    n = locs.shape[0]
    D = distances(locs)
    il = np.tril_indices(n, -1)
    R_l, dRa_l, dRn_l = correlation_parts(D[il] / alpha, alpha, nu, dnu=dnu, partials=partials)

    def sym(vals, diag):
        M = np.zeros((n, n))
        M[il] = vals
        M = M + M.T
        M[np.diag_indices(n)] = diag
        return M

    R = sym(R_l, 1.0)
    out = {}
    if mode == 0:
        out["S"] = sigma2 * (R + jitter * np.eye(n))
        out["S_sigma2"] = R + jitter * np.eye(n)
    elif mode == 1:
        out["S"] = sigma2 * R + jitter * np.eye(n)
        out["S_sigma2"] = R
    else:
        raise ValueError(mode)
    if partials:
        out["S_alpha"] = sigma2 * sym(dRa_l, 0.0)
        out["S_nu"] = sigma2 * sym(dRn_l, 0.0)
    return out
