"""Textbook dense linear algebra for the oracle, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Algorithm 2 and 3 need the Cholesky factor Sigma = L L^T, log det Sigma = 2 sum log L_ii and the
solves L^-1 Z and Sigma^-1 Z.  These are written out as textbook blocked algorithms (unblocked
column steps inside a block, matrix products from numpy between blocks) so that they can be read
against their definitions.
"""
from __future__ import annotations

import numpy as np


class NotPositiveDefinite(ArithmeticError):
    """Raised when a Cholesky pivot is not strictly positive (or not finite)."""


def cholesky(A: np.ndarray, nb: int = 64, overwrite: bool = False) -> np.ndarray:
    """Lower-triangular L with A = L L^T, right-looking blocked algorithm (overwrite: factor A's
    own storage in place, for matrices too large to copy, updating only the lower part of the
    trailing matrix, a block of columns at a time)."""
    W = A if overwrite else np.array(A, dtype=np.float64, copy=True)
    n = W.shape[0]
    for k0 in range(0, n, nb):
        k1 = min(n, k0 + nb)
        for j in range(k0, k1):                      # diagonal block, column by column
            d = W[j, j] - W[j, k0:j] @ W[j, k0:j]
            if not (d > 0.0 and np.isfinite(d)):
                raise NotPositiveDefinite(f"pivot {j}: {d}")
            W[j, j] = np.sqrt(d)
            W[j + 1:k1, j] = (W[j + 1:k1, j] - W[j + 1:k1, k0:j] @ W[j, k0:j]) / W[j, j]
        for j in range(k0, k1):                      # panel below: X L_kk^T = A_panel
            W[k1:, j] = (W[k1:, j] - W[k1:, k0:j] @ W[j, k0:j]) / W[j, j]
        P = W[k1:, k0:k1]
        if overwrite:                                # trailing update, lower part, column chunks
            for c0 in range(k1, n, 4 * nb):          # (no (n - k1)^2 temporary)
                c1 = min(n, c0 + 4 * nb)
                W[c0:, c0:c1] -= P[c0 - k1:] @ P[c0 - k1:c1 - k1].T
        else:
            W[k1:, k1:] -= P @ P.T                   # trailing update
    if overwrite:
        for k0 in range(0, n, nb):                   # zero the strict upper triangle in blocks
            k1 = min(n, k0 + nb)
            W[k0:k1, k1:] = 0.0
            W[k0:k1, k0:k1] = np.tril(W[k0:k1, k0:k1])
        return W
    return np.tril(W)


def solve_lower(L: np.ndarray, B: np.ndarray, nb: int = 64) -> np.ndarray:
    """X with L X = B (forward substitution); B is a vector or a matrix."""
    X = np.array(B, dtype=np.float64, copy=True)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    n = L.shape[0]
    for k0 in range(0, n, nb):
        k1 = min(n, k0 + nb)
        for j in range(k0, k1):
            X[j] = (X[j] - L[j, k0:j] @ X[k0:j]) / L[j, j]
        X[k1:] -= L[k1:, k0:k1] @ X[k0:k1]
    return X[:, 0] if vec else X


def solve_lower_t(L: np.ndarray, B: np.ndarray, nb: int = 64) -> np.ndarray:
    """X with L^T X = B (back substitution); B is a vector or a matrix."""
    X = np.array(B, dtype=np.float64, copy=True)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    n = L.shape[0]
    starts = list(range(0, n, nb))
    for k0 in reversed(starts):
        k1 = min(n, k0 + nb)
        for j in range(k1 - 1, k0 - 1, -1):
            X[j] = (X[j] - L[j + 1:k1, j] @ X[j + 1:k1]) / L[j, j]
        X[:k0] -= L[k0:k1, :k0].T @ X[k0:k1]
    return X[:, 0] if vec else X


def logdet_from_cholesky(L: np.ndarray) -> float:
    """log det(L L^T) = 2 sum_i log L_ii (Algorithm 2)."""
    return float(2.0 * np.sum(np.log(np.diag(L))))


def trace_product(A: np.ndarray, B: np.ndarray) -> float:
    """trace(A B) = sum_jk A_jk B_kj, the definition written out."""
    return float(np.sum(A * B.T))


def trace_product_eq4(A: np.ndarray, B: np.ndarray) -> float:
    """trace(A B) by the paper's Frobenius identity, Eq. 4:
    (||A + B^T||_F^2 - ||A||_F^2 - ||B||_F^2) / 2."""
    fro2 = lambda M: float(np.sum(M * M))  # noqa: E731
    return 0.5 * (fro2(A + B.T) - fro2(A) - fro2(B))
