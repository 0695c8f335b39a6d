"""Helpers for the GPU parity tests: library build/load, skips, and mapping the library's
reordered lower-tile slabs back to dense matrices in the caller's order (data movement only)."""
import os

import numpy as np
import pytest


def have_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def require_gpu():
    if not have_gpu():
        pytest.skip("needs a CUDA GPU")
    from paper_2601_11437_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    _lib.load()


def slab_to_dense(slab: np.ndarray, nb: int, T: int, n: int, lower_only: bool = False) -> np.ndarray:
    """Lower-tile slab (column-major tiles, tile-column order) -> dense (n, n) matrix in the
    library's (reordered) index order.  lower_only: return the lower triangle (a factor L);
    otherwise mirror the lower triangle into the upper one (a symmetric matrix)."""
    M = np.zeros((T * nb, T * nb))
    t = 0
    for j in range(T):
        for i in range(j, T):
            M[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = slab[t * nb * nb:(t + 1) * nb * nb].reshape(nb, nb).T
            t += 1
    low = np.tril(M)
    M = low if lower_only else low + np.tril(M, -1).T
    return M[:n, :n]


def rel_err(a, b) -> float:
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def tile_entry_index(r, c, nb: int, T: int):
    """Flat slab index of entry (r, c), r >= c (arrays), in the library's lower-tile layout."""
    r = np.asarray(r)
    c = np.asarray(c)
    i, j = r // nb, c // nb
    t = j * T - j * (j - 1) // 2 + (i - j)
    return t * nb * nb + (r % nb) + (c % nb) * nb


def slab_lower_solve(slab: np.ndarray, nb: int, T: int, b: np.ndarray) -> np.ndarray:
    """y = L^-1 b with L given as a lower-tile slab (host-side check of the device solve)."""
    import scipy.linalg as sl
    y = np.zeros(T * nb)
    y[:len(b)] = b
    for m in range(T):
        t = m * T - m * (m - 1) // 2
        Lmm = slab[t * nb * nb:(t + 1) * nb * nb].reshape(nb, nb).T
        y[m * nb:(m + 1) * nb] = sl.solve_triangular(Lmm, y[m * nb:(m + 1) * nb], lower=True)
        for i in range(m + 1, T):
            ti = t + (i - m)
            Lim = slab[ti * nb * nb:(ti + 1) * nb * nb].reshape(nb, nb).T
            y[i * nb:(i + 1) * nb] -= Lim @ y[m * nb:(m + 1) * nb]
    return y
