"""Seeded synthetic inputs shared by the CUDA path's tests and bench and by the oracle's tests.

This module holds none of the method's arithmetic.  It provides
  * a counter-based random number generator (SplitMix64: Steele, Lea & Flood, OOPSLA 2014),
    written with numpy uint64 wrap-around arithmetic so every machine gets the same bits;
  * i.i.d. uniform locations on [0,1]^2 and i.i.d. standard normal draws (Box-Muller);
  * the workload recipes (sizes, seeds, true and starting parameters) of the Matern
    maximum-likelihood workloads.

The field itself, z = L_true e with L_true the Cholesky factor of Sigma(theta_true), is the
method's arithmetic and is therefore produced elsewhere (by the oracle, for the stored fields).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (bijective 64-bit mixer)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def random_u64(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` 64-bit words of SplitMix64 stream `stream` under `seed` (counter based)."""
    key = _mix64(np.array([(seed & 0xFFFFFFFF) << 32 | (stream & 0xFFFFFFFF)], dtype=np.uint64))[0]
    ctr = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = key + ctr * _GOLDEN
    return _mix64(state)


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each (exact, platform independent)."""
    return (random_u64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


STREAM_LOCS = 1
STREAM_NORMAL = 2
STREAM_BATCH = 3


def uniform_locations(n: int, seed: int) -> np.ndarray:
    """n locations i.i.d. uniform on [0,1)^2, shape (n, 2), row-major float64."""
    u = uniform01(seed, STREAM_LOCS, 2 * n)
    return np.ascontiguousarray(u.reshape(n, 2))


def standard_normal(n: int, seed: int) -> np.ndarray:
    """n i.i.d. N(0,1) draws by the Box-Muller transform of the uniform stream."""
    m = (n + 1) // 2
    u = uniform01(seed, STREAM_NORMAL, 2 * m).reshape(m, 2)
    r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))          # 1 - u in (0, 1]
    a = 2.0 * math.pi * u[:, 1]
    e = np.empty(2 * m)
    e[0::2] = r * np.cos(a)
    e[1::2] = r * np.sin(a)
    return e[:n]


@dataclass(frozen=True)
class Workload:
    """One Matern MLE workload: locations U[0,1]^2 (seeded), field z ~ N(0, Sigma(theta_true))."""
    name: str
    n: int
    seed: int
    theta_true: tuple
    theta0: tuple
    jitter: float = 1e-8
    description: str = ""

    def locations(self) -> np.ndarray:
        return uniform_locations(self.n, self.seed)

    def normals(self) -> np.ndarray:
        return standard_normal(self.n, self.seed)


WORKLOADS = {
    "n400": Workload("n400", 400, 0, (1.0, 0.1, 0.5), (0.5, 0.05, 1.0),
                     description="FP64, n=400, theta_true=(1, 0.1, 0.5), start (0.5, 0.05, 1.0)"),
    "n16384": Workload("n16384", 16384, 1, (1.0, 0.1, 1.2), (0.5, 0.05, 0.8),
                       description="FP64, n=16384, theta_true=(1, 0.1, 1.2), start (0.5, 0.05, 0.8)"),
    "n4096": Workload("n4096", 4096, 3, (1.0, 0.1, 1.2), (0.5, 0.05, 0.8),
                      description="FP64, n=4096 (profiling-size case of the n=16384 workload)"),
    "n65536": Workload("n65536", 65536, 2, (1.0, 0.05, 0.8), (0.7, 0.035, 0.64),
                       description="n=65536, theta_true=(1, 0.05, 0.8), start theta_true*(0.7,0.7,0.8)"),
    "n32768": Workload("n32768", 32768, 5, (1.0, 0.1, 1.5), (1.0, 0.1, 1.5),
                       description="FP64 adjoint, n=32768, evaluated at theta_true=(1, 0.1, 1.5)"),
}


def subsample(w: Workload, n_sub: int, seed_sub: int) -> np.ndarray:
    """Indices of a seeded subsample (without replacement) of the workload's locations."""
    keys = random_u64(seed_sub, STREAM_LOCS, w.n)
    return np.sort(np.argsort(keys, kind="stable")[:n_sub])


@dataclass(frozen=True)
class BatchField:
    n: int
    seed: int
    theta_true: tuple
    theta0: tuple


def batched_fields(count: int = 2048, seed: int = 4, n_lo: int = 256, n_hi: int = 4096) -> list:
    """Independent fields with n log-uniform in [n_lo, n_hi] and per-field true parameters
    sigma^2 ~ U[0.5, 2], alpha ~ U[0.02, 0.3], nu ~ U[0.3, 2.5]; start = truth * (0.7, 0.7, 0.8)."""
    u = uniform01(seed, STREAM_BATCH, 4 * count).reshape(count, 4)
    out = []
    for f in range(count):
        n = int(round(math.exp(math.log(n_lo) + u[f, 0] * (math.log(n_hi) - math.log(n_lo)))))
        th = (0.5 + 1.5 * u[f, 1], 0.02 + 0.28 * u[f, 2], 0.3 + 2.2 * u[f, 3])
        out.append(BatchField(n, seed * 1_000_003 + f, th, (0.7 * th[0], 0.7 * th[1], 0.8 * th[2])))
    return out


# Simulation study (Sec. 3): five true parameter settings, three sample sizes, replicated
# realisations, Fisher-BT started from the L9 design of Table 1 over the box below.
SIM_SETTINGS = ((1.0, 0.1, 0.5), (0.1, 0.1, 0.1), (0.05, 0.05, 0.05), (2.0, 0.8, 1.0), (1.5, 1.55, 1.3))
SIM_SIZES = (1600, 3600, 6400)
SIM_BOX = ((0.01, 0.01, 0.01), (5.0, 5.0, 2.0))
SIM_SEED = 7


def sim_locations(n: int) -> np.ndarray:
    """The design for sample size n: one seeded set of uniform locations, shared by all
    settings and realisations (the study varies the realisation, not the design)."""
    return uniform_locations(n, SIM_SEED * 1_000 + n)


def sim_normals(setting: int, n: int, rep: int) -> np.ndarray:
    """Standard normal vector of realisation rep of (setting, n)."""
    return standard_normal(n, SIM_SEED * 100_000_000 + setting * 1_000_000 + n * 100 + rep)
