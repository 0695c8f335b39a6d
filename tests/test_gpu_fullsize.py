"""Parity at the full n = 16,384 workload in the launch configuration the bench times (tile size
128): sampled covariance entries against the oracle one by one, and properties that hold at any
size (L L^T = Sigma on sampled entries, the log-likelihood rebuilt from the device factor, the
score equal to finite differences of the device log-likelihood, a symmetric PSD Fisher matrix)."""
import hashlib
import json
import math
import os

import numpy as np
import pytest

from oracle import matern
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import require_gpu, slab_lower_solve, tile_entry_index

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "fp64_emulated"])
def full(request):
    require_gpu()
    import paper_2601_11437_gb300 as fbt
    w = inputs.WORKLOADS["n16384"]
    locs = w.locations()
    meta = json.load(open(os.path.join(ROOT, "tests", "golden", "fields", "n16384_z.json")))
    assert hashlib.sha256(np.ascontiguousarray(locs, dtype="<f8").tobytes()).hexdigest() == meta["locations_sha256"]
    z = np.load(os.path.join(ROOT, "tests", "golden", "fields", "n16384_z.npy"))
    ctx = fbt.fbt_create(locs, z, nb=128, precision=request.param)
    yield fbt, w, locs, z, ctx
    fbt.fbt_destroy(ctx)


def sample_pairs(n, count, seed):
    u = inputs.random_u64(seed, 7, 2 * count).reshape(count, 2) % np.uint64(n)
    r, c = u[:, 0].astype(np.int64), u[:, 1].astype(np.int64)
    return np.maximum(r, c), np.minimum(r, c)


def test_sampled_generation_entries(full):
    fbt, w, locs, z, ctx = full
    g = ctx.geometry()
    theta = w.theta0
    fbt.fbt_generate(ctx, theta, True)
    perm = fbt.fbt_copy_perm(ctx)
    r, c = sample_pairs(w.n, 3000, 11)
    idx = tile_entry_index(r, c, g["nb"], g["tiles"])
    lr, lc = locs[perm[r]], locs[perm[c]]
    h = np.sqrt((lr[:, 0] - lc[:, 0]) ** 2 + (lr[:, 1] - lc[:, 1]) ** 2)
    R, dRa, dRn = matern.correlation_parts(h / theta[1], theta[1], theta[2])
    diag = r == c
    ref = {0: theta[0] * np.where(diag, 1 + w.jitter, R), 1: theta[0] * dRa, 2: theta[0] * dRn}
    for which in (0, 1, 2):
        got = fbt.fbt_copy_slab(ctx, which)[idx]
        scale = np.max(np.abs(ref[which]))
        assert np.max(np.abs(got - ref[which])) <= 1e-12 * scale, which


def test_factor_reproduces_sigma_and_loglik(full):
    fbt, w, locs, z, ctx = full
    g = ctx.geometry()
    nb, T = g["nb"], g["tiles"]
    theta = w.theta_true
    ll = fbt.mle_loglik(ctx, theta)
    L = fbt.fbt_copy_slab(ctx, 0)
    perm = fbt.fbt_copy_perm(ctx)
    # log-likelihood rebuilt on the host from the device factor (Algorithm 2's last steps)
    d = L[tile_entry_index(np.arange(w.n), np.arange(w.n), nb, T)]
    assert np.all(d > 0)
    y = slab_lower_solve(L, nb, T, z[perm])
    ll_host = -0.5 * w.n * math.log(2 * math.pi) - np.sum(np.log(d)) - 0.5 * float(y @ y)
    assert ll == pytest.approx(ll_host, rel=1e-11)
    # (L L^T)_rc = Sigma_rc on sampled entries (rows of L gathered from the slab)
    r, c = sample_pairs(w.n, 200, 12)

    def row(i, upto):
        k = np.arange(upto + 1)
        return L[tile_entry_index(np.full_like(k, i), k, nb, T)]

    lr, lc = locs[perm[r]], locs[perm[c]]
    h = np.sqrt((lr[:, 0] - lc[:, 0]) ** 2 + (lr[:, 1] - lc[:, 1]) ** 2)
    R, _, _ = matern.correlation_parts(h / theta[1], theta[1], theta[2], partials=False)
    for q in range(len(r)):
        s_ref = theta[0] * (1 + w.jitter) if r[q] == c[q] else theta[0] * R[q]
        llt = float(row(r[q], c[q]) @ row(c[q], c[q]))
        assert abs(llt - s_ref) <= 1e-12 * theta[0]


def test_score_equals_finite_differences_and_fisher_is_psd(full):
    fbt, w, locs, z, ctx = full
    theta = np.array(w.theta0)
    ll, g, I = fbt.mle_eval(ctx, theta)
    assert ll == pytest.approx(fbt.mle_loglik(ctx, theta), rel=1e-12)
    np.testing.assert_array_equal(I, I.T)
    ev = np.linalg.eigvalsh(I)
    assert ev.min() > 0
    assert I[0, 0] == pytest.approx(w.n / (2 * theta[0] ** 2), rel=1e-15)
    for i in range(3):
        h = 1e-4 * theta[i]
        def cd(hh):
            tp, tm = theta.copy(), theta.copy()
            tp[i] += hh
            tm[i] -= hh
            return (fbt.mle_loglik(ctx, tp) - fbt.mle_loglik(ctx, tm)) / (2 * hh)
        fd = (4 * cd(h / 2) - cd(h)) / 3
        assert g[i] == pytest.approx(fd, rel=2e-6), (i, g[i], fd)
