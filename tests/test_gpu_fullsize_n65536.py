"""Parity at the n = 65,536 workload in the launch configuration the bench times (emulated-FP64
tile products, tile size 128): sampled covariance entries against the oracle one by one, and
properties that hold at any size (L L^T = Sigma on sampled entries, the log-likelihood rebuilt
from the device factor, the score equal to finite differences of the device log-likelihood, a
symmetric PSD Fisher matrix with the closed-form sigma^2 entry).

The factor slab (17 GB) is copied device to device into a torch buffer; sampled entries are
gathered there and only they come back to the host.  The forward solve of the rebuilt
log-likelihood runs tile column by tile column with torch on the device (data movement and
checking only)."""
import hashlib
import json
import math
import os

import numpy as np
import pytest

from oracle import matern
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import require_gpu, tile_entry_index

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NAME = "n65536"


@pytest.fixture(scope="module")
def full():
    require_gpu()
    import torch
    import paper_2601_11437_gb300 as fbt
    w = inputs.WORKLOADS[NAME]
    locs = w.locations()
    meta = json.load(open(os.path.join(ROOT, "tests", "golden", "fields", f"{NAME}_z.json")))
    assert hashlib.sha256(np.ascontiguousarray(locs, dtype="<f8").tobytes()).hexdigest() == meta["locations_sha256"]
    z = np.load(os.path.join(ROOT, "tests", "golden", "fields", f"{NAME}_z.npy"))
    ctx = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    g = ctx.geometry()
    buf = torch.empty(g["tiles"] * (g["tiles"] + 1) // 2 * g["nb"] ** 2, dtype=torch.float64, device="cuda")
    yield fbt, torch, w, locs, z, ctx, buf
    fbt.fbt_destroy(ctx)
    del buf
    torch.cuda.empty_cache()


def copy_slab(fbt, torch, ctx, which, buf):
    fbt._check(fbt._lib.load().fbt_copy_slab(ctx.handle, which, fbt.C.c_void_p(buf.data_ptr()), 1), "fbt_copy_slab")
    torch.cuda.synchronize()
    return buf


def gather(torch, buf, idx):
    return buf[torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int64)).to(buf.device)].cpu().numpy()


def sample_pairs(n, count, seed):
    u = inputs.random_u64(seed, 7, 2 * count).reshape(count, 2) % np.uint64(n)
    r, c = u[:, 0].astype(np.int64), u[:, 1].astype(np.int64)
    return np.maximum(r, c), np.minimum(r, c)


def test_sampled_generation_entries(full):
    fbt, torch, w, locs, z, ctx, buf = full
    g = ctx.geometry()
    theta = w.theta0
    fbt.fbt_generate(ctx, theta, True)
    perm = fbt.fbt_copy_perm(ctx)
    r, c = sample_pairs(w.n, 3000, 13)
    idx = tile_entry_index(r, c, g["nb"], g["tiles"])
    lr, lc = locs[perm[r]], locs[perm[c]]
    h = np.sqrt((lr[:, 0] - lc[:, 0]) ** 2 + (lr[:, 1] - lc[:, 1]) ** 2)
    R, dRa, dRn = matern.correlation_parts(h / theta[1], theta[1], theta[2])
    diag = r == c
    ref = {0: theta[0] * np.where(diag, 1 + w.jitter, R), 1: theta[0] * dRa, 2: theta[0] * dRn}
    for which in (0, 1, 2):
        got = gather(torch, copy_slab(fbt, torch, ctx, which, buf), idx)
        scale = np.max(np.abs(ref[which]))
        assert np.max(np.abs(got - ref[which])) <= 1e-12 * scale, which


def test_factor_reproduces_sigma_and_loglik(full):
    fbt, torch, w, locs, z, ctx, buf = full
    g = ctx.geometry()
    nb, T = g["nb"], g["tiles"]
    assert T * nb == w.n
    theta = w.theta_true
    ll = fbt.mle_loglik(ctx, theta)
    L = copy_slab(fbt, torch, ctx, 0, buf)
    perm = fbt.fbt_copy_perm(ctx)
    d = gather(torch, L, tile_entry_index(np.arange(w.n), np.arange(w.n), nb, T))
    assert np.all(d > 0)
    # y = L^-1 z[perm], tile column by tile column (the tiles of one column are contiguous)
    y = torch.from_numpy(np.ascontiguousarray(z[perm])).to(L.device)
    for m in range(T):
        t = m * T - m * (m - 1) // 2
        Lmm = L[t * nb * nb:(t + 1) * nb * nb].view(nb, nb).t()
        ym = torch.linalg.solve_triangular(Lmm, y[m * nb:(m + 1) * nb].view(nb, 1), upper=False).view(nb)
        y[m * nb:(m + 1) * nb] = ym
        if m + 1 < T:
            below = L[(t + 1) * nb * nb:(t + T - m) * nb * nb].view(T - m - 1, nb, nb).transpose(1, 2)
            y[(m + 1) * nb:] -= (below @ ym).reshape(-1)
    yy = float(torch.dot(y, y))
    ll_host = -0.5 * w.n * math.log(2 * math.pi) - float(np.sum(np.log(d))) - 0.5 * yy
    assert ll == pytest.approx(ll_host, rel=1e-10)
    # (L L^T)_rc = Sigma_rc on sampled entries (rows of L gathered from the slab)
    r, c = sample_pairs(w.n, 200, 14)

    def row(i, upto):
        k = np.arange(upto + 1)
        return gather(torch, L, tile_entry_index(np.full_like(k, i), k, nb, T))

    lr, lc = locs[perm[r]], locs[perm[c]]
    h = np.sqrt((lr[:, 0] - lc[:, 0]) ** 2 + (lr[:, 1] - lc[:, 1]) ** 2)
    R, _, _ = matern.correlation_parts(h / theta[1], theta[1], theta[2], partials=False)
    for q in range(len(r)):
        s_ref = theta[0] * (1 + w.jitter) if r[q] == c[q] else theta[0] * R[q]
        llt = float(row(r[q], c[q]) @ row(c[q], c[q]))
        assert abs(llt - s_ref) <= 1e-12 * theta[0]


def test_score_equals_finite_differences_and_fisher_is_psd(full):
    fbt, torch, w, locs, z, ctx, buf = full
    theta = np.array(w.theta0)
    ll, gr, I = fbt.mle_eval(ctx, theta)
    assert ll == pytest.approx(fbt.mle_loglik(ctx, theta), rel=1e-12)
    np.testing.assert_array_equal(I, I.T)
    assert np.linalg.eigvalsh(I).min() > 0
    assert I[0, 0] == pytest.approx(w.n / (2 * theta[0] ** 2), rel=1e-15)
    for i in range(3):
        h = 1e-4 * theta[i]

        def cd(hh):
            tp, tm = theta.copy(), theta.copy()
            tp[i] += hh
            tm[i] -= hh
            return (fbt.mle_loglik(ctx, tp) - fbt.mle_loglik(ctx, tm)) / (2 * hh)
        fd = (4 * cd(h / 2) - cd(h)) / 3
        assert gr[i] == pytest.approx(fd, rel=1e-5), (i, gr[i], fd)
