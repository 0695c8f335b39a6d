"""The autotuners: the FP64-accurate configuration per size band (FP64 DFMA tiles of 64 against
tensor-core tiles of 128) and the host-thread count of the batched entry points.  They choose how
the work runs, never what it computes: the chosen configurations agree with the oracle within
1e-10 per component, and the tuned thread count leaves the batched results bitwise unchanged."""
import numpy as np
import pytest

from oracle import fields, likelihood
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    require_gpu()


def test_fp64_path_autotune_picks_a_measured_configuration_and_caches_it():
    import paper_2601_11437_gb300 as fbt
    n = 600
    locs = inputs.uniform_locations(n, 51)
    z = fields.sample_field(locs, inputs.standard_normal(n, 51), (1.0, 0.1, 0.9))
    theta = (0.8, 0.08, 0.8)
    p, nb, secs, cached = fbt.fbt_autotune(locs, z, theta)
    assert (p, nb) in ((fbt.PREC_FP64, 64), (fbt.PREC_FP64_EMULATED, 128))
    assert secs["fp64_nb64"] > 0 and secs["emulated_nb128"] > 0 and not cached
    fastest = (fbt.PREC_FP64, 64) if secs["fp64_nb64"] < secs["emulated_nb128"] else (fbt.PREC_FP64_EMULATED, 128)
    assert (p, nb) == fastest
    # the same size band: the cached choice, without measuring
    p2, nb2, secs2, cached2 = fbt.fbt_autotune(locs[:520], z[:520], theta)
    assert cached2 and (p2, nb2) == (p, nb) and secs2 == secs
    ctx = fbt.fbt_create(locs, z, nb=nb, precision=p)
    ll, g, I = fbt.mle_eval(ctx, theta)
    ref = likelihood.loglik_score_fisher(locs, z, theta)
    assert abs(ll - ref.loglik) <= 1e-10 * abs(ref.loglik)
    assert np.all(np.abs(g - ref.score) <= 1e-10 * np.abs(ref.score))
    assert np.all(np.abs(I - ref.fisher) <= 1e-10 * np.abs(ref.fisher))
    fbt.fbt_destroy(ctx)


def test_batch_thread_autotune_leaves_results_unchanged():
    import paper_2601_11437_gb300 as fbt
    fl = inputs.batched_fields(12, seed=4, n_lo=100, n_hi=700)
    data = []
    for f in fl:
        locs = inputs.uniform_locations(f.n, f.seed)
        data.append((f, locs, fields.sample_field(locs, inputs.standard_normal(f.n, f.seed), f.theta_true)))
    ctxs = [fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED) for _, locs, z in data]
    thetas = np.array([f.theta0 for f, _, _ in data])
    best, secs = fbt.fbt_tune_batch_threads(ctxs, thetas, candidates=(2, 4, 8))
    assert best in (2, 4, 8) and all(v > 0 for v in secs.values())
    assert secs[best] == min(secs.values())
    a, sa = fbt.mle_eval_batch(ctxs, thetas[:, None, :], full=False, nthreads=best)
    b, sb = fbt.mle_eval_batch(ctxs, thetas[:, None, :], full=False, nthreads=1)
    assert (sa == 0).all() and np.array_equal(a, b)
    for c in ctxs:
        fbt.fbt_destroy(c)
