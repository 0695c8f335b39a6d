"""GPU tests of the batched-fields entry points: many independent fields, driven by a pool of
host threads on their own streams, must give bitwise the results of the same fields evaluated
one by one (every kernel's reductions have a fixed order), and the oracle's within 1e-10."""
import numpy as np
import pytest

from oracle import fields, likelihood
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import rel_err, require_gpu

pytestmark = pytest.mark.gpu

TOL_EVAL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def gpu():
    require_gpu()


@pytest.fixture(scope="module")
def small_batch():
    """Ten fields of the batched recipe, with n log-uniform in [100, 900] (oracle-sized)."""
    out = []
    for f in inputs.batched_fields(10, seed=4, n_lo=100, n_hi=900):
        locs = inputs.uniform_locations(f.n, f.seed)
        z = fields.sample_field(locs, inputs.standard_normal(f.n, f.seed), f.theta_true)
        out.append((f, locs, z))
    return out


def contexts(batch, precision, nb=128):
    import paper_2601_11437_gb300 as fbt
    return [fbt.fbt_create(locs, z, nb=nb, precision=precision) for _, locs, z in batch]


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "fp64_emulated", "mixed"])
def test_eval_batch_is_bitwise_the_one_by_one_path(small_batch, precision):
    import paper_2601_11437_gb300 as fbt
    thetas = np.array([[f.theta0, f.theta_true] for f, _, _ in small_batch])       # (F, 2, 3)
    ll, g, I, st = fbt.mle_eval_batch(contexts(small_batch, precision), thetas, nthreads=4)
    assert (st == fbt.FBT_OK).all()
    single = contexts(small_batch, precision)
    for q, c in enumerate(single):
        for j in range(2):
            l1, g1, I1 = fbt.mle_eval(c, thetas[q, j])
            assert ll[q, j] == l1 and np.array_equal(g[q, j], g1) and np.array_equal(I[q, j], I1)
    # loglik-only batch: the Algorithm 2 values
    ll2, st2 = fbt.mle_eval_batch(contexts(small_batch, precision), thetas, full=False)
    assert (st2 == fbt.FBT_OK).all()
    for q, c in enumerate(single):
        for j in range(2):
            assert ll2[q, j] == fbt.mle_loglik(c, thetas[q, j])


def test_eval_batch_matches_oracle(small_batch):
    import paper_2601_11437_gb300 as fbt
    sub = sorted(small_batch, key=lambda b: b[0].n)[:4]
    thetas = np.array([[f.theta0] for f, _, _ in sub])
    ll, g, I, st = fbt.mle_eval_batch(contexts(sub, 0), thetas)
    for q, (f, locs, z) in enumerate(sub):
        ref = likelihood.loglik_score_fisher(locs, z, f.theta0)
        assert ll[q, 0] == pytest.approx(ref.loglik, rel=TOL_EVAL)
        assert rel_err(g[q, 0], ref.score) < TOL_EVAL
        assert rel_err(I[q, 0], ref.fisher) < TOL_EVAL


def test_thread_count_does_not_change_results(small_batch):
    import paper_2601_11437_gb300 as fbt
    thetas = np.array([[f.theta0] for f, _, _ in small_batch])
    a = fbt.mle_eval_batch(contexts(small_batch, 1), thetas, nthreads=1)
    b = fbt.mle_eval_batch(contexts(small_batch, 1), thetas, nthreads=10)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def _same_state(a, b):
    return (list(a.theta) == list(b.theta) and a.loglik == b.loglik and list(a.score) == list(b.score)
            and list(a.fisher) == list(b.fisher) and (a.n_ll, a.n_grad, a.iter, a.state) ==
            (b.n_ll, b.n_grad, b.iter, b.state))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp64_emulated"])
def test_run_batch_is_bitwise_the_one_by_one_runs(small_batch, precision):
    import paper_2601_11437_gb300 as fbt
    sub = small_batch[:6]
    theta0s = np.array([f.theta0 for f, _, _ in sub])
    states, status = fbt.fisher_bt_run_batch(contexts(sub, precision), theta0s)
    assert (status == fbt.FBT_OK).all()
    for q, c in enumerate(contexts(sub, precision)):
        ref = fbt.fisher_bt_run(c, theta0s[q])
        assert _same_state(states[q], ref), q
        assert states[q].state in (fbt.CONVERGED, fbt.DONE_NM)


def test_lockstep_steps_match_one_by_one_steps(small_batch):
    import paper_2601_11437_gb300 as fbt
    sub = small_batch[:5]
    theta0s = np.array([f.theta0 for f, _, _ in sub])
    ctxs = contexts(sub, 1)
    states, status = fbt.fisher_bt_start_batch(ctxs, theta0s)
    assert (status == fbt.FBT_OK).all()
    for _ in range(40):
        if all(s.state != fbt.RUNNING for s in states):
            break
        assert (fbt.fisher_bt_step_batch(ctxs, states) == fbt.FBT_OK).all()
    for q, c in enumerate(contexts(sub, 1)):
        ref = fbt.fisher_bt_start(c, theta0s[q])
        while ref.state == fbt.RUNNING and ref.iter < 40:
            fbt.fisher_bt_step(c, ref)
        assert _same_state(states[q], ref), q


def test_batch_statuses_and_argument_checks(small_batch):
    import paper_2601_11437_gb300 as fbt
    sub = small_batch[:3]
    ctxs = contexts(sub, 0)
    thetas = np.array([[f.theta0] for f, _, _ in sub])
    thetas[1, 0, 1] = -0.1                      # outside the domain: that field only
    ll, st = fbt.mle_eval_batch(ctxs, thetas, full=False)
    assert st[1, 0] == fbt.FBT_ERR_DOMAIN and ll[1, 0] == -np.inf
    assert st[0, 0] == st[2, 0] == fbt.FBT_OK
    with pytest.raises(fbt.FbtError) as e:      # one context twice would race with itself
        fbt.mle_eval_batch([ctxs[0], ctxs[0]], thetas[:2], full=False)
    assert e.value.status == fbt.FBT_ERR_ARG
