"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element on
seeded inputs (several tiles and a ragged tail), plus edge cases and error statuses."""
import math

import numpy as np
import pytest

from oracle import fields, linalg, likelihood, matern, fisher_bt
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import rel_err, require_gpu, slab_to_dense

pytestmark = pytest.mark.gpu

# Tolerances.  Covariance entries: both sides evaluate the same exact function to ~1e-15
# relative, and x = h / alpha rounds differently by an ulp, which moves R by ~x eps; 1e-12 of the
# largest entry covers both.  l / score / Fisher: 1e-10 relative (FP64 path).
TOL_ENTRY = 1e-12
TOL_EVAL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def gpu():
    require_gpu()


def field(n, seed, theta_true=(1.0, 0.1, 0.5)):
    locs = inputs.uniform_locations(n, seed)
    z = fields.sample_field(locs, inputs.standard_normal(n, seed), theta_true)
    return locs, z


def dense_from_ctx(fbt, ctx, which, lower_only=False):
    g = ctx.geometry()
    return slab_to_dense(fbt.fbt_copy_slab(ctx, which), g["nb"], g["tiles"], g["n"], lower_only)


@pytest.mark.parametrize("n,nb", [(1, 64), (63, 64), (200, 64), (333, 128), (400, 128)])
@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (0.5, 0.05, 1.0), (1.3, 0.2, 1.73), (0.8, 0.03, 0.31)])
def test_generation_matches_oracle(n, nb, theta):
    import paper_2601_11437_gb300 as fbt
    locs, z = inputs.uniform_locations(n, 11), inputs.standard_normal(n, 11)
    ctx = fbt.fbt_create(locs, z, nb=nb)
    fbt.fbt_generate(ctx, theta, True)
    perm = fbt.fbt_copy_perm(ctx)
    assert sorted(perm.tolist()) == list(range(n))
    ref = matern.covariance(locs[perm], theta)
    for which, key in ((0, "S"), (1, "S_alpha"), (2, "S_nu")):
        got = dense_from_ctx(fbt, ctx, which)
        assert rel_err(got, ref[key]) < TOL_ENTRY, (which, rel_err(got, ref[key]))
    fbt.fbt_destroy(ctx)


@pytest.mark.parametrize("theta", [(0.05, 0.05, 0.05), (0.1, 0.1, 0.1), (1.5, 1.55, 1.3), (2.0, 0.8, 1.0),
                                   (1.0, 0.02, 2.5), (1.0, 0.3, 4.0), (1.0, 0.015, 0.6)],
                         ids=["nu0.05", "nu0.1", "alpha1.55", "alpha0.8", "nu2.5", "nu4", "alpha0.015"])
def test_generation_matches_oracle_at_extreme_parameters(theta):
    # the simulation study's settings and beyond: tiny nu (slowly decaying quadrature terms),
    # ranges far above the domain (every x below 1, many nodes) and far below it (x up to 90,
    # the finer levels), large nu
    import paper_2601_11437_gb300 as fbt
    n = 257
    locs, z = inputs.uniform_locations(n, 12), inputs.standard_normal(n, 12)
    ctx = fbt.fbt_create(locs, z, nb=128)
    fbt.fbt_generate(ctx, theta, True)
    perm = fbt.fbt_copy_perm(ctx)
    ref = matern.covariance(locs[perm], theta)
    for which, key in ((0, "S"), (1, "S_alpha"), (2, "S_nu")):
        got = dense_from_ctx(fbt, ctx, which)
        assert rel_err(got, ref[key]) < TOL_ENTRY, (which, rel_err(got, ref[key]))
    fbt.fbt_destroy(ctx)


def test_padding_is_identity():
    import paper_2601_11437_gb300 as fbt
    n, nb = 70, 64
    ctx = fbt.fbt_create(inputs.uniform_locations(n, 2), inputs.standard_normal(n, 2), nb=nb)
    fbt.fbt_generate(ctx, (1.0, 0.1, 0.7), True)
    g = ctx.geometry()
    full = slab_to_dense(fbt.fbt_copy_slab(ctx, 0), nb, g["tiles"], g["npad"])
    np.testing.assert_array_equal(full[n:, n:], np.eye(g["npad"] - n))
    np.testing.assert_array_equal(full[n:, :n], 0.0)
    for which in (1, 2):
        d = slab_to_dense(fbt.fbt_copy_slab(ctx, which), nb, g["tiles"], g["npad"])
        np.testing.assert_array_equal(d[n:, :], 0.0)


@pytest.mark.parametrize("n,nb,precision", [(63, 64, 0), (257, 64, 0), (400, 128, 0), (400, 128, 1), (1000, 128, 1)])
def test_cholesky_factor_matches_oracle(n, nb, precision):
    import paper_2601_11437_gb300 as fbt
    locs, z = field(n, 5)
    theta = (1.0, 0.1, 0.5)
    ctx = fbt.fbt_create(locs, z, nb=nb, with_derivatives=False, precision=precision)
    ll = fbt.mle_loglik(ctx, theta)
    perm = fbt.fbt_copy_perm(ctx)
    S = matern.covariance(locs[perm], theta, partials=False)["S"]
    Lref = linalg.cholesky(S)
    Lgpu = dense_from_ctx(fbt, ctx, 0, lower_only=True)
    assert rel_err(Lgpu, Lref) < 1e-12
    assert ll == pytest.approx(likelihood.loglik(locs, z, theta), rel=TOL_EVAL)


CASES = [
    ("n400_theta0", 400, 0, (1.0, 0.1, 0.5), (0.5, 0.05, 1.0), 128),
    ("n400_truth", 400, 0, (1.0, 0.1, 0.5), (1.0, 0.1, 0.5), 64),
    ("ragged_333", 333, 3, (1.0, 0.1, 1.2), (0.7, 0.08, 0.9), 64),
    ("ragged_650", 650, 4, (1.5, 0.07, 0.8), (1.2, 0.05, 0.63), 128),
    ("single_tile", 50, 6, (1.0, 0.2, 2.2), (1.1, 0.18, 1.9), 64),
]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp64_emulated"])
@pytest.mark.parametrize("name,n,seed,theta_true,theta,nb", CASES, ids=[c[0] for c in CASES])
def test_loglik_score_fisher_match_oracle(name, n, seed, theta_true, theta, nb, precision):
    import paper_2601_11437_gb300 as fbt
    if precision == 1:
        nb = 128           # the emulated path works on 128 x 128 tiles
    locs, z = field(n, seed, theta_true)
    ctx = fbt.fbt_create(locs, z, nb=nb, precision=precision)
    ll, g, I = fbt.mle_eval(ctx, theta)
    ref = likelihood.loglik_score_fisher(locs, z, theta)
    assert ll == pytest.approx(ref.loglik, rel=TOL_EVAL)
    assert rel_err(g, ref.score) < TOL_EVAL, (g, ref.score)
    assert rel_err(I, ref.fisher) < TOL_EVAL, (I, ref.fisher)
    np.testing.assert_array_equal(I, I.T)
    assert fbt.mle_loglik(ctx, theta) == pytest.approx(ref.loglik, rel=TOL_EVAL)
    fbt.fbt_destroy(ctx)


def test_results_are_bitwise_reproducible_and_order_invariant():
    import paper_2601_11437_gb300 as fbt
    locs, z = field(300, 9)
    theta = (0.9, 0.09, 0.7)
    ctx = fbt.fbt_create(locs, z, nb=64)
    a = fbt.mle_eval(ctx, theta)
    b = fbt.mle_eval(ctx, theta)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    ctx2 = fbt.fbt_create(locs, z, nb=64, reorder=False)
    c = fbt.mle_eval(ctx2, theta)
    assert c[0] == pytest.approx(a[0], rel=1e-11)
    assert rel_err(c[1], a[1]) < 1e-9 and rel_err(c[2], a[2]) < 1e-10


def test_domain_and_not_pd_statuses():
    import paper_2601_11437_gb300 as fbt
    locs, z = field(100, 2)
    ctx = fbt.fbt_create(locs, z, nb=64)
    assert fbt.mle_loglik(ctx, (1.0, -0.1, 0.5)) == -math.inf
    assert fbt.mle_loglik(ctx, (1.0, 0.1, float("nan"))) == -math.inf
    with pytest.raises(fbt.FbtError) as e:
        fbt.mle_eval(ctx, (0.0, 0.1, 0.5))
    assert e.value.status == fbt.FBT_ERR_DOMAIN
    # two coincident locations, no jitter, sigma^2 = 1: the second pivot is exactly 0
    same = np.array([[0.25, 0.5], [0.25, 0.5]])
    c2 = fbt.fbt_create(same, np.array([0.3, -0.2]), nb=64, jitter=0.0)
    assert fbt.mle_loglik(c2, (1.0, 0.1, 0.5)) == -math.inf
    with pytest.raises(fbt.FbtError) as e:
        fbt.mle_eval(c2, (1.0, 0.1, 0.5))
    assert e.value.status == fbt.FBT_ERR_NOT_PD
    # the context stays usable after a failed evaluation
    assert np.isfinite(fbt.mle_loglik(ctx, (1.0, 0.1, 0.5)))


def test_set_field_and_device_inputs():
    import torch
    import paper_2601_11437_gb300 as fbt
    locs, z = field(180, 12)
    theta = (1.0, 0.1, 0.5)
    ctx = fbt.fbt_create(torch.tensor(locs, device="cuda"), torch.tensor(z, device="cuda"), nb=64)
    ll0 = fbt.mle_loglik(ctx, theta)
    assert ll0 == pytest.approx(likelihood.loglik(locs, z, theta), rel=TOL_EVAL)
    z2 = -0.5 * z
    fbt.fbt_set_field(ctx, z2)
    assert fbt.mle_loglik(ctx, theta) == pytest.approx(likelihood.loglik(locs, z2, theta), rel=TOL_EVAL)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp64_emulated"])
def test_fisher_bt_run_matches_oracle_trajectory(precision):
    import paper_2601_11437_gb300 as fbt
    w = inputs.WORKLOADS["n400"]
    locs = w.locations()
    z = fields.sample_field(locs, w.normals(), w.theta_true)
    ctx = fbt.fbt_create(locs, z, nb=128, precision=precision)
    st = fbt.fisher_bt_run(ctx, theta0=w.theta0)
    ref = fisher_bt.run(likelihood.DenseEvaluator(locs, z), theta0=w.theta0)
    assert st.state == ref.state
    assert (st.iter, st.n_ll, st.n_grad) == (ref.iter, ref.n_ll, ref.n_grad)
    np.testing.assert_allclose(np.array(st.theta[:]), ref.theta, rtol=1e-8)
    assert st.loglik == pytest.approx(ref.loglik, rel=1e-10)
    if st.state == fbt.CONVERGED:
        assert np.linalg.norm(np.array(st.score[:])) <= 1e-3


def test_l9_start_matches_oracle():
    import paper_2601_11437_gb300 as fbt
    locs, z = field(300, 14, (1.0, 0.1, 0.5))
    lo, hi = (0.01, 0.01, 0.01), (5.0, 5.0, 2.0)
    ctx = fbt.fbt_create(locs, z, nb=64)
    st = fbt.fisher_bt_start(ctx, theta_lo=lo, theta_hi=hi)
    ref = fisher_bt.start(likelihood.DenseEvaluator(locs, z), theta_lo=lo, theta_hi=hi)
    np.testing.assert_array_equal(np.array(st.theta[:]), ref.theta)
    assert (st.n_ll, st.n_grad, st.state) == (ref.n_ll, ref.n_grad, ref.state) == (10, 1, st.state)
    assert st.loglik == pytest.approx(ref.loglik, rel=TOL_EVAL)


def test_shift_to_nelder_mead_and_final_fisher(monkeypatch):
    import paper_2601_11437_gb300 as fbt
    locs, z = field(200, 15, (1.0, 0.1, 0.5))
    bt = fbt.default_bt_opts()
    bt.max_grad_calls = 1                 # force the shift after the second gradient call
    ctx = fbt.fbt_create(locs, z, nb=64)
    st = fbt.fisher_bt_run(ctx, theta0=(0.5, 0.05, 1.0), bt=bt)
    monkeypatch.setattr(fisher_bt, "MAX_GRAD_CALLS", 1)
    ref = fisher_bt.run(likelihood.DenseEvaluator(locs, z), theta0=(0.5, 0.05, 1.0))
    assert st.state == fbt.DONE_NM and ref.state == fisher_bt.DONE_NM
    np.testing.assert_allclose(np.array(st.theta[:]), ref.theta, rtol=1e-4)
    assert st.loglik == pytest.approx(ref.loglik, rel=1e-8)
    Iref = likelihood.loglik_score_fisher(locs, z, tuple(st.theta[:])).fisher
    assert rel_err(np.array(st.fisher[:]).reshape(3, 3), Iref) < TOL_EVAL


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp64_emulated"])
def test_factor_reuse_at_the_accepted_point_is_bitwise_identical(precision):
    # Algorithm 1 evaluates l at the accepted point in the line search and then runs the Fisher
    # iteration there: the second evaluation reuses the Cholesky factor of the first
    import paper_2601_11437_gb300 as fbt
    locs, z = field(300, 16, (1.0, 0.1, 0.9))
    theta = (0.9, 0.08, 1.1)
    a = fbt.fbt_create(locs, z, nb=128, precision=precision)
    b = fbt.fbt_create(locs, z, nb=128, precision=precision)
    ll_a = fbt.mle_loglik(a, theta)
    ea = fbt.mle_eval(a, theta)
    assert fbt.fbt_factor_reuses(a) == 1
    eb = fbt.mle_eval(b, theta)
    assert fbt.fbt_factor_reuses(b) == 0
    assert ea[0] == eb[0] == ll_a
    assert np.array_equal(ea[1], eb[1]) and np.array_equal(ea[2], eb[2])
    # a different theta, or a generation in between, does not reuse
    fbt.mle_loglik(a, (0.9, 0.08, 1.2))
    fbt.mle_eval(a, theta)
    assert fbt.fbt_factor_reuses(a) == 1


def test_mixed_path_matches_oracle_at_default_tolerance_and_emulated_when_strict():
    import paper_2601_11437_gb300 as fbt
    locs, z = field(650, 4, (1.5, 0.07, 0.8))
    theta = (1.2, 0.05, 0.63)
    ref = likelihood.loglik_score_fisher(locs, z, theta)
    mixed = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_MIXED)          # tol 1e-12
    ll, g, I = fbt.mle_eval(mixed, theta)
    assert ll == pytest.approx(ref.loglik, rel=1e-9)
    assert rel_err(g, ref.score) < 1e-8 and rel_err(I, ref.fisher) < 1e-8
    # a tolerance below every product's size keeps all 8 digit planes: the emulated-FP64 results
    strict = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_MIXED, mixed_tol=1e-300)
    emu = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    a, b = fbt.mle_eval(strict, theta), fbt.mle_eval(emu, theta)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    # a loose tolerance drops planes and moves the result, within its bound
    loose = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_MIXED, mixed_tol=1e-6)
    c = fbt.mle_eval(loose, theta)
    assert c[0] != b[0] and abs(c[0] - b[0]) < 1e-3 * abs(b[0])


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp64_emulated"])
def test_line_search_partials_are_kept_for_the_accepted_point(precision):
    # the line search's Algorithm 2 evaluation writes Sigma_alpha and Sigma_nu with Sigma; the
    # Algorithm 3 evaluation at the accepted candidate then generates nothing, bitwise the same
    import paper_2601_11437_gb300 as fbt
    locs, z = field(500, 17, (1.0, 0.1, 0.9))
    a = fbt.fbt_create(locs, z, nb=128, precision=precision)
    st = fbt.fisher_bt_start(a, (0.8, 0.08, 1.0))
    fbt.fbt_profile(a, True)
    fbt.fisher_bt_step(a, st)
    prof = fbt.fbt_profile_read(a)
    fbt.fbt_profile(a, False)
    assert prof["generate_deriv"]["launches"] == st.halvings + 1
    assert "generate" not in prof
    b = fbt.fbt_create(locs, z, nb=128, precision=precision)
    ll, g, I = fbt.mle_eval(b, tuple(st.theta))
    assert st.loglik == ll
    assert np.array_equal(np.array(st.score[:]), g) and np.array_equal(np.array(st.fisher[:]).reshape(3, 3), I)
    # a plain mle_loglik in between (another theta) leaves the kept partials usable only at theirs
    th = tuple(st.theta)
    fbt.mle_loglik(a, (0.7, 0.07, 0.9))
    e = fbt.mle_eval(a, th)
    assert e[0] == ll and np.array_equal(e[1], g)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp64_emulated"])
def test_graph_replay_is_bitwise_the_direct_path(precision):
    # every evaluation kind, several times: the first runs directly, the second is captured, the
    # rest replay the graph; a context with graphs off must give the same bits throughout
    import paper_2601_11437_gb300 as fbt
    locs, z = field(420, 23, (1.0, 0.1, 0.9))
    a = fbt.fbt_create(locs, z, nb=128, precision=precision)
    b = fbt.fbt_create(locs, z, nb=128, precision=precision)
    fbt.fbt_set_graphs(b, False)
    for ctx in (a, b):
        ctx.trace = []
    thetas = [(0.9, 0.08, 1.1), (1.1, 0.12, 0.8), (0.7, 0.05, 1.4)]
    for rep in range(3):
        for th in thetas:
            for ctx in (a, b):
                ctx.trace.append(fbt.mle_loglik(ctx, th))                 # Algorithm 2
                ll, g, I = fbt.mle_eval(ctx, th)                           # reuses the factor
                ctx.trace += [ll, *g, *I.ravel()]
                st = fbt.fisher_bt_start(ctx, th)                          # fresh eval + step machinery
                fbt.fisher_bt_step(ctx, st)                                # kept partials path
                ctx.trace += [st.loglik, *st.theta[:], *st.score[:]]
    assert a.trace == b.trace
    assert fbt.fbt_graph_count(a) >= 3 and fbt.fbt_graph_count(b) == 0, fbt._lib.load().fbt_last_cuda_error()
