"""Pins for the oracle's dense linear algebra and Algorithms 2 and 3 (CPU only): library
routines, brute force in 50-digit arithmetic, the n = 1 closed form, finite differences of the
log-likelihood, the information identity by Monte Carlo, Eq. 4, and invariances."""
import math

import numpy as np
import pytest

from oracle import linalg, likelihood, matern, fields
from paper_2601_11437_gb300 import inputs


def spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


@pytest.mark.parametrize("n,nb", [(1, 64), (7, 3), (64, 64), (130, 32), (200, 64)])
def test_cholesky_and_solves(n, nb):
    A = spd(n, n)
    L = linalg.cholesky(A, nb=nb)
    assert np.all(np.triu(L, 1) == 0)
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(L @ L.T, A, rtol=1e-12, atol=1e-10)
    B = np.random.default_rng(1).standard_normal((n, 3))
    np.testing.assert_allclose(L @ linalg.solve_lower(L, B, nb=nb), B, atol=1e-10)
    np.testing.assert_allclose(L.T @ linalg.solve_lower_t(L, B, nb=nb), B, atol=1e-10)
    sign, ld = np.linalg.slogdet(A)
    assert sign == 1 and linalg.logdet_from_cholesky(L) == pytest.approx(ld, rel=1e-13)
    assert linalg.logdet_from_cholesky(L) == pytest.approx(np.sum(np.log(np.linalg.eigvalsh(A))), rel=1e-12)


@pytest.mark.parametrize("n,nb", [(1, 8), (37, 8), (100, 8), (131, 16)])
def test_cholesky_in_place_matches_the_library(n, nb):
    # the in-place variant used for the stored fields: trailing updates in column chunks of
    # 4 nb (several per step at these sizes) and the strict upper triangle zeroed block by block
    A = spd(n, 40 + n)
    W = np.array(A, copy=True)
    L = linalg.cholesky(W, nb=nb, overwrite=True)
    assert L is W and np.all(np.triu(L, 1) == 0)
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(L @ L.T, A, rtol=1e-12, atol=1e-10)


def test_cholesky_rejects_indefinite():
    A = spd(20, 3)
    A[5, 5] = -1.0
    with pytest.raises(linalg.NotPositiveDefinite):
        linalg.cholesky(A)


def test_trace_identity_eq4():
    rng = np.random.default_rng(5)
    A, B = rng.standard_normal((30, 30)), rng.standard_normal((30, 30))
    assert linalg.trace_product(A, B) == pytest.approx(float(np.trace(A @ B)), rel=1e-12)
    assert linalg.trace_product_eq4(A, B) == pytest.approx(float(np.trace(A @ B)), rel=1e-10)


def test_loglik_n1_closed_form():
    # one location: Sigma = sigma^2 (1 + delta), l = -log(2 pi)/2 - log(Sigma)/2 - z^2/(2 Sigma)
    locs = np.array([[0.3, 0.4]])
    th = (1.7, 0.2, 0.9)
    s = th[0] * (1 + 1e-8)
    ref = -0.5 * math.log(2 * math.pi) - 0.5 * math.log(s) - 0.5 * 0.81 / s
    assert likelihood.loglik(locs, np.array([0.9]), th) == pytest.approx(ref, rel=1e-15)
    ev = likelihood.loglik_score_fisher(locs, np.array([0.9]), th)
    assert ev.score[1] == 0 and ev.score[2] == 0
    assert ev.score[0] == pytest.approx((0.81 / s - 1) / (2 * th[0]), rel=1e-14)


@pytest.mark.parametrize("n", [3, 8])
def test_against_50_digit_brute_force(n):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    locs = inputs.uniform_locations(n, 21 + n)
    z = inputs.standard_normal(n, 21 + n)
    th = (1.3, 0.3, 0.7)
    mats = matern.covariance(locs, th)
    S = mpmath.matrix(mats["S"].tolist())
    Si = S ** -1
    zz = mpmath.matrix(z.tolist())
    quad = (zz.T * Si * zz)[0]
    ll_ref = -n / 2 * mpmath.log(2 * mpmath.pi) - mpmath.log(mpmath.det(S)) / 2 - quad / 2
    ev = likelihood.loglik_score_fisher(locs, z, th)
    assert ev.loglik == pytest.approx(float(ll_ref), rel=1e-12)
    w = Si * zz
    for i, key in enumerate(("S_sigma2", "S_alpha", "S_nu")):
        Di = mpmath.matrix(mats[key].tolist())
        Ai = Si * Di
        tr = sum(Ai[k, k] for k in range(n))
        sc = -tr / 2 + (w.T * Di * w)[0] / 2
        assert ev.score[i] == pytest.approx(float(sc), rel=1e-10, abs=1e-12)
        for j, key2 in enumerate(("S_sigma2", "S_alpha", "S_nu")):
            Aj = Si * mpmath.matrix(mats[key2].tolist())
            fij = sum((Ai * Aj)[k, k] for k in range(n)) / 2
            assert ev.fisher[i, j] == pytest.approx(float(fij), rel=1e-10, abs=1e-12)


def _ll(locs, z, th):
    return likelihood.loglik(locs, z, th)


def test_score_against_richardson_finite_differences():
    n = 60
    locs = inputs.uniform_locations(n, 2)
    th = np.array([0.8, 0.15, 1.1])
    z = fields.sample_field(locs, inputs.standard_normal(n, 2), th)
    ev = likelihood.loglik_score_fisher(locs, z, th)
    for i in range(3):
        def f(hh):
            tp, tm = th.copy(), th.copy()
            tp[i] += hh
            tm[i] -= hh
            return (_ll(locs, z, tp) - _ll(locs, z, tm)) / (2 * hh)
        h = 1e-3 * th[i]
        fd = (4 * f(h / 2) - f(h)) / 3             # Richardson on the central difference
        assert ev.score[i] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_fisher_symmetric_psd_and_sigma2_closed_forms():
    n = 80
    locs = inputs.uniform_locations(n, 4)
    th = (1.2, 0.12, 0.9)
    z = inputs.standard_normal(n, 4)
    ev = likelihood.loglik_score_fisher(locs, z, th)
    np.testing.assert_array_equal(ev.fisher, ev.fisher.T)
    assert np.min(np.linalg.eigvalsh(ev.fisher)) > -1e-12 * np.max(np.abs(ev.fisher))
    assert ev.fisher[0, 0] == pytest.approx(n / (2 * th[0] ** 2), rel=1e-15)
    # Step 2's closed forms against Eq. 2 / Eq. 3 with Sigma_sigma2 written out: without jitter the
    # two jitter modes are the same matrix, and mode 1 takes the general route
    e0 = likelihood.loglik_score_fisher(locs, z, th, jitter=0.0, mode=0)
    e1 = likelihood.loglik_score_fisher(locs, z, th, jitter=0.0, mode=1)
    np.testing.assert_allclose(e0.score, e1.score, rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(e0.fisher, e1.fisher, rtol=1e-8)


def test_information_identity_monte_carlo():
    # E[grad l] = 0 and Cov(grad l) = I(theta) when z ~ N(0, Sigma(theta)): a dropped term, a wrong
    # sign or a transposed factor in Eq. 2 / Eq. 3 breaks one of the two
    n, draws = 12, 3000
    locs = inputs.uniform_locations(n, 9)
    th = (1.0, 0.25, 0.9)
    S = matern.covariance(locs, th)["S"]
    L = np.linalg.cholesky(S)
    e = inputs.standard_normal(n * draws, 99).reshape(draws, n)
    scores = np.array([likelihood.loglik_score_fisher(locs, L @ e[d], th).score for d in range(draws)])
    I = likelihood.loglik_score_fisher(locs, L @ e[0], th).fisher
    sd = np.sqrt(np.diag(I))
    mean = scores.mean(axis=0)
    assert np.all(np.abs(mean) < 5 * sd / math.sqrt(draws))
    C = np.cov(scores.T)
    Cn = C / np.outer(sd, sd)
    In = I / np.outer(sd, sd)
    assert np.max(np.abs(Cn - In)) < 0.12


def test_permutation_and_scale_invariance():
    n = 70
    locs = inputs.uniform_locations(n, 6)
    th = (0.9, 0.1, 0.8)
    z = fields.sample_field(locs, inputs.standard_normal(n, 6), th)
    ev = likelihood.loglik_score_fisher(locs, z, th)
    perm = np.random.default_rng(0).permutation(n)
    ep = likelihood.loglik_score_fisher(locs[perm], z[perm], th)
    assert ep.loglik == pytest.approx(ev.loglik, rel=1e-12)
    np.testing.assert_allclose(ep.score, ev.score, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(ep.fisher, ev.fisher, rtol=1e-10)
    c = 3.0          # (s, alpha) -> (c s, c alpha): Sigma unchanged, d/dalpha scales by 1/c
    es = likelihood.loglik_score_fisher(locs * c, z, (th[0], c * th[1], th[2]))
    # scaled coordinates round differently: agreement up to kappa(Sigma) * eps
    assert es.loglik == pytest.approx(ev.loglik, rel=1e-11)
    np.testing.assert_allclose(es.score, ev.score * np.array([1, 1 / c, 1]), rtol=1e-9, atol=1e-9)
    D = np.diag([1, 1 / c, 1])
    np.testing.assert_allclose(es.fisher, D @ ev.fisher @ D, rtol=1e-9)


def test_domain_errors():
    locs = inputs.uniform_locations(5, 1)
    with pytest.raises(ValueError):
        likelihood.loglik(locs, np.zeros(5), (1.0, -0.1, 0.5))
    ev = likelihood.DenseEvaluator(locs, np.zeros(5))
    assert ev.loglik((1.0, 0.1, 0.0)) == -math.inf


def test_blocked_covariance_and_field_match_the_dense_ones():
    # the column-block covariance and in-place factor behind the large stored fields, against
    # the dense covariance and factor on a size that spans several column blocks
    n, th = 300, (1.3, 0.12, 0.9)
    locs = inputs.uniform_locations(n, 17)
    e = inputs.standard_normal(n, 17)
    S = matern.covariance(locs, th, partials=False)["S"]
    Sb = fields.covariance_blocked(locs, th, block=64)
    np.testing.assert_allclose(Sb, S, rtol=1e-15, atol=0)
    Sl = fields.covariance_blocked(locs, th, block=64, lower_only=True)
    low = np.tril_indices(n)
    np.testing.assert_allclose(Sl[low], S[low], rtol=1e-15, atol=0)
    z = fields.sample_field(locs, e, th)
    zb = fields.sample_field_blocked(locs, e, th)
    np.testing.assert_allclose(zb, z, rtol=1e-9, atol=1e-12 * np.max(np.abs(z)))
