"""Per-component parity of l, the score and the Fisher matrix (Eq. 1-3) against the oracle.

Every entry is compared with its own oracle value (not with the largest entry of its vector or
matrix).  Two kinds of case:

* well-conditioned fields (kappa(Sigma) u <= 1e-11): every entry of l, grad l and I within 1e-10
  of its own oracle value, on the FP64, emulated-FP64 and mixed paths;
* extreme parameters (the simulation study's corners and beyond), where kappa(Sigma) reaches
  1e11 and no two correct FP64 implementations agree to 1e-10.  There each entry is held to a
  bound derived from the conditioning: a backward-stable Cholesky perturbs Sigma by
  E with |E| <~ sqrt(n) u |Sigma|, which moves Sigma^-1 by kappa sqrt(n) u relative, so
      |d l| <= tol |l|,  |d l_i| <= tol (|tr A_i| + |w^T Sigma_i w|) / 2,
      |d I_ij| <= tol sqrt(I_ii I_jj)      with tol = max(1e-10, 2 sqrt(n) kappa u)
  (the score's scale is the size of the two terms of Eq. 2 it is the difference of; the Fisher
  entry's is its Cauchy-Schwarz bound, as I_ij is an inner product <B_i, B_j> / 2).  Alongside,
  the factor's backward error is checked entry by entry, which does not depend on kappa(Sigma):
      |(L L^T - Sigma)_rc| <= 4 (n + kappa_d) u sqrt(Sigma_rr Sigma_cc)   (+ the mixed tolerance)
  where kappa_d = max_k kappa(L_kk) over the diagonal factor tiles: the tensor-core path solves
  each panel L_ik L_kk^T = A_ik by a product with the explicit inverse W_k = L_kk^-1, whose
  backward error grows with kappa(L_kk) (a triangular solve's would not).
"""
import math

import numpy as np
import pytest

from oracle import fields, likelihood, matern
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import require_gpu, slab_to_dense

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def gpu():
    require_gpu()


def field(n, seed, theta_true):
    locs = inputs.uniform_locations(n, seed)
    z = fields.sample_field(locs, inputs.standard_normal(n, seed), theta_true)
    return locs, z


def component_errors(got, ref, scale=None):
    """|got - ref| / max(|ref|, scale) entry by entry (scale: per-entry floor, or None)."""
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    den = np.abs(ref) if scale is None else np.maximum(np.abs(ref), np.asarray(scale, float))
    return np.abs(got - ref) / np.maximum(den, 1e-300)


def check_eval(ll, g, I, ref, tol, scaled=False):
    """l, score and Fisher entry by entry; scaled=True uses the cancellation scales above."""
    e_ll = abs(ll - ref.loglik) / abs(ref.loglik)
    s_scale = 0.5 * (np.abs(ref.trace) + np.abs(ref.qform)) if scaled else None
    d = np.sqrt(np.diag(ref.fisher))
    f_scale = np.outer(d, d) if scaled else None
    e_g = component_errors(g, ref.score, s_scale)
    e_I = component_errors(I, ref.fisher, f_scale)
    msg = f"l {e_ll:.2e} score {e_g} fisher {e_I.ravel()} (tol {tol:.1e})"
    assert e_ll <= tol and np.all(e_g <= tol) and np.all(e_I <= tol), msg
    return max(e_ll, e_g.max(), e_I.max())


CASES = [
    ("n400_theta0", 400, 0, (1.0, 0.1, 0.5), (0.5, 0.05, 1.0)),
    ("n400_truth", 400, 0, (1.0, 0.1, 0.5), (1.0, 0.1, 0.5)),
    ("ragged_333", 333, 3, (1.0, 0.1, 1.2), (0.7, 0.08, 0.9)),
    ("ragged_650", 650, 4, (1.5, 0.07, 0.8), (1.2, 0.05, 0.63)),
]


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "fp64_emulated", "mixed"])
@pytest.mark.parametrize("name,n,seed,theta_true,theta", CASES, ids=[c[0] for c in CASES])
def test_every_component_within_1e10(name, n, seed, theta_true, theta, precision):
    import paper_2601_11437_gb300 as fbt
    locs, z = field(n, seed, theta_true)
    nb = 64 if precision == 0 else 128
    ctx = fbt.fbt_create(locs, z, nb=nb, precision=precision)
    ll, g, I = fbt.mle_eval(ctx, theta)
    fbt.fbt_destroy(ctx)
    ref = likelihood.loglik_score_fisher(locs, z, theta)
    check_eval(ll, g, I, ref, TOL)


EXTREME = [(0.05, 0.05, 0.05), (1.0, 0.015, 0.6), (1.0, 0.3, 4.0), (1.5, 1.55, 1.3)]


def kappa(S):
    ev = np.linalg.eigvalsh(S)
    return float(ev[-1] / ev[0])


@pytest.mark.parametrize("precision", [1, 2], ids=["fp64_emulated", "mixed"])
@pytest.mark.parametrize("theta", EXTREME, ids=["nu0.05", "alpha0.015", "nu4", "alpha1.55"])
def test_extreme_parameters_on_the_tensor_core_paths(theta, precision):
    import paper_2601_11437_gb300 as fbt
    n = 1000
    locs, z = field(n, 31, theta)
    ctx = fbt.fbt_create(locs, z, nb=128, precision=precision)
    ll = fbt.mle_loglik(ctx, theta)
    perm = fbt.fbt_copy_perm(ctx)
    g_ = ctx.geometry()
    Lg = slab_to_dense(fbt.fbt_copy_slab(ctx, 0), g_["nb"], g_["tiles"], n, lower_only=True)
    ll2, g, I = fbt.mle_eval(ctx, theta)
    fbt.fbt_destroy(ctx)
    assert ll2 == ll
    S = matern.covariance(locs[perm], theta, partials=False)["S"]
    # the factor's backward error, entry by entry (independent of kappa(Sigma)); the diagonal
    # tiles' condition numbers come from the oracle's factor in the library's order
    Lref = np.linalg.cholesky(S)
    nb = g_["nb"]
    kd = max(np.linalg.cond(Lref[k:k + nb, k:k + nb]) for k in range(0, n, nb))
    d = np.sqrt(np.diag(S))
    bound = 4 * (n + kd) * U * np.outer(d, d)
    if precision == 2:
        T = g_["tiles"]
        bound = bound + 4 * T * 1e-12 * theta[0]          # default mixed_tol 1e-12 per tile product
    E = np.abs(Lg @ Lg.T - S)
    assert np.all(E <= bound), f"backward error {np.max(E / bound):.2f} of its bound"
    k = kappa(S)
    tol = max(TOL, 2 * math.sqrt(n) * k * U)
    ref = likelihood.loglik_score_fisher(locs, z, theta)
    check_eval(ll2, g, I, ref, tol, scaled=True)
