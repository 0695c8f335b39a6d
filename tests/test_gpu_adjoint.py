"""GPU parity of the adjoint gradient (Eq. 2 in trace form, Sigma^-1 from the factor, partials
regenerated inside the reduction) against the oracle's score, the Fisher path's score and
central finite differences of l; and the torch.autograd wrapper built on it."""
import numpy as np
import pytest

from oracle import fields, likelihood
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import rel_err, require_gpu

pytestmark = pytest.mark.gpu

# l is the Algorithm 2 value (same kernels as mle_loglik): 1e-10 relative.  The adjoint score is
# <w w^T - Sigma^-1, Sigma_i> / 2 with Sigma^-1 formed explicitly; its rounding error grows with
# kappa(Sigma) * eps * ||Sigma^-1|| ||Sigma_i|| instead of the transformed-trace form's, and
# 1e-8 relative to the largest score component bounds it on these fields (kappa up to ~1e7).
TOL_LL = 1e-10
TOL_GRAD = 1e-8


@pytest.fixture(scope="module", autouse=True)
def gpu():
    require_gpu()


def field(n, seed, theta_true):
    locs = inputs.uniform_locations(n, seed)
    return locs, fields.sample_field(locs, inputs.standard_normal(n, seed), theta_true)


CASES = [
    ("single_tile", 50, 6, (1.0, 0.2, 2.2), (1.1, 0.18, 1.9)),
    ("n400_theta0", 400, 0, (1.0, 0.1, 0.5), (0.5, 0.05, 1.0)),
    ("ragged_650", 650, 4, (1.5, 0.07, 0.8), (1.2, 0.05, 0.63)),
    ("ragged_1000", 1000, 9, (1.0, 0.1, 1.5), (0.9, 0.12, 1.3)),
]


@pytest.mark.parametrize("precision", [1, 2], ids=["fp64_emulated", "mixed"])
@pytest.mark.parametrize("name,n,seed,theta_true,theta", CASES, ids=[c[0] for c in CASES])
def test_adjoint_gradient_matches_oracle_score(name, n, seed, theta_true, theta, precision):
    import paper_2601_11437_gb300 as fbt
    locs, z = field(n, seed, theta_true)
    ref = likelihood.loglik_score_fisher(locs, z, theta)
    ctx = fbt.fbt_create(locs, z, nb=128, precision=precision)
    ll, g = fbt.mle_loglik_grad(ctx, theta)
    assert ll == pytest.approx(ref.loglik, rel=TOL_LL)
    assert rel_err(g, ref.score) < TOL_GRAD, (g, ref.score)
    # the sigma^2 component is Algorithm 3's closed form, the same as the Fisher path's
    _, g_eval, _ = fbt.mle_eval(ctx, theta)
    assert g[0] == g_eval[0]
    assert rel_err(g, g_eval) < TOL_GRAD
    fbt.fbt_destroy(ctx)


def test_adjoint_gradient_matches_central_differences():
    import paper_2601_11437_gb300 as fbt
    locs, z = field(700, 21, (1.0, 0.1, 0.9))
    theta = np.array([0.9, 0.085, 1.1])
    ctx = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    _, g = fbt.mle_loglik_grad(ctx, theta)
    fd = np.empty(3)
    for i in range(3):
        h = 1e-5 * theta[i]
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (fbt.mle_loglik(ctx, tp) - fbt.mle_loglik(ctx, tm)) / (2 * h)
    # central differences: truncation ~h^2 l''' and rounding ~eps |l| / h
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * np.abs(g).max())
    fbt.fbt_destroy(ctx)


def test_adjoint_reuses_the_factor_and_keeps_l_bitwise():
    import paper_2601_11437_gb300 as fbt
    locs, z = field(300, 16, (1.0, 0.1, 0.9))
    theta = (0.9, 0.08, 1.1)
    a = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    b = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    ll = fbt.mle_loglik(a, theta)
    ll_a, g_a = fbt.mle_loglik_grad(a, theta)
    assert fbt.fbt_factor_reuses(a) == 1
    ll_b, g_b = fbt.mle_loglik_grad(b, theta)
    assert fbt.fbt_factor_reuses(b) == 0
    assert ll == ll_a == ll_b
    assert np.array_equal(g_a, g_b)
    # and again: deterministic, and the inverse pass left the factor intact
    ll_c, g_c = fbt.mle_loglik_grad(b, theta)
    assert fbt.fbt_factor_reuses(b) == 1
    assert ll_c == ll_b and np.array_equal(g_c, g_b)


def test_adjoint_argument_checks():
    import paper_2601_11437_gb300 as fbt
    locs, z = field(200, 2, (1.0, 0.1, 0.5))
    native = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64)
    with pytest.raises(fbt.FbtError) as e:
        fbt.mle_loglik_grad(native, (1.0, 0.1, 0.5))
    assert e.value.status == fbt.FBT_ERR_ARG
    emu = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    with pytest.raises(fbt.FbtError) as e:
        fbt.mle_loglik_grad(emu, (1.0, -0.1, 0.5))
    assert e.value.status == fbt.FBT_ERR_DOMAIN


def test_autograd_function_backward_is_the_adjoint():
    import torch
    import paper_2601_11437_gb300 as fbt
    locs, z = field(500, 5, (1.0, 0.1, 0.7))
    ctx = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    theta = torch.tensor([0.8, 0.07, 0.9], dtype=torch.float64, requires_grad=True)
    ll = fbt.MaternLogLik.apply(ctx, theta)
    (-2.0 * ll).backward()
    ref = likelihood.loglik_score_fisher(locs, z, tuple(theta.detach().tolist()))
    assert ll.item() == pytest.approx(ref.loglik, rel=TOL_LL)
    assert rel_err(theta.grad.numpy(), -2.0 * ref.score) < TOL_GRAD
