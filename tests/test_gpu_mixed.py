"""The mixed path's tolerance switch, its per-tier task counts and the polish phase of
Algorithm 1 on mixed contexts.

* Tolerance 0 keeps all 7 digit planes: bitwise the emulated-FP64 results.
* Every tile product's tier follows from its operand tiles' largest entries against
  tau = mixed_tol * sigma^2, and every tier keeps the product within tau / 2: a looser tolerance
  skips more products, and l moves from the emulated value by no more than the products' bound.
* fisher_bt_run on a mixed context iterates in mixed precision until the Fisher direction is
  small, then switches to FP64-accurate products and finishes Algorithm 1 there: its estimate
  and counters after the switch match an FP64-accurate run continued from the same point, and
  the paper's stopping rule holds on FP64-accurate values.
"""
import numpy as np
import pytest

from oracle import fields, matern
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    require_gpu()


@pytest.fixture(scope="module")
def fld():
    locs = inputs.uniform_locations(650, 4)
    z = fields.sample_field(locs, inputs.standard_normal(650, 4), (1.5, 0.07, 0.8))
    return locs, z


def test_tolerance_zero_is_bitwise_emulated(fld):
    import paper_2601_11437_gb300 as fbt
    locs, z = fld
    theta = (1.2, 0.05, 0.63)
    mixed = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_MIXED, mixed_tol=1e-6)
    emu = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    assert fbt.fbt_get_mixed_tol(mixed) == 1e-6
    loose = fbt.mle_eval(mixed, theta)
    fbt.fbt_set_mixed_tol(mixed, 0.0)
    a, b = fbt.mle_eval(mixed, theta), fbt.mle_eval(emu, theta)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert loose[0] != b[0]
    with pytest.raises(fbt.FbtError):
        fbt.fbt_set_mixed_tol(emu, 0.0)          # not a mixed context
    with pytest.raises(fbt.FbtError):
        fbt.fbt_set_mixed_tol(mixed, -1.0)


@pytest.mark.parametrize("tol", [1e-12, 1e-9, 1e-6, 1e-4])
def test_tiers_and_the_tolerance_bound(fld, tol):
    import paper_2601_11437_gb300 as fbt
    locs, z = fld
    theta = (1.2, 0.05, 0.63)
    emu = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED, with_derivatives=False)
    ll_e = fbt.mle_loglik(emu, theta)
    ctx = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_MIXED, mixed_tol=tol, with_derivatives=False)
    fbt.fbt_mixed_counts(ctx, reset=True)
    ll_m = fbt.mle_loglik(ctx, theta)
    c = fbt.fbt_mixed_counts(ctx)
    # the Cholesky's trailing updates of a T = 6 tile factorisation: sum over k of (T-k-1)(T-k)/2
    # target tiles, two tasks each
    T = 6
    assert sum(c.values()) == sum((T - k - 1) * (T - k) for k in range(T - 1))
    # each entry of Sigma receives at most T - 1 tile products, each within tau / 2, so the
    # computed factor is that of Sigma + E with |E_ij| <= (T - 1) tau / 2 (plus rounding), and to
    # first order |d l| <= 1/2 |tr(Sigma^-1 E)| + 1/2 |w^T E w| <= 1/2 ||E||_2 (n / lambda_min + |w|^2)
    S = matern.covariance(locs, theta, partials=False)["S"]
    lam_min = np.linalg.eigvalsh(S)[0]
    w = np.linalg.solve(S, z)
    n = len(z)
    E2 = n * (T - 1) * tol * theta[0] / 2
    bound = 0.5 * E2 * (n / lam_min + w @ w)
    assert abs(ll_m - ll_e) <= 2 * bound + 1e-10 * abs(ll_e), (ll_m, ll_e, bound)
    if tol >= 1e-6:
        assert c["skipped"] + c["planes1"] + c["planes3"] > 0


def test_polish_switches_to_fp64_accurate_products_and_matches_the_emulated_estimate(fld):
    import paper_2601_11437_gb300 as fbt
    locs, z = fld
    theta0 = (1.0, 0.05, 0.7)
    emu = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    ref = fbt.fisher_bt_run(emu, theta0=theta0)
    assert ref.state == fbt.CONVERGED and ref.polish_iter == -1
    mixed = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_MIXED, mixed_tol=1e-6)
    st = fbt.fisher_bt_run(mixed, theta0=theta0)
    assert st.state == fbt.CONVERGED
    assert 0 <= st.polish_iter <= st.iter
    assert fbt.fbt_get_mixed_tol(mixed) == 1e-6                 # restored after the run
    th, th_ref = np.array(st.theta[:]), np.array(ref.theta[:])
    # the paper's stopping rule on FP64-accurate values: both estimates are stationary points of
    # the same l to ||grad l|| <= 1e-3, so they agree to about I^-1 1e-3
    assert np.linalg.norm(np.array(st.score[:])) <= 1e-3
    assert np.max(np.abs(th - th_ref) / th_ref) <= 1e-4
    # the estimate at the switch is within the polish step's reach of the final one
    tm = np.array(st.theta_mixed[:])
    assert np.max(np.abs(tm - th_ref) / th_ref) <= 1e-2
    # the polished state's l, score, Fisher are the emulated path's at the final theta
    fbt.fbt_set_mixed_tol(mixed, 0.0)
    ll, g, I = fbt.mle_eval(emu, tuple(th))
    assert st.loglik == ll and np.array_equal(np.array(st.score[:]), g)
