"""The bounded waits of the tensor-core tile-update kernel: a wait budget too small for the
copies and MMAs to land makes every evaluation stop early with FBT_ERR_TIMEOUT, without a fault,
and the context gives the normal results again once the default budget is restored.

The kernel's exit path after a wait has run out waits (with its own, default-sized budget) for
the bulk copies and tensor-core operations it already issued, then frees its tensor memory, so
nothing asynchronous is in flight when the CTA exits."""
import numpy as np
import pytest

from oracle import fields
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_a_wait_that_runs_out_returns_timeout_and_the_context_stays_usable():
    require_gpu()
    import paper_2601_11437_gb300 as fbt
    n = 400
    locs = inputs.uniform_locations(n, 41)
    z = fields.sample_field(locs, inputs.standard_normal(n, 41), (1.0, 0.1, 0.7))
    theta = (0.9, 0.09, 0.8)
    ctx = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    ref = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    expect = fbt.mle_eval(ref, theta)
    fbt.fbt_set_spin_budget(ctx, 1)                 # one try per wait: the first copy is not there yet
    with pytest.raises(fbt.FbtError) as e:
        fbt.mle_eval(ctx, theta)
    assert e.value.status == fbt.FBT_ERR_TIMEOUT
    with pytest.raises(fbt.FbtError) as e:          # Algorithm 2 runs the same kernel
        fbt.mle_loglik(ctx, theta)
    assert e.value.status == fbt.FBT_ERR_TIMEOUT
    fbt.fbt_set_spin_budget(ctx, 0)                 # default budget
    got = fbt.mle_eval(ctx, theta)
    assert got[0] == expect[0] and np.array_equal(got[1], expect[1]) and np.array_equal(got[2], expect[2])
    fbt.fbt_destroy(ctx)
    fbt.fbt_destroy(ref)
