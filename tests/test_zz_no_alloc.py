"""The allocation-free log-likelihood entry point (fbt_loglik_noalloc) against mle_loglik.

fbt_loglik_noalloc serves callers that cannot allocate device memory when they need l(theta):
its scratch is a fixed device array inside the library.  This file is collected last so that a
run stopping at the first failure has run every other test before it; it passes on its own in
a fresh process as well as after the rest of the suite.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import fields
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-10        # the relative tolerance of the FP64 parity tests


def noalloc_loglik(lib, locs, z, theta, jitter=1e-8, on_device=False):
    out = ctypes.c_double()
    th = (ctypes.c_double * 3)(*theta)
    if on_device:
        import torch
        tl = torch.tensor(locs, dtype=torch.float64, device="cuda")
        tz = torch.tensor(z, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = lib.fbt_loglik_noalloc(ctypes.c_void_p(tl.data_ptr()), ctypes.c_void_p(tz.data_ptr()), 1,
                                    len(z), th, jitter, ctypes.byref(out), None)
    else:
        locs = np.ascontiguousarray(locs, dtype=np.float64)
        z = np.ascontiguousarray(z, dtype=np.float64)
        st = lib.fbt_loglik_noalloc(locs.ctypes.data_as(ctypes.c_void_p), z.ctypes.data_as(ctypes.c_void_p), 0,
                                    len(z), th, jitter, ctypes.byref(out), None)
    return st, out.value


def test_noalloc_matches_mle_loglik_on_two_calls_in_a_row():
    require_gpu()
    import paper_2601_11437_gb300 as fbt
    lib = fbt._lib.load()
    assert lib.fbt_noalloc_max_n() == 1024
    cases = [
        (700, 21, (1.0, 0.1, 1.2), (0.8, 0.07, 0.9), False),   # larger problem first ...
        (333, 22, (1.0, 0.1, 0.5), (0.5, 0.05, 1.0), True),    # ... then a smaller one, device inputs
    ]
    for n, seed, th_true, theta, on_device in cases:
        locs = inputs.uniform_locations(n, seed)
        z = fields.sample_field(locs, inputs.standard_normal(n, seed), th_true)
        st, ll = noalloc_loglik(lib, locs, z, theta, on_device=on_device)
        assert st == 0, fbt.FbtError(st, "fbt_loglik_noalloc")
        ctx = fbt.fbt_create(locs, z, nb=64, with_derivatives=False)
        ref = fbt.mle_loglik(ctx, theta)
        fbt.fbt_destroy(ctx)
        assert math.isfinite(ll)
        assert ll == pytest.approx(ref, rel=TOL)


def test_noalloc_at_the_maximum_size():
    """n = FBT_NOALLOC_MAX_N: the tile slab nearly fills the scratch array."""
    require_gpu()
    import paper_2601_11437_gb300 as fbt
    lib = fbt._lib.load()
    n = lib.fbt_noalloc_max_n()
    locs = inputs.uniform_locations(n, 23)
    z = fields.sample_field(locs, inputs.standard_normal(n, 23), (1.0, 0.1, 0.8))
    theta = (0.9, 0.08, 0.7)
    st, ll = noalloc_loglik(lib, locs, z, theta)
    assert st == 0, fbt.FbtError(st, "fbt_loglik_noalloc")
    ctx = fbt.fbt_create(locs, z, nb=64, with_derivatives=False)
    ref = fbt.mle_loglik(ctx, theta)
    fbt.fbt_destroy(ctx)
    assert ll == pytest.approx(ref, rel=TOL)


def test_noalloc_call_after_a_failed_call_starts_clean():
    """A covariance that is not positive definite sets the status word; the next call clears it.

    All points at one location with no jitter give Sigma = sigma^2 * ones (rank one): with
    sigma^2 = 1 the second pivot of the Cholesky is exactly 0."""
    require_gpu()
    import paper_2601_11437_gb300 as fbt
    lib = fbt._lib.load()
    n = 50
    locs = np.tile([[0.25, 0.75]], (n, 1))
    z = inputs.standard_normal(n, 24)
    st, ll = noalloc_loglik(lib, locs, z, (1.0, 0.1, 0.5), jitter=0.0)
    assert st == fbt.FBT_ERR_NOT_PD and ll == -math.inf
    locs = inputs.uniform_locations(n, 24)
    z = fields.sample_field(locs, inputs.standard_normal(n, 24), (1.0, 0.1, 0.5))
    theta = (1.1, 0.09, 0.6)
    st, ll = noalloc_loglik(lib, locs, z, theta)
    assert st == 0 and math.isfinite(ll)
    ctx = fbt.fbt_create(locs, z, nb=64, with_derivatives=False)
    ref = fbt.mle_loglik(ctx, theta)
    fbt.fbt_destroy(ctx)
    assert ll == pytest.approx(ref, rel=TOL)


def test_noalloc_rejects_sizes_beyond_the_maximum_and_bad_parameters():
    require_gpu()
    import paper_2601_11437_gb300 as fbt
    lib = fbt._lib.load()
    n = lib.fbt_noalloc_max_n() + 1
    locs, z = inputs.uniform_locations(n, 1), inputs.standard_normal(n, 1)
    st, _ = noalloc_loglik(lib, locs, z, (1.0, 0.1, 0.5))
    assert st == fbt.FBT_ERR_ARG
    st, ll = noalloc_loglik(lib, locs[:10], z[:10], (1.0, -0.1, 0.5))
    assert st == fbt.FBT_ERR_DOMAIN and ll == -math.inf
