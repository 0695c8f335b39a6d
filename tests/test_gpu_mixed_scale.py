"""The mixed-precision scale workload (n = 65,536, theta_true = (1, 0.05, 0.8)) on the seeded
4,096-point subsample (subsample seed 3): the mixed and the emulated-FP64 paths against the
oracle's l, score and Fisher at theta^(0), and the mixed path against the emulated one.  The
full-size comparison of the two paths (including the Fisher-BT estimates) is the bench's
`--compare-mixed` mode."""
import hashlib
import json
import os

import numpy as np
import pytest

from oracle import likelihood
from paper_2601_11437_gb300 import inputs
from tests.gpu_util import rel_err, require_gpu

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELD = os.path.join(ROOT, "tests", "golden", "fields", "n65536_z")


def test_subsample_of_the_mixed_workload_matches_oracle():
    require_gpu()
    if not os.path.exists(FIELD + ".npy"):
        pytest.skip("the n65536 field is not stored")
    import paper_2601_11437_gb300 as fbt
    w = inputs.WORKLOADS["n65536"]
    locs = w.locations()
    meta = json.load(open(FIELD + ".json"))
    assert hashlib.sha256(np.ascontiguousarray(locs, dtype="<f8").tobytes()).hexdigest() == meta["locations_sha256"]
    z = np.load(FIELD + ".npy")
    idx = inputs.subsample(w, 4096, 3)
    ls, zs = locs[idx], z[idx]
    ref = likelihood.loglik_score_fisher(ls, zs, w.theta0)
    out = {}
    for name, prec in (("emulated", fbt.PREC_FP64_EMULATED), ("mixed", fbt.PREC_MIXED)):
        ctx = fbt.fbt_create(ls, zs, nb=128, precision=prec)
        out[name] = fbt.mle_eval(ctx, w.theta0)
        fbt.fbt_destroy(ctx)
    ll, g, I = out["emulated"]
    assert ll == pytest.approx(ref.loglik, rel=1e-10)
    assert rel_err(g, ref.score) < 1e-10 and rel_err(I, ref.fisher) < 1e-10
    ll_m, g_m, I_m = out["mixed"]
    assert ll_m == pytest.approx(ref.loglik, rel=1e-9)
    assert rel_err(g_m, ref.score) < 1e-8 and rel_err(I_m, ref.fisher) < 1e-8
