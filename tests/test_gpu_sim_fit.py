"""A field of the simulation study (Sec. 3) at its hardest setting, (sigma^2, alpha, nu) =
(0.05, 0.05, 0.05), n = 1600, fitted by Algorithm 1 from the L9 design (Table 1) over the study's
box, against the oracle's Algorithm 1 on the same stored field.

The oracle's fit is stored in tests/golden/sim_fit_n1600_nu005_rep*.json, written by
tests/golden/make_sim_fit.py from oracle/ alone (it takes minutes on the host).  Compared: the L9
pick (the same candidate, so bit-equal), every Fisher-iteration point of the trajectory, the
call counters, the final state (a shift to Nelder-Mead where the oracle shifts), theta_hat, l
and the final Fisher matrix."""
import glob
import json
import os

import numpy as np
import pytest

from paper_2601_11437_gb300 import inputs
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
RECORDS = sorted(glob.glob(os.path.join(HERE, "golden", "sim_fit_n1600_nu005_rep*.json")))


def stored_field(rep):
    from tests.golden.make_sim_fit import stored_field as sf
    return sf(rep)


@pytest.mark.parametrize("path", RECORDS, ids=[os.path.basename(p)[:-5] for p in RECORDS])
def test_simulation_field_fit_matches_oracle_algorithm1(path):
    require_gpu()
    import paper_2601_11437_gb300 as fbt
    rec = json.load(open(path))
    locs, z = stored_field(rec["rep"])
    lo, hi = inputs.SIM_BOX
    ctx = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    # the trajectory, step by step: the L9 pick, then every accepted Fisher-BT step
    st = fbt.fisher_bt_start(ctx, theta_lo=lo, theta_hi=hi)
    np.testing.assert_array_equal(np.array(st.theta[:]), rec["l9_pick"])
    points = [list(st.theta)]
    logliks = [st.loglik]
    while st.state == fbt.RUNNING:
        fbt.fisher_bt_step(ctx, st)
        points.append(list(st.theta))
        logliks.append(st.loglik)
    assert len(points) == len(rec["fisher_points"])
    np.testing.assert_allclose(np.array(points), np.array(rec["fisher_points"]), rtol=1e-7)
    # l is a sum of terms of size O(n) (-n/2 log 2 pi, -1/2 log det, -1/2 z^T Sigma^-1 z) that
    # nearly cancel along this trajectory: 1e-10 of those terms, not of l itself
    n = len(z)
    np.testing.assert_allclose(np.array(logliks), np.array(rec["fisher_logliks"]), rtol=1e-10, atol=1e-10 * n)
    # the whole run (the same start), Nelder-Mead included where the oracle shifts
    fin = fbt.fisher_bt_run(ctx, theta_lo=lo, theta_hi=hi)
    assert fin.state == rec["state"]
    assert (fin.iter, fin.n_ll, fin.n_grad) == (rec["iter"], rec["n_ll"], rec["n_grad"])
    np.testing.assert_allclose(np.array(fin.theta[:]), rec["theta_hat"], rtol=1e-6)
    assert fin.loglik == pytest.approx(rec["loglik"], rel=1e-10, abs=1e-10 * n)
    I, Iref = np.array(fin.fisher[:]).reshape(3, 3), np.array(rec["fisher"]).reshape(3, 3)
    d = np.sqrt(np.diag(Iref))
    assert np.all(np.abs(I - Iref) <= 1e-6 * np.outer(d, d))
    fbt.fbt_destroy(ctx)
