"""Write the oracle's Algorithm 1 fit of one simulation-study field (oracle only).

TEST INFRASTRUCTURE.  The field is realisation `rep` of the hardest setting of Sec. 3,
(sigma^2, alpha, nu) = (0.05, 0.05, 0.05), at n = 1600 on the study's shared design, as stored
by `python -m oracle.make_fields sim50`.  The fit starts from the L9 design (Table 1) over the
study's box theta^(l) = (0.01, 0.01, 0.01), theta^(u) = (5, 5, 2); at this setting the Fisher
iteration reaches the call limits of Sec. 2.1 and shifts to Nelder-Mead.  The record holds the
L9 pick, every Fisher-iteration point with its l, the counters, the final state, theta_hat, l and
the final Fisher matrix.

    python tests/golden/make_sim_fit.py [rep]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import fisher_bt, likelihood  # noqa: E402
from paper_2601_11437_gb300 import inputs  # noqa: E402

SETTING = 2          # (0.05, 0.05, 0.05)
N = 1600


def stored_field(rep: int, name: str = "sim50"):
    meta = json.load(open(os.path.join(HERE, "fields", f"{name}_z.json")))
    zall = np.load(os.path.join(HERE, "fields", f"{name}_z.npy"))
    reps = meta["reps"]
    o = 0
    for n in inputs.SIM_SIZES:
        for si in range(len(inputs.SIM_SETTINGS)):
            if n == N and si == SETTING:
                return inputs.sim_locations(n), zall[o + rep * n:o + (rep + 1) * n].copy()
            o += reps * n
    raise KeyError((N, SETTING))


def main(rep: int):
    locs, z = stored_field(rep)
    lo, hi = inputs.SIM_BOX
    t0 = time.time()
    ev = likelihood.DenseEvaluator(locs, z)
    st = fisher_bt.run(ev, theta_lo=lo, theta_hi=hi)
    rec = {"setting": list(inputs.SIM_SETTINGS[SETTING]), "n": N, "rep": rep, "field": "sim50",
           "box": [list(lo), list(hi)],
           "l9_pick": [float(v) for v in st.history[0][0]],
           "fisher_points": [[float(v) for v in th] for th, _ in st.history],
           "fisher_logliks": [float(ll) for _, ll in st.history],
           "state": int(st.state), "iter": int(st.iter), "n_ll": int(st.n_ll), "n_grad": int(st.n_grad),
           "theta_hat": [float(v) for v in st.theta], "loglik": float(st.loglik),
           "score": [float(v) for v in st.score], "fisher": np.asarray(st.fisher).ravel().tolist(),
           "command": f"python tests/golden/make_sim_fit.py {rep}", "seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, f"sim_fit_n{N}_nu005_rep{rep}.json"), "w") as fh:
        json.dump(rec, fh, indent=1)
    print({k: rec[k] for k in ("state", "iter", "n_ll", "n_grad", "theta_hat", "loglik", "seconds")})


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 0)
