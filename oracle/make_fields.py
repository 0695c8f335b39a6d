"""Write the stored synthetic fields z = L_true e of the large workloads (oracle only).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  For each named workload the locations and the
standard normal vector e come from the shared seeded generators; z = L_true e is computed with the
oracle's own Matern covariance and textbook Cholesky (fields.sample_field) and saved with a
checksum of the locations it belongs to.

    python -m oracle.make_fields n16384
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

from . import fields

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden", "fields")


def locations_sha256(locs: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(locs, dtype="<f8").tobytes()).hexdigest()


def main(names):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2601_11437_gb300 import inputs
    os.makedirs(OUT, exist_ok=True)
    for name in names:
        w = inputs.WORKLOADS[name]
        t0 = time.time()
        locs = w.locations()
        if w.n > 20000:
            z = fields.sample_field_blocked(locs, w.normals(), w.theta_true, jitter=w.jitter)
        else:
            z = fields.sample_field(locs, w.normals(), w.theta_true, jitter=w.jitter)
        np.save(os.path.join(OUT, f"{name}_z.npy"), z.astype("<f8"))
        meta = dict(workload=name, n=w.n, seed=w.seed, theta_true=w.theta_true, jitter=w.jitter,
                    locations_sha256=locations_sha256(locs), generator="oracle.fields.sample_field" + ("_blocked" if w.n > 20000 else ""),
                    command=f"python -m oracle.make_fields {name}", seconds=round(time.time() - t0, 1))
        with open(os.path.join(OUT, f"{name}_z.json"), "w") as f:
            json.dump(meta, f, indent=1)
        print(meta)


if __name__ == "__main__":
    main(sys.argv[1:] or ["n16384"])
