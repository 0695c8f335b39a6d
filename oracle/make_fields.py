"""Write the stored synthetic fields z = L_true e of the large workloads (oracle only).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  For each named workload the locations and the
standard normal vector e come from the shared seeded generators; z = L_true e is computed with the
oracle's own Matern covariance and textbook Cholesky (fields.sample_field) and saved with a
checksum of the locations it belongs to.

    python -m oracle.make_fields n16384
    python -m oracle.make_fields batch2048      (the batched-fields workload, 2048 fields)
    python -m oracle.make_fields sim50          (the simulation study, 50 realisations each)
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

from . import fields, linalg

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden", "fields")


def locations_sha256(locs: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(locs, dtype="<f8").tobytes()).hexdigest()


def write_batch(inputs, count: int, name: str):
    """The batched-fields workload: every field's z, concatenated in field order, with the
    per-field offsets and a checksum of all locations."""
    t0 = time.time()
    fl = inputs.batched_fields(count)
    zs, h = [], hashlib.sha256()
    for f in fl:
        locs = inputs.uniform_locations(f.n, f.seed)
        h.update(np.ascontiguousarray(locs, dtype="<f8").tobytes())
        zs.append(fields.sample_field(locs, inputs.standard_normal(f.n, f.seed), f.theta_true))
    offsets = np.concatenate([[0], np.cumsum([f.n for f in fl])]).tolist()
    np.save(os.path.join(OUT, f"{name}_z.npy"), np.concatenate(zs).astype("<f8"))
    meta = dict(workload=name, fields=count, offsets_end=offsets[-1], locations_sha256=h.hexdigest(),
                recipe="paper_2601_11437_gb300.inputs.batched_fields", generator="oracle.fields.sample_field",
                command=f"python -m oracle.make_fields {name}", seconds=round(time.time() - t0, 1))
    with open(os.path.join(OUT, f"{name}_z.json"), "w") as fh:
        json.dump(meta, fh, indent=1)
    print(meta)


def write_sim(inputs, reps: int, name: str):
    """The simulation-study fields: for every setting and size, z_r = L e_r for r < reps with one
    oracle factor L of Sigma(theta_true) per (setting, size) on the shared design."""
    t0 = time.time()
    zs, h = [], hashlib.sha256()
    for n in inputs.SIM_SIZES:
        locs = inputs.sim_locations(n)
        h.update(np.ascontiguousarray(locs, dtype="<f8").tobytes())
        for si, th in enumerate(inputs.SIM_SETTINGS):
            S = fields.covariance_blocked(locs, th, jitter=1e-8, lower_only=True)
            L = linalg.cholesky(S, nb=256, overwrite=True)
            for r in range(reps):
                zs.append(L @ inputs.sim_normals(si, n, r))
            del S, L
    np.save(os.path.join(OUT, f"{name}_z.npy"), np.concatenate(zs).astype("<f8"))
    meta = dict(workload=name, reps=reps, order="for n in SIM_SIZES: for setting: for rep", jitter=1e-8,
                settings=inputs.SIM_SETTINGS, sizes=inputs.SIM_SIZES, locations_sha256=h.hexdigest(),
                recipe="paper_2601_11437_gb300.inputs.sim_locations / sim_normals",
                generator="oracle.fields.covariance_blocked + oracle.linalg.cholesky",
                command=f"python -m oracle.make_fields {name}", seconds=round(time.time() - t0, 1))
    with open(os.path.join(OUT, f"{name}_z.json"), "w") as fh:
        json.dump(meta, fh, indent=1)
    print(meta)


def main(names):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2601_11437_gb300 import inputs
    os.makedirs(OUT, exist_ok=True)
    for name in names:
        if name.startswith("batch"):
            write_batch(inputs, int(name[len("batch"):]), name)
            continue
        if name.startswith("sim"):
            write_sim(inputs, int(name[len("sim"):]), name)
            continue
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
