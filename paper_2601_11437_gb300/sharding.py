"""Sharding of independent fields across ranks (one GPU per rank): the batched-fields workload
is the part of the method that partitions, with no exchange on the data path.  Fields go to
ranks by their cost (about n^3 per evaluation), largest first to the least-loaded rank; after
the fields are fitted, each field's 13-double result record (l, score, Fisher) is gathered in
field order.  Host-side logic only."""
from __future__ import annotations

import numpy as np


def partition(costs, world: int) -> list:
    """Field indices per rank: greedy longest-processing-time assignment, deterministic (ties by
    index and by rank number)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        shards[r].append(i)
        load[r] += float(costs[i])
    return [sorted(s) for s in shards]


RECORD = 13   # l, score[3], fisher[9]


def gather_records(local_index, local_records, nfields: int, group=None) -> np.ndarray:
    """All ranks' (field index, 13-double record) pairs assembled into a (nfields, 13) array in
    field order on every rank (torch.distributed all_gather of fixed-size tensors)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    local_index = np.asarray(local_index, dtype=np.int64)
    local_records = np.asarray(local_records, dtype=np.float64).reshape(-1, RECORD)
    count = len(local_index)
    # buffers sized by the largest shard
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([count], dtype=torch.int64), group=group)
    cap = max(1, int(max(int(s.item()) for s in sizes)))
    idx = torch.full((cap,), -1, dtype=torch.int64)
    rec = torch.zeros((cap, RECORD), dtype=torch.float64)
    idx[:count] = torch.from_numpy(local_index)
    rec[:count] = torch.from_numpy(local_records)
    all_idx = [torch.empty_like(idx) for _ in range(world)]
    all_rec = [torch.empty_like(rec) for _ in range(world)]
    dist.all_gather(all_idx, idx, group=group)
    dist.all_gather(all_rec, rec, group=group)
    out = np.full((nfields, RECORD), np.nan)
    seen = np.zeros(nfields, dtype=bool)
    for ii, rr in zip(all_idx, all_rec):
        ii = ii.numpy()
        rr = rr.numpy()
        for j, f in enumerate(ii):
            if f < 0:
                continue
            if seen[f]:
                raise RuntimeError(f"field {f} reported by two ranks")
            seen[f] = True
            out[f] = rr[j]
    if not seen.all():
        raise RuntimeError("fields missing from the gather")
    return out
