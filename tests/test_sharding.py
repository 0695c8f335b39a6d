"""Host-side logic of the multi-rank batched-fields path: the cost-balanced partition, and the
gather of per-field result records across world_size 2 gloo ranks (CPU, no GPU)."""
import os
import socket

import numpy as np
import pytest

from paper_2601_11437_gb300 import inputs, sharding


def test_partition_covers_every_field_once_and_balances_cost():
    fl = inputs.batched_fields(256)
    costs = [f.n ** 3 for f in fl]
    for world in (1, 2, 3, 8):
        shards = sharding.partition(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(fl)))
        loads = [sum(costs[i] for i in s) for s in shards]
        # greedy LPT: the imbalance is at most the largest single cost
        assert max(loads) - min(loads) <= max(costs)
    assert sharding.partition(costs, 2) == sharding.partition(costs, 2)   # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nfields, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [(f * 37) % 11 + 1 for f in range(nfields)]
        mine = sharding.partition(costs, world)[rank]
        records = np.array([[f + k / 16.0 for k in range(sharding.RECORD)] for f in mine])
        out = sharding.gather_records(mine, records, nfields)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_gather_records_across_two_gloo_ranks():
    import torch.multiprocessing as mp
    nfields, world = 23, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, nfields, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = np.array([[f + k / 16.0 for k in range(sharding.RECORD)] for f in range(nfields)])
    for r in range(world):
        np.testing.assert_array_equal(got[r], expect)
