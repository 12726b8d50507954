"""Instance sharding of the batched solve: a deterministic split that every
rank computes alone, checked on two gloo ranks (CPU)."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_2302_00752_gb300.shard import loads, partition_instances


def test_partition_covers_and_balances():
    w = [W.generic_stamp_count(2 * 10, s, 3) for s in range(5, 42, 2)] * 7
    for world in (1, 2, 3, 8):
        parts = partition_instances(w, world)
        ids = sorted(i for p in parts for i in p)
        assert ids == list(range(len(w)))
        ld = loads(w, parts)
        assert max(ld) - min(ld) <= max(w)       # LPT bound


def _worker(rank, world, port, weights, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = partition_instances(weights, world)[rank]
    t = torch.zeros(len(weights), dtype=torch.int64)
    t[mine] = rank + 1
    dist.all_reduce(t)
    q.put((rank, mine, t.tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree():
    weights = [float(i % 7 + 1) for i in range(29)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, weights, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    owners = res[0][2]
    assert res[1][2] == owners
    assert all(o in (1, 2) for o in owners)          # each instance owned by exactly one rank
    mine = {r: m for r, m, _ in res}
    assert sorted(mine[0] + mine[1]) == list(range(len(weights)))
