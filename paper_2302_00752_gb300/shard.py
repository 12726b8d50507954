"""Instance sharding for the batched solve on several GPUs.

The batched workload's instances are independent systems, so ranks split them
with no exchange on the data path: longest-processing-time-first greedy
assignment by an estimated cost (operator nonzeros), deterministic so every
rank computes the same split without communicating.
"""
from __future__ import annotations

import heapq


def partition_instances(weights, world):
    """Assign instance i (cost weights[i]) to ranks 0..world-1.  Returns one
    ascending list of instance ids per rank.  Heaviest first; each goes to the
    least-loaded rank, ties to the lowest rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(weights[i]), r))
    return [sorted(ids) for ids in out]


def loads(weights, parts):
    return [sum(float(weights[i]) for i in ids) for ids in parts]
