"""Sharding independent parts over the ranks of a job (one process per GPU).

The parts of a batch, the requests of a stream and the nodes of a scene are ordered
independently of one another (Sec. 3.4: every node's surfel set is computed on its own),
so they shard with no collective on the data path: each rank orders the parts that the
longest-processing-time rule assigns it, and the results are gathered to rank 0 over
torch.distributed (host objects; gloo or NCCL).  A single part is never split across
ranks: its greedy steps need the global maximum after every pick.
"""
from __future__ import annotations

import heapq
import math


def part_cost(n: int) -> float:
    """Relative ordering cost of an n-surfel part: the update sweeps visit about
    c * n * ln(n) points (each new point's ball holds about n / k points at step k)."""
    return float(n) * math.log(float(n) + 2.0)


def lpt_assign(sizes, world: int) -> list[list[int]]:
    """Longest processing time first: parts in decreasing cost (ties to the lower index),
    each to the rank with the least cost assigned so far (ties to the lower rank).
    Returns, per rank, its part indices in increasing order."""
    if world < 1:
        raise ValueError("world must be at least 1")
    order = sorted(range(len(sizes)), key=lambda i: (-part_cost(int(sizes[i])), i))
    heap = [(0.0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + part_cost(int(sizes[i])), r))
    return [sorted(o) for o in out]


def shard(sizes, world: int, rank: int) -> list[int]:
    """The part indices rank `rank` of `world` orders."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    return lpt_assign(sizes, world)[rank]


def order_sharded(keys, order_fn, world: int = 1, rank: int = 0, dist=None, **kw):
    """Orders this rank's LPT shard of `keys` (one entry per part, any type order_fn
    takes) with order_fn(keys_subset, part_ids, **kw) -> list of per-part results, and
    gathers every rank's results to rank 0.  Rank 0 returns the results of all parts in
    part order; the other ranks return None.  Part i is ordered with part_id = i, so its
    result does not depend on the rank that ordered it."""
    sizes = [len(k) for k in keys]
    mine = shard(sizes, world, rank)
    res = order_fn([keys[i] for i in mine], mine, **kw)
    local = dict(zip(mine, res))
    if world == 1 or dist is None:
        return [local[i] for i in range(len(keys))]
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(local, gathered, dst=0)
    if rank != 0:
        return None
    merged = {}
    for part in gathered:
        merged.update(part)
    return [merged[i] for i in range(len(keys))]


def gpu_order_fn(keys, part_ids, seed: int = 0, scales=None):
    """order_fn for order_sharded on this rank's GPU: one bs_order_batched launch over
    the shard (CUDA int64 key tensors), results copied to the host as numpy arrays."""
    from . import bs
    if not keys:
        return []
    out = bs.order_batched(keys, seeds=[seed] * len(keys), part_ids=list(part_ids),
                           scales=None if scales is None else [scales[i] for i in part_ids])
    return [tuple(t.cpu().numpy() for t in o) for o in out]
