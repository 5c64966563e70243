"""Splitting a batch of independent contractions over the ranks of a job.

The batched form has no exchange step: every pair is an independent problem,
so N GPUs each contract a disjoint subset of the pairs and only the results
travel.  Pairs are dealt by longest-processing-time first on their predicted
cost (the same flop model as the in-launch queue), which keeps the largest
rank load within one pair of the mean.  Host logic only; the gather works on
any torch.distributed backend (gloo on the host, NCCL on the GPUs).
"""
from __future__ import annotations

import heapq


def lpt_shards(costs, world: int):
    """Partition item indices 0..len(costs)-1 over ``world`` ranks.

    Items are taken in order of decreasing cost (ties by index) and each goes
    to the currently least loaded rank (ties by rank).  Returns one list of
    item indices per rank, each in the order the items were dealt."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return shards


def shard_loads(costs, shards):
    """Total cost per rank."""
    return [sum(float(costs[i]) for i in s) for s in shards]


def gather_values(local_index, local_values, n_items: int, group=None):
    """Assemble per-item float64 results computed on different ranks.

    ``local_index`` lists the items this rank computed and ``local_values``
    their results.  Every rank receives the full length-``n_items`` tensor
    (items nobody computed stay NaN)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n_local = torch.tensor([len(local_index)], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, n_local, group=group)
    width = int(max(int(c.item()) for c in counts))
    idx = torch.full((width,), -1, dtype=torch.int64)
    val = torch.full((width,), float("nan"), dtype=torch.float64)
    if len(local_index):
        idx[: len(local_index)] = torch.as_tensor(list(local_index), dtype=torch.int64)
        val[: len(local_index)] = torch.as_tensor(list(local_values), dtype=torch.float64)
    all_idx = [torch.empty_like(idx) for _ in range(world)]
    all_val = [torch.empty_like(val) for _ in range(world)]
    dist.all_gather(all_idx, idx, group=group)
    dist.all_gather(all_val, val, group=group)
    out = torch.full((n_items,), float("nan"), dtype=torch.float64)
    for ii, vv in zip(all_idx, all_val):
        keep = ii >= 0
        out[ii[keep]] = vv[keep]
    return out


def max_over_ranks(value: float, group=None) -> float:
    """Largest value of a scalar over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
