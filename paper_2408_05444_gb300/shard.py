"""Sharding of independent systems across ranks (one process per GPU).

Batched systems (one per colour channel of many images) are independent: each
rank solves its own subset and no collective touches the data path.  The
assignment is longest-processing-time first: systems sorted by decreasing
work (rows x columns of R), each given to the rank with the least work so far;
ties go to the lower rank and the lower system index, so every rank computes
the same assignment without communicating.
"""
from __future__ import annotations

import heapq


def shard_systems(work, world):
    """work: per-system cost (e.g. m * n).  Returns a list of `world` lists of
    system indices (each list in increasing index order)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda s: (-work[s], s))
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    out = [[] for _ in range(world)]
    for s in order:
        load, r = heapq.heappop(heap)
        out[r].append(s)
        heapq.heappush(heap, (load + work[s], r))
    return [sorted(x) for x in out]


def my_systems(work, rank, world):
    return shard_systems(work, world)[rank]


def max_over_ranks(value, group=None):
    """Largest value over all ranks (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
