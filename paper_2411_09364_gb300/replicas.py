"""Host-side logic for running on N GPUs of one node.

The single-domain solve does not shard without all-to-all pencil transposes
(not built), so N GPUs run replicas; a batch of independent domains is split
across ranks by a greedy size-balanced assignment, with no collective on the
data path.  Timing takes the maximum over ranks.
"""
from __future__ import annotations

import os


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def shard_domains(sizes, world: int):
    """Greedy longest-processing-time assignment: list of index lists, one per rank."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += sizes[i]
    return [sorted(x) for x in out]


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
