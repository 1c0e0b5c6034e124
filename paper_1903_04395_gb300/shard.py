"""Sharding colorings over ranks (one process per GPU).

Colorings are independent iterations of the estimator (Section 2.1; the
iteration count of Section 5.1 multiplies whole passes), so the counting path
shards by coloring with no exchange in the data path: every rank holds the
graph and counts a contiguous range of the seed sequence.  The only
collectives are after the counting - gathering the per-coloring colorful
maps (one double each) and taking the slowest rank's time.  These helpers
work on any torch.distributed backend (gloo on CPU, nccl on GPUs).
"""
from __future__ import annotations

import math

import numpy as np


def shard_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced range [lo, hi) of n_total items for `rank` of `world`."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_total >= 0")
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_seeds(first_seed: int, n_total: int, rank: int, world: int) -> np.ndarray:
    """The seeds of this rank's colorings: first_seed + i for i in its shard."""
    lo, hi = shard_range(n_total, rank, world)
    return np.arange(first_seed + lo, first_seed + hi, dtype=np.uint64)


def estimate_from_maps(maps, template, colors: int = 0) -> float:
    """The estimate over all ranks' colorful maps (gathered in seed order), computed by libsgc's
    sgc_estimate_from_maps for `template` (a Template or its handle)."""
    from . import sgc_estimate_from_maps
    handle = getattr(template, "handle", template)
    return sgc_estimate_from_maps(handle, maps, colors)


def gather_maps(local_maps, n_total: int, group=None) -> np.ndarray:
    """All ranks' per-coloring maps in seed order (every rank gets the whole array)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    lo, hi = shard_range(n_total, rank, world)
    local = np.asarray(local_maps, dtype=np.float64)
    if local.size != hi - lo:
        raise ValueError(f"rank {rank} holds {local.size} maps, its shard has {hi - lo}")
    width = math.ceil(n_total / world) if world else 0
    buf = torch.zeros(width, dtype=torch.float64)
    buf[:local.size] = torch.from_numpy(local)
    if dist.get_backend(group) == "nccl":
        buf = buf.cuda()
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    out = np.empty(n_total, dtype=np.float64)
    for r, part in enumerate(parts):
        a, b = shard_range(n_total, r, world)
        out[a:b] = part[:b - a].cpu().numpy()
    return out


def max_over_ranks(x: float, group=None) -> float:
    """The largest value of x over the ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
