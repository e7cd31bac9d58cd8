"""Host-side logic for running the path on several GPUs (one process each).

Gridding shards naturally: subgrids are independent, so ranks can own
disjoint baselines (the paper distributes channel ranges, Section 3.5) and
grid into their own FP64 master-grid replicas; the one exchange step is a sum
of those replicas.  Degridding needs the model grid on every rank and no
exchange.  The timing convention of a multi-rank run is the maximum over
ranks.  All functions take a torch.distributed process group and work with
either backend (gloo on CPU tensors, nccl on CUDA tensors).
"""
from __future__ import annotations

import numpy as np


def shard_baselines(n_baselines: int, rank: int, world: int) -> np.ndarray:
    """Baselines owned by `rank`: a round-robin split, so every rank gets
    long and short baselines alike (similar work per rank)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return np.arange(rank, n_baselines, world, dtype=np.int64)


def reduce_grids(grid, group=None):
    """Sum the ranks' master-grid replicas in place (all-reduce)."""
    import torch.distributed as dist

    dist.all_reduce(grid, op=dist.ReduceOp.SUM, group=group)
    return grid


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Maximum of a per-rank scalar (elapsed time) over all ranks."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sub_observation(obs, baselines: np.ndarray):
    """The part of an observation that one rank grids: its baselines' uvw."""
    import copy

    sub = copy.copy(obs)
    sub.baselines = obs.baselines[baselines]
    sub.uvw = np.ascontiguousarray(obs.uvw[baselines])
    return sub
