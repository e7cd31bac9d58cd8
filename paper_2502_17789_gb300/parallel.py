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
    """Sum the ranks' master-grid replicas in place (all-reduce); complex
    grids travel as their real and imaginary parts."""
    import torch
    import torch.distributed as dist

    buf = torch.view_as_real(grid) if grid.is_complex() else grid
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return grid


def sharded_step(grid_fn, degrid_fn, grid, world: int, group=None):
    """One grid + degrid step of a rank that owns a baseline shard: zero its
    master-grid replica, grid its visibilities into it (grid_fn(grid)), sum
    the replicas over the ranks (the one exchange step; skipped on one rank),
    then predict its visibilities from the model grid (degrid_fn()).  After
    it every rank holds the grid of the whole observation."""
    grid.zero_()
    grid_fn(grid)
    if world > 1:
        reduce_grids(grid, group)
    degrid_fn()
    return grid


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Maximum of a per-rank scalar (elapsed time) over all ranks."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def shard_observation(obs, rank: int, world: int):
    """(sub-observation, baseline indices) of `rank`'s round-robin shard;
    the whole observation on one rank."""
    bls = shard_baselines(obs.n_baselines, rank, world)
    return (obs, bls) if world == 1 else (sub_observation(obs, bls), bls)


def sub_observation(obs, baselines: np.ndarray):
    """The part of an observation that one rank grids: its baselines' uvw."""
    import copy

    sub = copy.copy(obs)
    sub.baselines = obs.baselines[baselines]
    sub.uvw = np.ascontiguousarray(obs.uvw[baselines])
    return sub
