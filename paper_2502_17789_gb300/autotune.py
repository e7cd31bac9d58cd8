"""Autotuner for the batched launch.

Chooses, for one observation, the subgrid size L, the launch mode (one block
per work item, or a persistent grid draining the work queue), the gridder's
records per chunk (how many staged visibilities one bulk copy brings into
shared memory; Section 3.2 leaves the gridder's thread shape a per-device
tunable) and the degridder's channels per lane (1: one visibility per lane;
2 or 4: phasors of later channels by rotation), by timing a grid + degrid
pass on the observation's own plans with CUDA events.  The search is
staged: every (L, mode) with the default chunk and one channel per lane,
then the chunk for the best (L, mode), then the channels per lane for the
best of those.  The winner is cached in a JSON file keyed by the GPU and
the observation's shape.  Changing L changes the partition and hence the
numbers (legitimately: each L has its own oracle result); the other choices
do not.

The timing function is injectable so the selection and cache logic can be
tested without a GPU.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

CANDIDATE_L = (64, 96, 128)
MODES = ("blocks", "persistent")
GRID_CHUNKS = (32, 48, 64)      # staged records per gridder chunk; 48 is the library's default
DEGRID_CHANNELS = (1, 2, 4)     # channels per degridder lane; 1 is the library's default
DEFAULT_CHUNK, DEFAULT_CHANNELS = 48, 1


@dataclass
class Choice:
    subgrid_size: int
    mode: str
    grid_chunk: int
    degrid_channels: int
    ms: float
    timings: dict = field(default_factory=dict)

    def as_dict(self):
        return {"subgrid_size": self.subgrid_size, "mode": self.mode, "grid_chunk": self.grid_chunk,
                "degrid_channels": self.degrid_channels, "ms": self.ms, "timings": self.timings}

    def plan_kwargs(self, idg) -> dict:
        """Keyword arguments of idg.Plan that apply this choice."""
        return {"subgrid_size": self.subgrid_size, "flags": idg.IDG_PERSISTENT if self.mode == "persistent" else 0,
                "grid_chunk": self.grid_chunk, "degrid_channels": self.degrid_channels}


def shape_key(obs, device_name: str) -> str:
    """Cache key: GPU name, geometry and table shape.  The longest baseline
    (in grid pixels at the top frequency) stands in for the occupancy
    distribution, which depends on L."""
    u = np.abs(obs.uvw[..., :2]).max() * obs.freqs.max() / 299792458.0 * obs.image_size if obs.n_vis else 0.0
    return (f"{device_name}|N{obs.grid_size}|fov{obs.image_size:.6g}|P{obs.kernel_padding}|bl{obs.n_baselines}"
            f"|t{obs.n_timesteps}|ch{obs.n_channels}|int{obs.n_intervals}|reach{int(u)}")


def _load_cache(path):
    if path and os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _save_cache(path, cache):
    if not path:
        return
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def gpu_measure(obs, subgrid_size, mode, grid_chunk=DEFAULT_CHUNK, degrid_channels=DEFAULT_CHANNELS, trials=2,
                aterms=None, graph=False, vis=None):
    """Time one grid + degrid pass (ms, best of `trials`) on a plan with the
    given settings; None if the plan cannot be made (e.g. w too large).
    With `graph`, the passes are CUDA-graph replays on a side stream."""
    import torch

    from . import idg

    dev = torch.device("cuda")
    side = torch.cuda.Stream(dev) if graph else None
    flags = idg.IDG_PERSISTENT if mode == "persistent" else 0
    try:
        plan = idg.Plan(obs, subgrid_size=subgrid_size, flags=flags, stream=side.cuda_stream if graph else None,
                        grid_chunk=grid_chunk, degrid_channels=degrid_channels)
    except idg.IdgError:
        return None
    own_vis = vis is None
    if own_vis:
        g = torch.Generator(device=dev)
        g.manual_seed(0)
        vis = torch.randn((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64,
                          device=dev, generator=g)
    if aterms is None:
        from . import synth
        aterms = synth.aterms_identity(obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    A = torch.as_tensor(aterms, device=dev)
    N = obs.grid_size
    G = torch.zeros((4, N, N), dtype=torch.complex128, device=dev)
    out = torch.empty_like(vis)
    s = side if graph else torch.cuda.current_stream(dev)
    if graph:
        torch.cuda.synchronize(dev)  # inputs made on the current stream are ready for the side stream
    best = None
    for t in range(trials + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        if graph:
            plan.grid_graph(vis, A, G)
            plan.degrid_graph(G, A, out)
        else:
            plan.grid(vis, A, G)
            plan.degrid(G, A, out)
        e1.record(s)
        plan.synchronize()
        if t > 0:
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    plan.close()
    del G, out
    if own_vis:
        del vis
    torch.cuda.empty_cache()
    return best


def autotune(obs, *, candidates=CANDIDATE_L, modes=MODES, chunks=GRID_CHUNKS, channels=DEGRID_CHANNELS,
             cache_path=None, device_name=None, measure=None, refresh=False) -> Choice:
    """Return the fastest (L, mode, chunk, channels per lane) for `obs`,
    from the cache when the key is present, else by the staged search."""
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    measure = measure or gpu_measure
    key = shape_key(obs, device_name)
    cache = _load_cache(cache_path)
    if not refresh and key in cache:
        c = cache[key]
        return Choice(c["subgrid_size"], c["mode"], c.get("grid_chunk", DEFAULT_CHUNK),
                      c.get("degrid_channels", DEFAULT_CHANNELS), c["ms"], c.get("timings", {}))
    timings = {}
    best = None

    def trial(L, mode, chunk, ch):
        nonlocal best
        name = f"L{L}/{mode}/chunk{chunk}/ch{ch}"
        if name in timings:
            return
        ms = measure(obs, L, mode, chunk, ch)
        timings[name] = ms
        if ms is not None and (best is None or ms < best.ms):
            best = Choice(L, mode, chunk, ch, ms)

    for L in candidates:                    # stage 1: subgrid size and launch mode
        for mode in modes:
            trial(L, mode, DEFAULT_CHUNK, DEFAULT_CHANNELS)
    if best is None:
        raise RuntimeError("autotune: no candidate configuration could be planned for this observation")
    for chunk in chunks:                    # stage 2: gridder records per chunk
        trial(best.subgrid_size, best.mode, chunk, DEFAULT_CHANNELS)
    for ch in channels:                     # stage 3: degridder channels per lane
        trial(best.subgrid_size, best.mode, best.grid_chunk, ch)
    best.timings = timings
    cache[key] = best.as_dict()
    _save_cache(cache_path, cache)
    return best
