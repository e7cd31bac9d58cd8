"""Autotuner for the batched launch.

Chooses, for one observation, the subgrid size L, the launch mode (one block
per work item, or a persistent grid draining the work queue), the gridder's
records per chunk (how many staged visibilities one bulk copy brings into
shared memory; Section 3.2 leaves the gridder's thread shape a per-device
tunable), the degridder's kind (tensor cores, or the FP32 pipe with 1, 2 or
4 channels per lane: phasors of later channels by rotation) and whether the
gridder also runs on the tensor cores, by timing a grid + degrid pass on the
observation's own plans with CUDA events.  The search is staged: every (L,
mode) with the library's defaults, then the chunk for the best (L, mode),
then the degridder's kind, then the gridder's unit.  The winner is cached in a JSON file keyed by the GPU and
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
DEGRID_CHANNELS = (1, 2, 4)     # channels per lane of the FP32 degridder
# multiply-accumulate units (idg.h): 1 both kernels on FP32, 2 both on the tensor cores, 3 the degridder
# on the tensor cores (the library's default)
MAC_FP32, MAC_TENSOR, MAC_TENSOR_DEGRID = 1, 2, 3
DEFAULT_CHUNK, DEFAULT_CHANNELS, DEFAULT_MAC = 48, 1, MAC_TENSOR_DEGRID


@dataclass
class Choice:
    subgrid_size: int
    mode: str
    grid_chunk: int
    degrid_channels: int
    ms: float
    timings: dict = field(default_factory=dict)
    mac_unit: int = DEFAULT_MAC

    def as_dict(self):
        return {"subgrid_size": self.subgrid_size, "mode": self.mode, "grid_chunk": self.grid_chunk,
                "degrid_channels": self.degrid_channels, "mac_unit": self.mac_unit, "ms": self.ms,
                "timings": self.timings}

    def plan_kwargs(self, idg) -> dict:
        """Keyword arguments of idg.Plan that apply this choice."""
        return {"subgrid_size": self.subgrid_size, "flags": idg.IDG_PERSISTENT if self.mode == "persistent" else 0,
                "grid_chunk": self.grid_chunk, "degrid_channels": self.degrid_channels, "mac_unit": self.mac_unit}


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


def gpu_measure(obs, subgrid_size, mode, grid_chunk=DEFAULT_CHUNK, degrid_channels=DEFAULT_CHANNELS,
                mac_unit=DEFAULT_MAC, trials=2, aterms=None, graph=False, vis=None):
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
                        grid_chunk=grid_chunk, degrid_channels=degrid_channels, mac_unit=mac_unit)
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
    """Return the fastest (L, mode, chunk, degridder kind, gridder unit) for `obs`,
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
                      c.get("degrid_channels", DEFAULT_CHANNELS), c["ms"], c.get("timings", {}),
                      c.get("mac_unit", MAC_FP32))
    timings = {}
    best = None

    mac_names = {MAC_FP32: "fp32", MAC_TENSOR: "tensor", MAC_TENSOR_DEGRID: "tensor-degrid"}

    def trial(L, mode, chunk, ch, mac):
        nonlocal best
        name = f"L{L}/{mode}/chunk{chunk}/ch{ch}/{mac_names[mac]}"
        if name in timings:
            return
        ms = measure(obs, L, mode, chunk, ch, mac)
        timings[name] = ms
        if ms is not None and (best is None or ms < best.ms):
            best = Choice(L, mode, chunk, ch, ms, mac_unit=mac)

    for L in candidates:                    # stage 1: subgrid size and launch mode
        for mode in modes:
            trial(L, mode, DEFAULT_CHUNK, DEFAULT_CHANNELS, DEFAULT_MAC)
    if best is None:
        raise RuntimeError("autotune: no candidate configuration could be planned for this observation")
    for chunk in chunks:                    # stage 2: gridder records per chunk
        trial(best.subgrid_size, best.mode, chunk, DEFAULT_CHANNELS, best.mac_unit)
    for ch in channels:                     # stage 3: the degridder on the FP32 pipe, 1, 2 or 4 channels per lane
        trial(best.subgrid_size, best.mode, best.grid_chunk, ch, MAC_FP32)
    if best.mac_unit != MAC_FP32:           # stage 4: the gridder on the tensor cores too
        trial(best.subgrid_size, best.mode, best.grid_chunk, 1, MAC_TENSOR)
    best.timings = timings
    cache[key] = best.as_dict()
    _save_cache(cache_path, cache)
    return best
