#!/usr/bin/env python3
"""Benchmark of the IDG hot path: gridded + degridded visibilities per second.

Workload (default): the MWA-like observation -- 128 stations (8128 baselines)
uniform in a 3 km disk, 56 timesteps x 2 s, 24 channels 140-170 MHz, 4-pol
complex64 visibilities from 200 point sources plus 1 Jy Gaussian noise,
4096^2 FP64 master grid, 96^2 subgrids, kernel padding 18, FOV 0.5 rad,
per-station A-terms every 8 s on 9 x 9 nodes (Gaussian beam x Kolmogorov
phase screen), synthetic and seeded.

One step = idg_grid of all visibilities into a zeroed master grid plus
idg_degrid of all visibilities from a model grid.  value = 2 * n_vis * steps
/ device time.  The inputs (350 MB visibilities, 1 GiB grids) are larger than
L2, so no flush is needed between steps.

The e2e leg measures the same steps through the C ABI with the inputs in
pinned host memory and the results read back every step; the copies run on
two copy streams with double buffers, overlapping the kernels of the
neighbouring steps, and within a step the model grid's copy overlaps the
gridding and the output grid's copy the degridding.

Further legs on the same device: Stokes-I mode, w layers (the same array
with station heights of 50 m rms), the A-term power normalisation (grid and
invert), the image-domain wrapper and the serving comparison.

--impl reference times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gridded+degridded visibilities/sec at 1 GB300 (FP32-batched vs plain) and % FP32/SFU roofline"
UNIT = "vis/s"
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM per clock
FLOP_PER_VISPX = 34.0            # 16 FMA (4-pol complex MAC) + 1 FMA (phase) = 17 FMA per visibility-pixel
SM_MAX_MHZ_FALLBACK = 2070.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "kernel_traffic.json")
CSRC = os.path.join(ROOT, "paper_2502_17789_gb300", "csrc")
# ncu recipes behind profiles/: the launch list of the bench's own workload (device time of every
# launch, one pass), and per kernel the DRAM bytes of its first two launches on the 90-station
# reduction of the same workload (a few GB on the device), which --record-traffic scales to a
# full-size launch by the algorithmic bytes of the two launches
BENCH_SHORT = ('python bench.py --steps 2 --warmup 1 --no-cpu-baseline --no-e2e --serving-requests 0 '
               '--image-steps 0 --stokes-steps 0 --wlayer-steps 0 --normalize-steps 0 --uneven-steps 0 '
               '--small-steps 0')
NCU_LAUNCH_LIST = ('ncu --metrics gpu__time_duration.sum --clock-control none --kernel-name-base demangled '
                   '-k regex:"idg::" -c 400 --csv --log-file launches.csv ' + BENCH_SHORT)
TRAFFIC_STATIONS = 90
MAC_NAMES = {1: "FP32 pipe (gridder and degridder)", 2: "tensor cores (gridder and degridder)",
             3: "FP32-pipe gridder, tensor-core degridder"}


def ncu_traffic_command(kern: str) -> str:
    mac = {"gridder": " --mac-unit 3", "gridder_tc": " --mac-unit 2", "degridder": " --mac-unit 1"}.get(kern, "")
    return (f'ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none '
            f'--kernel-name-base demangled -k regex:"idg::{kern}_kernel<" -c 2 --csv '
            f'--log-file traffic_{kern}.csv {BENCH_SHORT} --stations {TRAFFIC_STATIONS}{mac}')
KERNEL_SOURCES = {"gridder": ["gridder.cu", "gridder_kernels.cuh", "kernels_common.cuh", "idg_internal.h"],
                  "degridder": ["degridder.cu", "degridder_kernels.cuh", "kernels_common.cuh", "idg_internal.h"],
                  "degridder_tc": ["degridder.cu", "degridder_tc_kernels.cuh", "degridder_kernels.cuh",
                                   "kernels_common.cuh", "idg_internal.h"],
                  "gridder_tc": ["gridder.cu", "gridder_tc_kernels.cuh", "kernels_common.cuh", "idg_internal.h"]}


def kernel_of(kind: str, mac_unit: int) -> str:
    """The kernel (ncu name prefix, traffic key) a plan with `mac_unit` in use
    runs for the timing class `kind` (gridder or degridder)."""
    if kind == "gridder":
        return "gridder_tc" if mac_unit == 2 else "gridder"
    return "degridder" if mac_unit == 1 else "degridder_tc"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", type=int, default=2, help="workload index (1 small, 2 MWA-like)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-baseline sample budget")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (small profiling runs)")
    ap.add_argument("--stations", type=int, default=None, help="reduce the workload's stations (profiling)")
    ap.add_argument("--timesteps", type=int, default=None, help="reduce the workload's timesteps (profiling)")
    ap.add_argument("--record-traffic", metavar="DIR", default=None,
                    help="read traffic_gridder.csv and traffic_degridder.csv (the ncu_traffic_command captures) "
                         "from DIR and store each kernel's DRAM bytes per launch, scaled to a launch of the "
                         "default workload and keyed by the digest of its sources, in profiles/kernel_traffic.json")
    ap.add_argument("--image-steps", type=int, default=2,
                    help="timed invert + predict calls of the image-domain wrapper; 0 = skip")
    ap.add_argument("--stokes-steps", type=int, default=5,
                    help="timed grid + degrid steps of the same workload in Stokes-I mode (one grid plane); 0 = skip")
    ap.add_argument("--wlayer-steps", type=int, default=3,
                    help="timed grid + degrid steps with w layers (IDG_W_LAYERS) on the same array with station "
                         "heights of 50 m rms; 0 = skip")
    ap.add_argument("--normalize-steps", type=int, default=3,
                    help="timed grid and invert calls with the A-term power normalisation "
                         "(IDG_NORMALIZE_ATERM) on the same workload; 0 = skip")
    ap.add_argument("--uneven-steps", type=int, default=2,
                    help="timed CUDA-graph replays of grid + degrid of the 256-station uneven workload "
                         "(352.5 M visibilities, 8192^2 grid, L = 64); 0 = skip")
    ap.add_argument("--small-steps", type=int, default=50,
                    help="timed CUDA-graph replays of grid + degrid of the small 32-station workload; 0 = skip")
    ap.add_argument("--serving-requests", type=int, default=24,
                    help="requests of the serving comparison (batched vs plain at 2x plain capacity); 0 = skip")
    ap.add_argument("--mac-unit", type=int, default=0, choices=[0, 1, 2, 3],
                    help="the multiply-accumulate unit of the main, uneven and small legs (idg_geometry.mac_unit: 0 the library's default, "
                         "1 FP32 pipe, 2 tensor cores for both kernels, 3 tensor-core degridder only)")
    ap.add_argument("--aterms", choices=["beam", "full"], default="beam",
                    help="beam: the scalar beam x screen gain (diagonal Jones); full: the same plus 5%% "
                         "polarisation leakage, so every Jones matrix is full")
    return ap.parse_args()


# --------------------------------------------------------------------------- workload

def make_workload(idx: int, device, stations=None, timesteps=None, aterm_kind="beam"):
    import torch
    from paper_2502_17789_gb300 import synth

    obs = synth.config(idx, seed=0, n_stations=stations, n_timesteps=timesteps)
    rng = np.random.default_rng(0)
    model = synth.beam_screen_model(rng, rms_rad=2.0)
    aterms = synth.aterms_beam_screen(obs, model) if idx != 1 else \
        synth.aterms_identity(obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    n_src, half = (20, 0.0873) if idx == 1 else (200, 0.16)
    sky = synth.point_sources(rng, n_src, half)
    vis = synth.simulate_visibilities(obs, sky, model if idx != 1 else None, noise_sigma=1.0, rng=rng,
                                      device=str(device))
    if aterm_kind == "full":
        aterms = synth.aterms_with_leakage(np.random.default_rng(1), aterms, 0.05)
    desc = workload_description(idx, obs, stations, timesteps, aterm_kind)
    return obs, torch.as_tensor(aterms, device=device), vis, desc


def workload_description(idx, obs, stations=None, timesteps=None, aterm_kind="beam") -> str:
    desc = {1: "32 stations in a 1 km disk (496 baselines), 16 x 8 s, 8 ch 150-157 MHz, 512^2 grid, L=32, P=12, "
               "FOV 0.35, identity A-terms, 20 sources + noise",
            2: "128 stations in a 3 km disk (8128 baselines), 56 x 2 s, 24 ch 140-170 MHz, 4096^2 FP64 grid, "
               "L=96, P=18, FOV 0.5, A-terms per 8 s on 9x9 nodes (Gaussian beam x Kolmogorov screen, 2 rad rms), "
               "200 sources + 1 Jy noise"}.get(idx, obs.name)
    if aterm_kind == "full":
        desc += ", full-Jones A-terms (5% leakage)"
    if stations or timesteps:
        desc = f"REDUCED ({obs.n_stations} stations, {obs.n_timesteps} timesteps) " + desc
    return desc


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == len(self.FIELDS):
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        pw = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        for r in rows:
            for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], r[4:]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- CPU baseline (oracle)

def _oracle_sample(obs, aterms_np, vis_np, grid_np, budget_s: float, seed: int = 0):
    """Time the FP64 oracle on a seeded random sample of subgrids whose size
    is calibrated to `budget_s` seconds of grid + degrid work."""
    import oracle

    geom = oracle.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                           aterm_nodes=obs.aterm_nodes)
    full = oracle.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    rng = np.random.default_rng(seed)
    order = rng.permutation(full.subgrids.shape[0])
    A = aterms_np.astype(np.complex128)

    def subplan(idx):
        idx = np.sort(idx)
        sg = full.subgrids[idx]
        remap = {int(o): n for n, o in enumerate(idx)}
        segs = np.array([[remap[int(s[0])], s[1], s[2], s[3]] for s in full.segments if int(s[0]) in remap], np.int32)
        return oracle.Plan(sg, segs), int(sum((r[2] - r[1]) * (r[4] - r[3]) for r in sg))

    args = lambda pl: (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)
    vis128 = vis_np.astype(np.complex128)

    def run(pl):
        t0 = time.perf_counter()
        oracle.grid(*args(pl), vis128, A)
        oracle.degrid(*args(pl), grid_np, A)
        return time.perf_counter() - t0

    n = min(os.cpu_count() or 4, len(order))
    pl, nv = subplan(order[:n])
    t = run(pl)
    per_vis = t / max(nv, 1)
    target_vis = budget_s / max(per_vis, 1e-12)
    cum = np.cumsum([(full.subgrids[o][2] - full.subgrids[o][1]) * (full.subgrids[o][4] - full.subgrids[o][3])
                     for o in order])
    n = int(min(len(order), max(1, np.searchsorted(cum, target_vis) + 1)))
    pl, nv = subplan(order[:n])
    return pl, nv, n, run


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(obs, aterms_np, vis_np, grid_np, budget_s):
    pl, nv, n, run = _oracle_sample(obs, aterms_np, vis_np, grid_np, budget_s)
    t = run(pl)
    cores = os.cpu_count()
    return {"value": 2.0 * nv / t, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{n} seeded-random subgrids ({nv} visibilities) of the workload, grid + degrid, "
                      f"FP64 C oracle with OpenMP over subgrids, {t:.1f} s",
            "seconds": t}


# --------------------------------------------------------------------------- native arm

# --------------------------------------------------------------------------- DRAM traffic

def source_digest(kern: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kern]:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kern: str, workload: str):
    """Per-launch DRAM bytes (read + write) of `kern` from the last ncu
    capture, or None if the kernel's sources changed since or the capture
    was of another workload."""
    try:
        with open(TRAFFIC_FILE) as f:
            entry = json.load(f).get(kern)
    except (OSError, ValueError):
        return None
    if not entry or entry.get("source_sha256") != source_digest(kern) or entry.get("workload") != workload:
        return None
    return entry.get("dram_bytes_per_launch")


def algorithmic_bytes_per_launch(kern: str, obs, L: int) -> float:
    """DRAM bytes a launch must move, averaged over the plan's batches:
    gridder 128 B staged record read per visibility + 32 B subgrid image
    written per pixel; degridder 32 B image read per pixel + 32 B per
    visibility written (host-only plan, no device work)."""
    from paper_2502_17789_gb300 import idg

    g, keep = idg.make_geometry(obs.grid_size, L, obs.kernel_padding, obs.image_size, aterm_nodes=obs.aterm_nodes,
                                flags=idg.IDG_HOST_ONLY)
    h = idg.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets)
    try:
        st = idg.idg_plan_stats(h)
    finally:
        idg.idg_plan_destroy(h)
    n_sg = st.n_subgrids - st.n_subgrids_dropped
    n_vis = st.n_vis - st.n_vis_dropped
    # the same batching rule as the library (1 GiB of subgrid images per batch)
    per_sg = 4 * L * L * 8
    n_batches = max(1, -(-n_sg // max(1, (1 << 30) // per_sg)))
    pix = n_sg * L * L * 32.0
    total = (128.0 * n_vis + pix) if kern.startswith("gridder") else (pix + 32.0 * n_vis)
    return total / n_batches


def record_traffic(folder: str, full_obs, workload: str):
    """Per-launch DRAM bytes (read + write) of the gridder and degridder from
    their captures on the 90-station case, scaled to a full-size launch by
    the ratio of algorithmic bytes per launch."""
    import csv
    import collections
    from paper_2502_17789_gb300 import synth

    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    small = synth.config(2, seed=0, n_stations=TRAFFIC_STATIONS)
    out = {}
    for kern in KERNEL_SOURCES:
        if not os.path.exists(os.path.join(folder, f"traffic_{kern}.csv")):
            continue
        with open(os.path.join(folder, f"traffic_{kern}.csv")) as f:
            rows = [r for r in csv.reader(f)]
        hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "Metric Name" in r)
        h = rows[hi]
        ki, mi, vi, ui, ii = (h.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit", "ID"))
        per = collections.defaultdict(float)
        for r in rows[hi + 1:]:
            if len(r) > vi and r[mi] in ("dram__bytes_read.sum", "dram__bytes_write.sum") and \
                    f"{kern}_kernel" in r[ki] and not (kern.startswith("gridder") and "degridder" in r[ki]):
                per[r[ii]] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1.0)
        if not per:
            continue
        measured = sum(per.values()) / len(per)
        alg_small = algorithmic_bytes_per_launch(kern, small, small.subgrid_size)
        alg_full = algorithmic_bytes_per_launch(kern, full_obs, full_obs.subgrid_size)
        out[kern] = {"dram_bytes_per_launch": measured * alg_full / alg_small,
                     "captured_bytes_per_launch": measured, "captured_launches": len(per),
                     "captured_over_algorithmic": measured / alg_small,
                     "algorithmic_bytes_per_launch": alg_full,
                     "source_sha256": source_digest(kern), "workload": workload,
                     "command": ncu_traffic_command(kern) + f"; python bench.py --record-traffic <dir>",
                     "note": f"captured on the {TRAFFIC_STATIONS}-station case, scaled to a full-size launch "
                             "by algorithmic bytes per launch"}
    with open(TRAFFIC_FILE, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1))


def _graph_legs(plan, vis, A, G, out, steps, side):
    """Mean ms of grid and degrid CUDA-graph replays, after one warm-up replay."""
    import torch
    plan.grid_graph(vis, A, G)
    plan.degrid_graph(G, A, out)
    plan.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    g_ms = d_ms = 0.0
    for _ in range(steps):
        e[0].record(side)
        plan.grid_graph(vis, A, G)
        e[1].record(side)
        plan.degrid_graph(G, A, out)
        e[2].record(side)
        plan.synchronize()
        g_ms += e[0].elapsed_time(e[1])
        d_ms += e[1].elapsed_time(e[2])
    return g_ms / steps, d_ms / steps


def _kernel_fracs(plan, vis, A, G, out, n_sm, sm_max, r_vp_meas):
    """Per-kernel device time of one profiled (non-graph) grid + degrid, and
    the gridder's and degridder's fractions of the nominal and measured R_vp."""
    plan.profile(True)
    plan.profile_read()
    plan.grid(vis, A, G)
    plan.degrid(G, A, out)
    prof = plan.profile_read()
    plan.profile(False)
    vispx = float(plan.stats().vis_pixels)
    r_vp_nom = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / (FLOP_PER_VISPX / 2.0)
    kern = {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items()}
    for k in ("gridder", "degridder"):
        if prof[k][0] > 0:
            r = vispx / (prof[k][0] * 1e-3)
            kern[k].update(vispx_per_s=r, frac_nominal=round(r / r_vp_nom, 4), frac_measured=round(r / r_vp_meas, 4))
    return kern


def uneven_leg(idg, synth, dev, steps, n_sm, sm_max, r_vp_meas, mac_unit=0):
    import torch
    t0 = time.time()
    obs = synth.config(4, seed=0)
    model = synth.beam_screen_model(np.random.default_rng(0), rms_rad=2.0)
    A = torch.as_tensor(synth.aterms_beam_screen(obs, model), device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    vis = torch.randn((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64, device=dev,
                      generator=g)
    side = torch.cuda.Stream(dev)
    L = 64
    plan = idg.Plan(obs, subgrid_size=L, stream=side.cuda_stream, grid_chunk=64, mac_unit=mac_unit)
    t_plan = time.time() - t0
    st = plan.stats()
    N = obs.grid_size
    G = torch.zeros((4, N, N), dtype=torch.complex128, device=dev)
    out = torch.empty_like(vis)
    torch.cuda.synchronize(dev)
    g_ms, d_ms = _graph_legs(plan, vis, A, G, out, steps, side)
    kern = _kernel_fracs(plan, vis, A, G, out, n_sm, sm_max, r_vp_meas)
    sg = plan.subgrids()
    nv = (sg[:, 2] - sg[:, 1]) * (sg[:, 4] - sg[:, 3])
    res = {"value": 2.0 * obs.n_vis / ((g_ms + d_ms) * 1e-3), "unit": UNIT, "steps": steps,
           "workload": "256 stations, log-normal radii (median 300 m, <= 3 km), 32640 baselines, 360 x 0.5 s, "
                       "30 ch 140-170 MHz, 8192^2 FP64 grid, L = 64, P = 18, FOV 0.5, A-terms every 4 s "
                       "(beam x screen), random visibilities",
           "n_vis": int(obs.n_vis),
           "launch": "one block per work item, CUDA-graph replay, " + MAC_NAMES.get(int(st.mac_unit), "?") +
                     (" (the autotuner's choice on GB300)" if int(st.mac_unit) == 2 else "") +
                     ("; FP32 gridder chunks of 64 records" if int(st.mac_unit) != 2 else ""),
           "graph_replay_ms": {"grid": g_ms, "degrid": d_ms}, "subgrids": int(st.n_subgrids),
           "vis_per_subgrid_min_median_max": [int(nv.min()), int(np.median(nv)), int(nv.max())],
           "vis_pixels_per_direction": float(st.vis_pixels), "kernels": kern, "plan_seconds": t_plan}
    plan.close()
    del G, out, vis
    torch.cuda.empty_cache()
    return res


def small_leg(idg, dev, steps, n_sm, sm_max, r_vp_meas, mac_unit=0):
    import torch
    obs, A, vis, _ = make_workload(1, dev)
    side = torch.cuda.Stream(dev)
    plan = idg.Plan(obs, stream=side.cuda_stream, mac_unit=mac_unit)
    N = obs.grid_size
    G = torch.zeros((4, N, N), dtype=torch.complex128, device=dev)
    out = torch.empty_like(vis)
    torch.cuda.synchronize(dev)
    g_ms, d_ms = _graph_legs(plan, vis, A, G, out, steps, side)
    kern = _kernel_fracs(plan, vis, A, G, out, n_sm, sm_max, r_vp_meas)
    res = {"value": 2.0 * obs.n_vis / ((g_ms + d_ms) * 1e-3), "unit": UNIT, "steps": steps,
           "workload": workload_description(1, obs), "n_vis": int(obs.n_vis),
           "launch": "one block per work item, CUDA-graph replay", "graph_replay_ms": {"grid": g_ms, "degrid": d_ms},
           "kernels": kern}
    plan.close()
    return res


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_2502_17789_gb300 import build as libbuild
    from paper_2502_17789_gb300 import idg, parallel, synth

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    libbuild.build()
    obs, A_d, vis_full, desc = make_workload(args.workload, dev, args.stations, args.timesteps, args.aterms)
    stream = torch.cuda.current_stream(dev)
    # N GPUs share one observation (Section 3.5: workers own subsets of the data): rank r grids the
    # baselines r, r + N, ... into its own FP64 master-grid replica, one all-reduce sums the replicas,
    # and every rank degrids its own baselines from the (replicated) model grid
    obs_r, shard = parallel.shard_observation(obs, rank, world)
    vis_d = vis_full if world == 1 else vis_full[torch.as_tensor(shard, device=dev)].contiguous()
    del vis_full
    plan = idg.Plan(obs_r, stream=stream.cuda_stream, mac_unit=args.mac_unit)
    st = plan.stats()
    N = obs.grid_size
    G_model = torch.zeros((4, N, N), dtype=torch.complex128, device=dev)
    plan.grid(vis_d, A_d, G_model)                     # the model grid the degrid leg predicts from
    if world > 1:
        parallel.reduce_grids(G_model)
    G_out = torch.empty_like(G_model)
    vis_pred = torch.empty_like(vis_d)

    def step():
        parallel.sharded_step(lambda g: plan.grid(vis_d, A_d, g), lambda: plan.degrid(G_model, A_d, vis_pred),
                              G_out, world)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    plan.profile(True)
    plan.profile_read()
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    prof = plan.profile_read()
    plan.profile(False)
    if world > 1:
        ms = parallel.max_over_ranks(ms, device=dev)
    total_vis = 2.0 * obs.n_vis * args.steps   # the whole observation, over all ranks
    value = total_vis / (ms * 1e-3)

    # roofline of the dominant kernel (gridder or degridder), live from the timed region
    kern = max(("gridder", "degridder"), key=lambda k: prof[k][0])
    k_ms, k_launches = prof[kern]
    vispx = float(st.vis_pixels) * args.steps
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    sm_max = float(peaks.get("sm_max_mhz", SM_MAX_MHZ_FALLBACK))
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved_vispx = vispx / (k_ms * 1e-3)
    achieved = achieved_vispx * FLOP_PER_VISPX / 1e12
    kern_name = kernel_of(kern, int(st.mac_unit))
    traffic = recorded_traffic(kern_name, desc)
    roofline = {"bound": "alu", "kernel": kern_name, "achieved": round(achieved, 3), "peak": round(peak_tflops, 3),
                "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4), "traffic": traffic,
                "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 flop x {sm_max:.0f} MHz (max SM clock)",
                "achieved_vispx_per_s": achieved_vispx, "flop_per_vispx": FLOP_PER_VISPX,
                "launches": k_launches, "avg_launch_ms": k_ms / max(k_launches, 1)}
    if clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = round(achieved / (peak_tflops * clocks["sm_mhz"] / sm_max), 4)
    # the same fractions against the rates the library's probe kernels measure on this device (FP32
    # FMA and __sincosf throughput): R_vp = min(F_fma / 17, F_sincos), one sincos per visibility-pixel
    f_fma, f_sin = idg.idg_peak_rates(stream.cuda_stream)
    clk = float(clocks.get("sm_mhz") or sm_max) * 1e6
    r_vp_meas = min(f_fma / (FLOP_PER_VISPX / 2.0), f_sin)
    r_vp_nom = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / (FLOP_PER_VISPX / 2.0)
    roofline["peak_measured"] = {
        "fma_per_s": f_fma, "sincos_per_s": f_sin, "vispx_per_s": r_vp_meas,
        "fma_lanes_per_clk_per_sm": f_fma / (n_sm * clk), "sincos_per_clk_per_sm": f_sin / (n_sm * clk),
        "clock_mhz": clk / 1e6,
        "basis": "idg_peak_rates: independent f32x2 FMA chains and __sincosf chains on every SM, CUDA events; "
                 "R_vp = min(F_fma / 17, F_sincos)"}
    roofline["frac_measured"] = round(achieved_vispx / r_vp_meas, 4)
    roofline["kernel_fractions"] = {
        k: {"vispx_per_s": vispx / (prof[k][0] * 1e-3), "frac_nominal": round(vispx / (prof[k][0] * 1e-3) / r_vp_nom, 4),
            "frac_measured": round(vispx / (prof[k][0] * 1e-3) / r_vp_meas, 4)} for k in ("gridder", "degridder")}
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps} for k, v in prof.items()}
    # the paper's kernel rates (Section 5.3: gridder 480 and degridder 400 M visibilities/s on an A100 at
    # 32 x 32 subgrids), beside this run's; a visibility costs L^2 pixel updates, so the per
    # visibility x pixel rates are the ones that compare across subgrid sizes
    paper_context = {"hardware": "NVIDIA A100 SXM 40 GB", "subgrid_size": 32,
                     "gridder_vis_per_s": 480e6, "degridder_vis_per_s": 400e6,
                     "gridder_vispx_per_s": 480e6 * 32 * 32, "degridder_vispx_per_s": 400e6 * 32 * 32,
                     "this_gridder_vispx_per_s": vispx / (prof["gridder"][0] * 1e-3),
                     "this_degridder_vispx_per_s": vispx / (prof["degridder"][0] * 1e-3),
                     "note": "context, not a target: the paper's dataset and visibility count differ"}
    gpu_launches = int(sum(v[1] for v in prof.values()))

    # image-domain wrapper (Eq. 11 / Eq. 12): invert = grid + master-grid transform + taper correction,
    # predict = the reverse; one timed call each after an untimed one that makes the cuFFT plan
    image_domain = None
    if world > 1:   # the legs below are single-GPU diagnostics of the same build
        args.image_steps = args.stokes_steps = args.wlayer_steps = args.normalize_steps = 0
        args.uneven_steps = args.small_steps = 0
    if args.image_steps > 0:
        img = torch.empty_like(G_out)
        plan.invert(vis_d, A_d, G_out, img)
        plan.predict(img, A_d, G_out, vis_pred)
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        inv_ms = pred_ms = 0.0
        for _ in range(args.image_steps):
            ev[0].record(stream)
            plan.invert(vis_d, A_d, G_out, img)
            ev[1].record(stream)
            plan.predict(img, A_d, G_out, vis_pred)
            ev[2].record(stream)
            torch.cuda.synchronize(dev)
            inv_ms += ev[0].elapsed_time(ev[1])
            pred_ms += ev[1].elapsed_time(ev[2])
        image_domain = {"invert_ms": inv_ms / args.image_steps, "predict_ms": pred_ms / args.image_steps,
                        "image": f"complex128 [4][{N}][{N}]", "transform": "cuFFT Z2Z, 4 planes"}
        del img

    # the same workload imaged in Stokes I (IDG_STOKES_I): one grid plane, a quarter of the subgrid
    # transforms, adder and splitter work; the phasor sums still carry the 4 correlations
    stokes_i = None
    if args.stokes_steps > 0:
        plan_i = idg.Plan(obs, flags=idg.IDG_STOKES_I, stream=stream.cuda_stream)
        Gi_model = torch.zeros(plan_i.grid_shape(), dtype=torch.complex128, device=dev)
        plan_i.grid(vis_d, A_d, Gi_model)
        Gi_out = torch.empty_like(Gi_model)

        def step_i():
            Gi_out.zero_()
            plan_i.grid(vis_d, A_d, Gi_out)
            plan_i.degrid(Gi_model, A_d, vis_pred)

        for _ in range(2):
            step_i()
        torch.cuda.synchronize(dev)
        plan_i.profile(True)
        plan_i.profile_read()
        e0.record(stream)
        for _ in range(args.stokes_steps):
            step_i()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        si_ms = e0.elapsed_time(e1)
        prof_i = plan_i.profile_read()
        plan_i.close()
        stokes_i = {"value": 2.0 * obs.n_vis * args.stokes_steps / (si_ms * 1e-3), "unit": UNIT,
                    "ms_per_step": si_ms / args.stokes_steps, "steps": args.stokes_steps,
                    "grid": f"complex128 [1][{N}][{N}]",
                    "kernels": {k: {"ms_per_step": v[0] / args.stokes_steps} for k, v in prof_i.items()}}
        del Gi_model, Gi_out

    def timed(fn, n):
        fn()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n

    # w layers (IDG_W_LAYERS, Section 2.4 with w-stacking): the same 128-station disk with station
    # heights of 50 m rms, so |w| spans several layers of 2 w_max; the visibilities and A-terms of the
    # main workload have the same shapes and are reused (their values do not change the work)
    w_layers = None
    if args.wlayer_steps > 0 and args.workload == 2 and args.stations is None and args.timesteps is None:
        rng_w = np.random.default_rng(1)
        enu = synth.stations_uniform_disk(rng_w, obs.n_stations, 3000.0)
        enu[:, 2] = rng_w.normal(0.0, 50.0, enu.shape[0])
        obs_w = synth.make_observation(enu, obs.n_timesteps, 2.0, obs.freqs, 4, obs.grid_size, obs.subgrid_size,
                                       obs.kernel_padding, obs.image_size, name="mwa-like-128-stations-50m-heights")
        plan_w = idg.Plan(obs_w, flags=idg.IDG_W_LAYERS, stream=stream.cuda_stream)
        st_w = plan_w.stats()
        Gw_model = torch.zeros(plan_w.grid_shape(), dtype=torch.complex128, device=dev)
        plan_w.grid(vis_d, A_d, Gw_model)
        Gw_out = torch.empty_like(Gw_model)

        def step_w():
            Gw_out.zero_()
            plan_w.grid(vis_d, A_d, Gw_out)
            plan_w.degrid(Gw_model, A_d, vis_pred)

        plan_w.profile(True)
        plan_w.profile_read()
        w_ms = timed(step_w, args.wlayer_steps)
        prof_w = plan_w.profile_read()
        # the layer count of the signed set {k * 2 w_max, k integer} without the conjugate mirror, for
        # the same visibilities: the set the paper's {w_max, 3 w_max, ...} with w >= 0 roughly halves
        w_lam = obs_w.uvw[:, :, 2][:, :, None] * (obs_w.freqs / synth.SPEED_OF_LIGHT)[None, None, :]
        signed_layers = int(np.unique(np.floor(w_lam / float(st_w.w_layer_step) + 0.5)).size)
        del w_lam
        w_layers = {"value": 2.0 * obs_w.n_vis / (w_ms * 1e-3), "unit": UNIT, "ms_per_step": w_ms,
                    "steps": args.wlayer_steps, "n_w_layers": int(st_w.n_w_layers),
                    "n_w_layers_signed_unmirrored": signed_layers,
                    "w_layer_step_wavelengths": float(st_w.w_layer_step), "subgrids": int(st_w.n_subgrids),
                    "grid": f"complex128 [{int(st_w.n_w_layers)}][4][{N}][{N}]",
                    "array": "the 128-station 3 km disk with station heights of 50 m rms",
                    "kernels": {k: {"ms_per_step": v[0] / (args.wlayer_steps + 1)} for k, v in prof_w.items()}}
        plan_w.close()
        del Gw_model, Gw_out

    # A-term power normalisation (IDG_NORMALIZE_ATERM, Section 3.3): gridding with the per-pixel
    # 1/||A_p^H A_q||_F and the weight map, and the normalised invert (grid, transform, taper and
    # weight correction), against the plain gridder and invert of the same workload above
    normalized = None
    if args.normalize_steps > 0:
        plan_n = idg.Plan(obs, flags=idg.IDG_NORMALIZE_ATERM, stream=stream.cuda_stream)
        Gn = torch.empty_like(G_out)

        def grid_n():
            Gn.zero_()
            plan_n.grid(vis_d, A_d, Gn)

        plan_n.profile(True)
        plan_n.profile_read()
        n_grid_ms = timed(grid_n, args.normalize_steps)
        prof_n = plan_n.profile_read()
        img_n = torch.empty_like(G_out)
        n_inv_ms = timed(lambda: plan_n.invert(vis_d, A_d, Gn, img_n), args.normalize_steps)
        normalized = {"grid_ms": n_grid_ms, "gridder_ms": prof_n["gridder"][0] / (args.normalize_steps + 1),
                      "plain_gridder_ms": kernels["gridder"]["ms_per_step"], "invert_ms": n_inv_ms,
                      "plain_invert_ms": image_domain["invert_ms"] if image_domain else None,
                      "steps": args.normalize_steps}
        plan_n.close()
        del Gn, img_n

    # end to end through the C ABI with host buffers: every step copies its inputs (visibilities and model
    # grid) from pinned host memory and reads its results (grid and predicted visibilities) back.  The
    # copies run on two copy streams with double-buffered device buffers, so step k+1's inputs and step
    # k-1's results move while step k's kernels run; every copy of every step is inside the timed region.
    e2e = None
    if args.no_e2e:
        args.e2e_steps = 0
    need_host = args.e2e_steps > 0 or (rank == 0 and world == 1 and not args.no_cpu_baseline)
    vis_h = vis_d.cpu().pin_memory() if need_host else None
    gmodel_h = G_model.cpu().pin_memory() if need_host else None
    if args.e2e_steps > 0:
        h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        vis_in = [torch.empty_like(vis_d) for _ in range(2)]
        gmodel_in = [torch.empty_like(G_model) for _ in range(2)]
        gout_d = [torch.empty_like(G_model) for _ in range(2)]
        vpred_d = [torch.empty_like(vis_d) for _ in range(2)]
        gout_h = [torch.empty(G_model.shape, dtype=G_model.dtype, pin_memory=True) for _ in range(2)]
        vpred_h = [torch.empty(vis_d.shape, dtype=vis_d.dtype, pin_memory=True) for _ in range(2)]
        ev = {k: [torch.cuda.Event() for _ in range(2)]
              for k in ("vis_ready", "gm_ready", "grid_done", "done", "grid_copied", "out_copied")}

        # per step: the gridder needs only the visibilities and the degridder only the model grid, so the
        # model grid's copy overlaps the gridding and the output grid's copy overlaps the degridding
        def e2e_steps(n, first=None):
            for k in range(n):
                b = k % 2
                with torch.cuda.stream(h2d):
                    if k == 0 and first is not None:
                        first.record(h2d)
                    if k >= 2:
                        h2d.wait_event(ev["grid_done"][b])   # step k-2 no longer reads vis_in[b]
                    vis_in[b].copy_(vis_h, non_blocking=True)
                    ev["vis_ready"][b].record(h2d)
                    if k >= 2:
                        h2d.wait_event(ev["done"][b])        # ... nor gmodel_in[b]
                    gmodel_in[b].copy_(gmodel_h, non_blocking=True)
                    ev["gm_ready"][b].record(h2d)
                stream.wait_event(ev["vis_ready"][b])
                if k >= 2:
                    stream.wait_event(ev["grid_copied"][b])  # step k-2's grid has left gout_d[b]
                gout_d[b].zero_()
                plan.grid(vis_in[b], A_d, gout_d[b])
                if world > 1:
                    parallel.reduce_grids(gout_d[b])
                ev["grid_done"][b].record(stream)
                stream.wait_event(ev["gm_ready"][b])
                if k >= 2:
                    stream.wait_event(ev["out_copied"][b])   # step k-2's visibilities have left vpred_d[b]
                plan.degrid(gmodel_in[b], A_d, vpred_d[b])
                ev["done"][b].record(stream)
                with torch.cuda.stream(d2h):
                    d2h.wait_event(ev["grid_done"][b])
                    gout_h[b].copy_(gout_d[b], non_blocking=True)
                    ev["grid_copied"][b].record(d2h)
                    d2h.wait_event(ev["done"][b])
                    vpred_h[b].copy_(vpred_d[b], non_blocking=True)
                    ev["out_copied"][b].record(d2h)
            return ev["out_copied"][(n - 1) % 2]

        e2e_steps(2)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        last = e2e_steps(args.e2e_steps, first=t0)
        d2h.wait_event(last)
        t1.record(d2h)
        torch.cuda.synchronize(dev)
        e2e_ms = t0.elapsed_time(t1)
        if world > 1:
            e2e_ms = parallel.max_over_ranks(e2e_ms, device=dev)
        e2e = {"value": 2.0 * obs.n_vis * args.e2e_steps / (e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(vis_h.numel() * 8 + gmodel_h.numel() * 16),
               "d2h_bytes_per_step": int(gout_h[0].numel() * 16 + vpred_h[0].numel() * 8),
               "ms_per_step": e2e_ms / args.e2e_steps,
               "copies": "pinned host buffers; H2D and D2H on two copy streams, double-buffered; the model "
                         "grid's H2D overlaps the gridding, the output grid's D2H the degridding, and the "
                         "neighbouring steps' copies the kernels"}
        del vis_in, gmodel_in, gout_d, vpred_d, gout_h, vpred_h

    # the 256-station uneven workload (352.5 M visibilities, subgrids of 360 to 10800 visibilities,
    # 8192^2 grid) at L = 64 with one block per work item and gridder chunks of 64 records, the
    # autotuner's choice on GB300, as CUDA-graph replays; random visibilities (the work does not depend
    # on their values)
    uneven = None
    if args.uneven_steps > 0 and args.stations is None and args.timesteps is None:
        uneven = uneven_leg(idg, synth, dev, args.uneven_steps, n_sm, sm_max, r_vp_meas, args.mac_unit)
    small = None
    if args.small_steps > 0:
        small = small_leg(idg, dev, args.small_steps, n_sm, sm_max, r_vp_meas, args.mac_unit)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the oracle baseline runs at N = 1 only
        cpu = cpu_baseline(obs, A_d.cpu().numpy(), vis_h.numpy(), gmodel_h.numpy(), args.cpu_seconds)

    # the serving form (continuous batching) beside the plain one-request-at-a-time form, on a Poisson stream
    # of snapshot requests at twice the plain capacity (rank 0 of a single-GPU run only)
    serving = None
    if rank == 0 and world == 1 and args.serving_requests > 0:
        from paper_2502_17789_gb300 import serve
        plan.close()
        del G_out, vis_pred
        torch.cuda.empty_cache()
        cmp = serve.compare(args.serving_requests, seed=0, loads=(2.0, "burst"),
                            modes=("plain", "streams", "batched"))

        def brief(r):
            return {"vis_per_s": r["throughput_vis_per_s"], "p50_ms": 1e3 * r["p50_latency_s"],
                    "p99_ms": 1e3 * r["p99_latency_s"], "requests_ok": r["ok"], "makespan_s": r["makespan_s"],
                    "host_plan_s": r["host_plan_s"], "gpu_s": r["gpu_s"]}
        serving = {"requests": args.serving_requests,
                   "plain_capacity_requests_per_s": cmp["calibration_plain_requests_per_s"],
                   "modes": {"plain": "one request at a time", "streams": "each request on its own stream",
                             "batched": "continuous batching: waves of admitted requests share one launch per "
                                        "kind of work (idg_grid_many / idg_degrid_many)"}}
        for key, name in (("load_2", "poisson_2x_plain_capacity"), ("burst", "burst_all_at_once")):
            serving[name] = {m: brief(cmp[key][m]) for m in ("plain", "streams", "batched")}
        plan = None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded point-source sky through beam x phase-screen A-terms, noise)",
        "config": {"workload": desc, "n_vis": obs.n_vis, "form": "plain (one observation per call)",
                   "l2": "inputs larger than L2 (350 MB visibilities, 1 GiB grids); no flush",
                   "parallelism": (f"baseline shards x{world} (round-robin), one NCCL all-reduce of the FP64 grid "
                                   f"per step" if world > 1 else "single GPU"),
                   "subgrids": st.n_subgrids, "segments": st.n_segments, "batches": st.n_batches,
                   "vis_pixels_per_direction": st.vis_pixels,
                   "mac_unit": MAC_NAMES.get(int(st.mac_unit), str(st.mac_unit))},
        "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e, "gpu_launches": gpu_launches,
        "kernels": kernels, "image_domain": image_domain, "paper_context": paper_context, "stokes_i": stokes_i, "w_layers": w_layers,
        "normalized": normalized, "serving": serving, "uneven": uneven, "small": small,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if plan is not None:
        plan.close()
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    from paper_2502_17789_gb300 import synth
    import oracle

    oracle.build()
    obs = synth.config(args.workload, seed=0)
    rng = np.random.default_rng(0)
    model = synth.beam_screen_model(rng, rms_rad=2.0)
    aterms = synth.aterms_beam_screen(obs, model) if args.workload != 1 else \
        synth.aterms_identity(obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    vis = synth.random_visibilities(rng, obs)
    N = obs.grid_size
    grid = np.zeros((4, N, N), np.complex128)
    grid[:, N // 2 - 64:N // 2 + 64, N // 2 - 64:N // 2 + 64] = 1.0
    budget = max(2.0, 150.0 / max(args.steps + args.warmup, 1))
    pl, nv, n, run = _oracle_sample(obs, aterms, vis, grid, budget)
    for _ in range(args.warmup):
        run(pl)
    t = [run(pl) for _ in range(args.steps)]
    total = sum(t)
    value = 2.0 * nv * args.steps / total
    sample = f"{n} seeded-random subgrids ({nv} visibilities) of the workload per step, grid + degrid"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_description(args.workload, obs), "n_vis": obs.n_vis},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.record_traffic:
        from paper_2502_17789_gb300 import synth
        obs = synth.config(args.workload, seed=0, n_stations=args.stations, n_timesteps=args.timesteps)
        desc = workload_description(args.workload, obs, args.stations, args.timesteps, args.aterms)
        record_traffic(args.record_traffic, obs, desc)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
