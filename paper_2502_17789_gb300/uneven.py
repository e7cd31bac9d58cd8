"""Uneven batched persistent launch on the 256-station workload.

256 stations with log-normal radii (baselines up to 6 km), 360 x 0.5 s,
30 channels 140-170 MHz, A-terms every 4 s (45 intervals) on 9 x 9 nodes,
8192^2 FP64 grid: subgrids hold 360 to 10800 visibilities and their A-term
segments 8 to 240.  The autotuner times a CUDA-graph replay of grid + degrid
for every (subgrid size, launch mode) candidate, then for the gridder's
records per chunk and the degridder's channels per lane, and keeps the
fastest; the chosen configuration is then timed over several replays.  Prints one JSON
line.  Parity of this workload against the FP64 oracle is checked by the
test suite on a stratified baseline sample.

    python -m paper_2502_17789_gb300.uneven [--steps 3] [--candidates 64 96 128]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

FLOP_PER_VISPX = 34.0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--candidates", type=int, nargs="+", default=[64, 96, 128])
    ap.add_argument("--modes", nargs="+", default=["blocks", "persistent"])
    ap.add_argument("--cache", default=None, help="autotune cache file (JSON)")
    ap.add_argument("--timesteps", type=int, default=None, help="shorten the run (smaller test)")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)

    import torch

    from . import autotune, idg, synth
    from .build import build

    build()
    dev = torch.device("cuda")
    t0 = time.time()
    obs = synth.config(4, seed=args.seed, n_timesteps=args.timesteps)
    model = synth.beam_screen_model(np.random.default_rng(args.seed), rms_rad=2.0)
    A = torch.as_tensor(synth.aterms_beam_screen(obs, model), device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(args.seed)
    vis = torch.randn((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64, device=dev,
                      generator=g)
    t_inputs = time.time() - t0

    # plans per candidate subgrid size: occupancy spread
    occupancy = {}
    for L in args.candidates:
        try:
            p = idg.Plan(obs, subgrid_size=L, flags=idg.IDG_HOST_ONLY)
        except idg.IdgError as e:
            occupancy[L] = {"error": str(e)}
            continue
        sg, seg = p.subgrids(), p.segments()
        nv = (sg[:, 2] - sg[:, 1]) * (sg[:, 4] - sg[:, 3])
        nseg = (seg[:, 3] - seg[:, 2]) * (sg[seg[:, 0], 4] - sg[seg[:, 0], 3])
        st = p.stats()
        occupancy[L] = {"subgrids": int(st.n_subgrids), "segments": int(st.n_segments),
                        "vis_per_subgrid": [int(nv.min()), int(np.median(nv)), int(nv.max())],
                        "vis_per_segment": [int(nseg.min()), int(np.median(nseg)), int(nseg.max())],
                        "vis_pixels": float(st.vis_pixels)}
        p.close()

    def measure(o, L, mode, chunk, channels, mac):
        return autotune.gpu_measure(o, L, mode, chunk, channels, mac, trials=1, aterms=A, graph=True, vis=vis)

    t1 = time.time()
    choice = autotune.autotune(obs, candidates=args.candidates, modes=args.modes, cache_path=args.cache,
                               device_name=torch.cuda.get_device_name(dev), measure=measure, refresh=True)
    t_tune = time.time() - t1

    # the chosen configuration: graph replays of grid + degrid on a side stream
    side = torch.cuda.Stream(dev)
    plan = idg.Plan(obs, stream=side.cuda_stream, **choice.plan_kwargs(idg))
    st = plan.stats()
    N = obs.grid_size
    G = torch.zeros((4, N, N), dtype=torch.complex128, device=dev)
    out = torch.empty_like(vis)
    torch.cuda.synchronize(dev)
    for _ in range(args.warmup):
        plan.grid_graph(vis, A, G)
        plan.degrid_graph(G, A, out)
    plan.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    grid_ms = degrid_ms = 0.0
    for _ in range(args.steps):
        e[0].record(side)
        plan.grid_graph(vis, A, G)
        e[1].record(side)
        plan.degrid_graph(G, A, out)
        e[2].record(side)
        plan.synchronize()
        grid_ms += e[0].elapsed_time(e[1])
        degrid_ms += e[1].elapsed_time(e[2])
    grid_ms /= args.steps
    degrid_ms /= args.steps
    # per-kernel split from one profiled (non-graph) pass
    plan.profile(True)
    plan.profile_read()
    plan.grid(vis, A, G)
    plan.degrid(G, A, out)
    prof = plan.profile_read()
    plan.profile(False)
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * 128 * 2 * 2070e6
    vispx = float(st.vis_pixels)
    kern = {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items()}
    for k in ("gridder", "degridder"):
        if prof[k][0] > 0:
            kern[k]["vispx_per_s"] = vispx / (prof[k][0] * 1e-3)
            kern[k]["frac_of_fp32_peak"] = round(vispx * FLOP_PER_VISPX / (prof[k][0] * 1e-3) / peak, 4)
    line = {"workload": "256 stations, log-normal radii (<= 3 km), 32640 baselines, 360 x 0.5 s, 30 ch 140-170 MHz, "
                        "8192^2 grid, P=18, FOV 0.5, A-terms every 4 s (beam x screen)",
            "n_vis": int(obs.n_vis), "choice": choice.as_dict(), "occupancy": occupancy,
            "plan": {"subgrids": int(st.n_subgrids), "segments": int(st.n_segments), "batches": int(st.n_batches),
                     "grid_items": int(st.n_grid_items), "degrid_items": int(st.n_degrid_items)},
            "graph_replay_ms": {"grid": grid_ms, "degrid": degrid_ms},
            "vis_per_s": 2.0 * obs.n_vis / ((grid_ms + degrid_ms) * 1e-3),
            "vis_pixels_per_direction": vispx, "kernels": kern,
            "seconds": {"inputs": t_inputs, "autotune": t_tune}}
    print(json.dumps(line), flush=True)
    plan.close()


if __name__ == "__main__":
    main()
