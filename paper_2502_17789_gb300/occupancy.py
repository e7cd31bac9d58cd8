"""Kernel throughput against subgrid occupancy (visibilities per subgrid).

Section 3.2 of the paper notes that a degridder with one thread per
visibility suffers when subgrids hold few visibilities, and proposes
switching designs by occupancy.  This measures both kernels on plans whose
subgrids hold a controlled number of visibilities: the MWA-like array (128
stations, 8128 baselines, 4096^2 grid, L = 96) observed with n_ch channels
and n_t timesteps, one A-term interval per timestep group, so that most
subgrids hold up to n_ch x n_t visibilities.  For each case: plan occupancy
(min / median / max), gridder and degridder device time (CUDA events around
each launch, one profiled pass after a warm-up pass) and their
visibility x pixel rates, as fractions of the nominal R_vp.

    python -m paper_2502_17789_gb300.occupancy [--cases 1x1 2x2 4x4 8x8 24x14 24x56]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

FLOP_PER_VISPX = 34.0


def run_case(idg, synth, torch, dev, n_ch, n_t, reps, degrid_channels=0):
    obs = synth.config(2, seed=0, n_channels=n_ch, n_timesteps=n_t)
    obs.aterm_offsets = np.array([0, n_t], np.int32)   # one A-term interval
    A = torch.as_tensor(synth.aterms_identity(obs.n_intervals, obs.n_stations, obs.aterm_nodes), device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    vis = torch.randn((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64, device=dev,
                      generator=g)
    plan = idg.Plan(obs, degrid_channels=degrid_channels)
    st = plan.stats()
    sg = plan.subgrids()
    nv = (sg[:, 2] - sg[:, 1]) * (sg[:, 4] - sg[:, 3])
    N = obs.grid_size
    G = torch.zeros((4, N, N), dtype=torch.complex128, device=dev)
    out = torch.empty_like(vis)
    plan.grid(vis, A, G)
    plan.degrid(G, A, out)
    plan.synchronize()
    plan.profile(True)
    plan.profile_read()
    for _ in range(reps):
        plan.grid(vis, A, G)
        plan.degrid(G, A, out)
    prof = plan.profile_read()
    plan.close()
    props = torch.cuda.get_device_properties(dev)
    r_vp = props.multi_processor_count * 128 * 2070e6 / (FLOP_PER_VISPX / 2)
    vispx = float(st.vis_pixels)
    res = {"channels": n_ch, "timesteps": n_t, "n_vis": int(obs.n_vis), "subgrids": int(st.n_subgrids),
           "vis_per_subgrid_min_median_max": [int(nv.min()), int(np.median(nv)), int(nv.max())],
           "degrid_items": int(st.n_degrid_items)}
    for k in ("gridder", "degridder", "fft_adder", "splitter_ifft", "stage"):
        ms = prof[k][0] / reps
        res[k + "_ms"] = round(ms, 3)
    for k in ("gridder", "degridder"):
        rate = vispx / (res[k + "_ms"] * 1e-3)
        res[k + "_vispx_per_s"] = rate
        res[k + "_frac"] = round(rate / r_vp, 4)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--cases", nargs="+", default=["1x1", "2x2", "4x4", "8x8", "16x16", "24x56"],
                    help="channels x timesteps per case")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
    import torch

    from . import idg, synth
    from .build import build

    build()
    dev = torch.device("cuda")
    rows = []
    for case in args.cases:
        n_ch, n_t = (int(x) for x in case.split("x"))
        rows.append(run_case(idg, synth, torch, dev, n_ch, n_t, args.reps))
        print(json.dumps(rows[-1]), flush=True)


if __name__ == "__main__":
    main()
