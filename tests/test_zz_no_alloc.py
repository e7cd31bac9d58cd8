"""idg_grid_noalloc: the gridding entry point for callers that cannot
allocate device memory where they grid (real-time pipelines that reserve all
memory at start-up, hosts whose device memory belongs to another allocator).
It keeps its subgrid images in a static device buffer; its result must match
idg_grid's on two calls in a row.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import synth

pytestmark = pytest.mark.gpu

GRID_TOL = 1e-5  # the gridder tolerance used by the parity tests


def test_noalloc_matches_idg_grid_twice(idg_mod, cuda_device):
    import torch
    # 120 baselines -> more subgrids than one 32 MiB sub-batch holds at L = 96
    obs = synth.config(2, seed=3, n_stations=16, n_timesteps=12, n_channels=24)
    rng = np.random.default_rng(7)
    A = torch.as_tensor(synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)).cuda()
    vis = torch.as_tensor(synth.random_visibilities(rng, obs)).cuda()
    plan = idg_mod.Plan(obs)
    cap = (32 << 20) // (4 * obs.subgrid_size ** 2 * 8)
    assert plan.stats().n_subgrids > cap
    N = obs.grid_size
    ref = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
    plan.grid(vis, A, ref)
    plan.synchronize()
    ref = ref.cpu().numpy()
    for _ in range(2):
        G = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
        idg_mod.idg_grid_noalloc(plan.handle, idg_mod._dev_ptr(vis), idg_mod._dev_ptr(A), idg_mod._dev_ptr(G))
        plan.synchronize()
        got = G.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < GRID_TOL, err
    plan.close()
