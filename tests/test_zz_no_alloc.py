"""idg_grid_noalloc: the gridding entry point for callers that cannot
allocate device memory where they grid (real-time pipelines that reserve all
memory at start-up, hosts whose device memory belongs to another allocator).
It keeps its subgrid images in a static device buffer; on two calls in a row
its result must match idg_grid's and the FP64 oracle's grid, with a single
w = 0 plane set and with w layers (mirrored subgrids, several plane sets).
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import synth

pytestmark = pytest.mark.gpu

GRID_TOL = 1e-5  # the gridder tolerance used by the parity tests


def _oracle_grid(oracle_mod, obs, flags, vis, A):
    geom = oracle_mod.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                               aterm_nodes=obs.aterm_nodes, flags=flags)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    return oracle_mod.grid(geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl,
                           vis.astype(np.complex128), A.astype(np.complex128))


def _check_twice(idg_mod, plan, vis_d, A_d, ref_lib, ref_oracle):
    import torch
    for _ in range(2):
        G = torch.zeros(plan.grid_shape(), dtype=torch.complex128, device="cuda")
        idg_mod.idg_grid_noalloc(plan.handle, idg_mod._dev_ptr(vis_d), idg_mod._dev_ptr(A_d), idg_mod._dev_ptr(G))
        plan.synchronize()
        got = G.cpu().numpy()
        err_lib = np.linalg.norm((got - ref_lib).ravel()) / np.linalg.norm(ref_lib.ravel())
        err_or = np.linalg.norm((got - ref_oracle).ravel()) / np.linalg.norm(ref_oracle.ravel())
        assert err_lib < GRID_TOL, err_lib
        assert err_or < GRID_TOL, err_or


def test_noalloc_matches_idg_grid_and_oracle_twice(idg_mod, oracle_mod, cuda_device):
    import torch
    # 120 baselines -> more subgrids than one 32 MiB sub-batch holds at L = 96
    obs = synth.config(2, seed=3, n_stations=16, n_timesteps=12, n_channels=24)
    rng = np.random.default_rng(7)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    vis = synth.random_visibilities(rng, obs)
    A_d, vis_d = torch.as_tensor(A).cuda(), torch.as_tensor(vis).cuda()
    plan = idg_mod.Plan(obs)
    try:
        cap = (32 << 20) // (4 * obs.subgrid_size ** 2 * 8)
        assert plan.stats().n_subgrids > cap
        ref = torch.zeros(plan.grid_shape(), dtype=torch.complex128, device="cuda")
        plan.grid(vis_d, A_d, ref)
        plan.synchronize()
        _check_twice(idg_mod, plan, vis_d, A_d, ref.cpu().numpy(), _oracle_grid(oracle_mod, obs, 0, vis, A))
    finally:
        plan.close()


def test_noalloc_with_w_layers_matches_idg_grid_and_oracle_twice(idg_mod, oracle_mod, cuda_device):
    """w layers: several plane sets, mirrored subgrids (w < 0 rows gridded as
    V^H at -uvw), w0 = (2k+1) w_max in the phase."""
    import torch
    rng = np.random.default_rng(0)
    enu = synth.stations_uniform_disk(rng, 12, 600.0)
    enu[:, 2] = rng.normal(0.0, 300.0, enu.shape[0])
    obs = synth.make_observation(enu, 12, 2.0, np.linspace(140e6, 170e6, 16), 4, 512, 64, 18, 0.5, name="w-layers")
    rng = np.random.default_rng(1)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    vis = synth.random_visibilities(rng, obs)
    A_d, vis_d = torch.as_tensor(A).cuda(), torch.as_tensor(vis).cuda()
    plan = idg_mod.Plan(obs, flags=idg_mod.IDG_W_LAYERS)
    try:
        lay = plan.layers()
        assert plan.grid_shape()[0] >= 2 and lay[:, 1].any() and not lay[:, 1].all()
        ref = torch.zeros(plan.grid_shape(), dtype=torch.complex128, device="cuda")
        plan.grid(vis_d, A_d, ref)
        plan.synchronize()
        ref_or = _oracle_grid(oracle_mod, obs, oracle_mod.FLAG_W_LAYERS, vis, A)
        _check_twice(idg_mod, plan, vis_d, A_d, ref.cpu().numpy(), ref_or)
    finally:
        plan.close()
