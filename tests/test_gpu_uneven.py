"""The 256-station uneven workload at full size (352.5 M visibilities,
8192^2 grid, A-terms every 4 s), in the persistent work-queue launch with
CUDA-graph replay and L = 64 (the autotuner's choice on GB300).

The oracle checks what it can compute a subgrid at a time: degridded
visibilities of an occupancy-stratified seeded sample of subgrids, and the
full grid of a sub-observation made of the sampled subgrids' baselines (the
planner partitions each baseline independently, so the sub-observation's
subgrids are the full plan's).  The full-size grid is checked through the
adjoint identity."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import parallel, synth

pytestmark = pytest.mark.gpu

GRID_TOL = 1e-5
DEGRID_TOL = 1e-5
L = 64


def _stratified(rng, counts, n):
    order = np.argsort(counts, kind="stable")
    picks = [order[int(q)] for q in np.linspace(0, len(order) - 1, n)]
    extra = rng.choice(len(order), size=n // 2, replace=False)
    return np.unique(np.concatenate([picks, extra]))


@pytest.fixture(scope="module")
def uneven(idg_mod, oracle_mod, cuda_device):
    import torch
    obs = synth.config(4, seed=0)
    model = synth.beam_screen_model(np.random.default_rng(0), rms_rad=2.0)
    A = synth.aterms_with_leakage(np.random.default_rng(1), synth.aterms_beam_screen(obs, model), 0.05)
    side = torch.cuda.Stream()
    plan = idg_mod.Plan(obs, subgrid_size=L, flags=idg_mod.IDG_PERSISTENT, stream=side.cuda_stream)
    geom = oracle_mod.Geometry(obs.grid_size, L, obs.kernel_padding, obs.image_size)
    ref_plan = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    g = torch.Generator(device="cuda")
    g.manual_seed(4)
    vis_d = torch.randn((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64,
                        device="cuda", generator=g)
    A_d = torch.as_tensor(A).cuda()
    torch.cuda.synchronize()
    yield dict(obs=obs, A=A, A_d=A_d, vis_d=vis_d, plan=plan, side=side, geom=geom, ref_plan=ref_plan)
    plan.close()


def test_uneven_plan_is_bit_exact(uneven):
    np.testing.assert_array_equal(uneven["plan"].subgrids(), uneven["ref_plan"].subgrids)
    np.testing.assert_array_equal(uneven["plan"].segments(), uneven["ref_plan"].segments)
    sg = uneven["ref_plan"].subgrids
    counts = (sg[:, 2] - sg[:, 1]) * (sg[:, 4] - sg[:, 3])
    assert counts.min() < 1000 and counts.max() >= 10000   # the uneven spread the workload is for


def _sample(uneven):
    full = uneven["ref_plan"]
    counts = (full.subgrids[:, 2] - full.subgrids[:, 1]) * (full.subgrids[:, 4] - full.subgrids[:, 3])
    idx = _stratified(np.random.default_rng(12), counts, 12)
    bls = np.unique(full.subgrids[idx, 0])
    return idx, bls


def test_uneven_degrid_sampled_subgrids(uneven, oracle_mod):
    import torch
    obs, plan, full = uneven["obs"], uneven["plan"], uneven["ref_plan"]
    N = obs.grid_size
    g = torch.Generator(device="cuda")
    g.manual_seed(6)
    G_d = torch.randn((4, N, N), dtype=torch.complex128, device="cuda", generator=g)
    V_d = torch.empty_like(uneven["vis_d"])
    torch.cuda.synchronize()
    plan.degrid_graph(G_d, uneven["A_d"], V_d)
    plan.synchronize()
    idx, bls = _sample(uneven)
    remap = {int(b): n for n, b in enumerate(bls)}
    keep = np.isin(full.segments[:, 0], idx)
    sub_sg = full.subgrids[np.sort(idx)].copy()
    pos = {int(o): n for n, o in enumerate(np.sort(idx))}
    segs = full.segments[keep].copy()
    segs[:, 0] = [pos[int(s)] for s in segs[:, 0]]
    sub_sg[:, 0] = [remap[int(b)] for b in sub_sg[:, 0]]
    sub_obs = parallel.sub_observation(obs, bls)
    V_ref = oracle_mod.degrid(uneven["geom"], obs.n_stations, sub_obs.baselines, sub_obs.uvw, obs.freqs,
                              obs.aterm_offsets, oracle_mod.Plan(sub_sg, segs), G_d.cpu().numpy(),
                              uneven["A"].astype(np.complex128))
    V = V_d[torch.as_tensor(bls, device="cuda")].cpu().numpy()
    mask = np.zeros(V.shape[:3], bool)
    for b, t0, t1, c0, c1, *_ in sub_sg:
        mask[b, t0:t1, c0:c1] = True
    got, ref = V[mask], V_ref[mask]
    err = np.sqrt(np.mean(np.abs(got - ref) ** 2)) / np.abs(ref).max()
    assert err < DEGRID_TOL, err


@pytest.mark.parametrize("tensor_gridder", [False, True])
def test_uneven_grid_sampled_baselines(uneven, idg_mod, oracle_mod, tensor_gridder):
    """Grid of the sampled subgrids' baselines, same plan rows, same launch
    mode, against the oracle; with the tensor-core gridder (the library's
    default, and the autotuner's choice for this workload on GB300) and with
    the FP32-pipe gridder."""
    import torch
    obs = uneven["obs"]
    _, bls = _sample(uneven)
    sub = parallel.sub_observation(obs, bls)
    side = uneven["side"]
    mac = idg_mod.IDG_MAC_TENSOR if tensor_gridder else idg_mod.IDG_MAC_TENSOR_DEGRID
    plan = idg_mod.Plan(sub, subgrid_size=L, flags=idg_mod.IDG_PERSISTENT, stream=side.cuda_stream, mac_unit=mac)
    assert plan.stats().mac_unit == mac
    try:
        full = uneven["ref_plan"]
        rows = full.subgrids[np.isin(full.subgrids[:, 0], bls)].copy()
        rows[:, 0] = np.searchsorted(bls, rows[:, 0])
        np.testing.assert_array_equal(plan.subgrids(), rows)
        vis_d = uneven["vis_d"][torch.as_tensor(bls, device="cuda")].contiguous()
        N = obs.grid_size
        G_d = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        plan.grid_graph(vis_d, uneven["A_d"], G_d)
        plan.synchronize()
        ref_plan = oracle_mod.plan(uneven["geom"], sub.uvw, obs.freqs, obs.aterm_offsets)
        G_ref = oracle_mod.grid(uneven["geom"], obs.n_stations, sub.baselines, sub.uvw, obs.freqs,
                                obs.aterm_offsets, ref_plan, vis_d.cpu().numpy().astype(np.complex128),
                                uneven["A"].astype(np.complex128))
        G = G_d.cpu().numpy()
        err = float(np.linalg.norm((G - G_ref).ravel()) / np.linalg.norm(G_ref.ravel()))
        assert err < GRID_TOL, err
    finally:
        plan.close()


def test_uneven_adjoint_identity_full_size(uneven):
    import torch
    obs, plan = uneven["obs"], uneven["plan"]
    N = obs.grid_size
    G_d = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(8)
    R = torch.randn((4, N, N), dtype=torch.complex128, device="cuda", generator=g)
    V_d = torch.empty_like(uneven["vis_d"])
    torch.cuda.synchronize()
    plan.grid_graph(uneven["vis_d"], uneven["A_d"], G_d)
    plan.degrid_graph(R, uneven["A_d"], V_d)
    plan.synchronize()
    lhs = torch.vdot(V_d.reshape(-1).to(torch.complex128), uneven["vis_d"].reshape(-1).to(torch.complex128))
    rhs = torch.vdot(R.reshape(-1), G_d.reshape(-1))
    assert abs(complex(lhs) - complex(rhs)) / abs(complex(rhs)) < GRID_TOL
