"""A-term power normalisation on the GPU (IDG_NORMALIZE_ATERM, Section 3.3)
against the FP64 oracle: every segment's corrected image divided per pixel by
||A_p^H A_q||_F, the weight map sum n_seg / f on the subgrid lattice, and the
normalised dirty image (idg_invert divides by the weights' average).
Tolerances as elsewhere: grid and taper-weighted image relative L2 <= 1e-5;
the weights (FP32 per thread, FP64 atomics) relative <= 1e-5."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _setup(idg_mod, oracle_mod, seed=0, diagonal=False, persistent=False):
    obs = synth.config(2, seed=seed, n_stations=14, n_timesteps=12, n_channels=16)
    rng = np.random.default_rng(seed + 1)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    if diagonal:
        A[..., 1] = 0.0
        A[..., 2] = 0.0
    vis = synth.random_visibilities(rng, obs).astype(np.complex64)
    flags = idg_mod.IDG_NORMALIZE_ATERM | (idg_mod.IDG_PERSISTENT if persistent else 0)
    plan = idg_mod.Plan(obs, flags=flags)
    geom = oracle_mod.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                               aterm_nodes=obs.aterm_nodes)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    args = (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)
    return obs, A, vis, plan, geom, args


@pytest.mark.parametrize("diagonal,persistent", [(False, False), (True, False), (False, True)])
def test_normalised_grid_and_weights(idg_mod, oracle_mod, cuda_device, diagonal, persistent):
    import torch
    obs, A, vis, plan, geom, args = _setup(idg_mod, oracle_mod, diagonal=diagonal, persistent=persistent)
    N, L = obs.grid_size, obs.subgrid_size
    G = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
    plan.grid(torch.as_tensor(vis).cuda(), torch.as_tensor(A).cuda(), G)
    plan.synchronize()
    G_ref, W_ref = oracle_mod.grid(*args, vis.astype(np.complex128), A.astype(np.complex128), normalize=True)
    err = np.linalg.norm(G.cpu().numpy() - G_ref) / np.linalg.norm(G_ref)
    assert err < TOL, err
    W = plan.aterm_weights(reset=True)
    assert W[L * L] == W_ref[L * L] == obs.n_baselines * obs.n_timesteps * obs.n_channels
    werr = np.abs(W[: L * L] - W_ref[: L * L]).max() / np.abs(W_ref[: L * L]).max()
    assert werr < TOL, werr
    # reset cleared them
    assert not plan.aterm_weights().any()
    plan.close()


def test_normalised_invert_matches_oracle(idg_mod, oracle_mod, cuda_device):
    import torch
    obs, A, vis, plan, geom, args = _setup(idg_mod, oracle_mod, seed=3)
    N = obs.grid_size
    G = torch.empty((4, N, N), dtype=torch.complex128, device="cuda")
    I = torch.empty_like(G)
    A_d = torch.as_tensor(A).cuda()
    V_d = torch.as_tensor(vis).cuda()
    for _ in range(2):   # invert resets the weights: a second call gives the same image
        plan.invert(V_d, A_d, G, I)
        plan.synchronize()
    ref = oracle_mod.invert(*args, vis.astype(np.complex128), A.astype(np.complex128), normalize=True)
    Wt = oracle_mod.image_taper(geom)[None]
    got = I.cpu().numpy()
    err = np.linalg.norm((got - ref) * Wt) / np.linalg.norm(ref * Wt)
    assert err < TOL, err
    plan.close()


def test_noalloc_refuses_normalised_plans(idg_mod, cuda_device):
    import torch
    obs = synth.config(1, seed=0, n_stations=8, n_timesteps=4)
    plan = idg_mod.Plan(obs, flags=idg_mod.IDG_NORMALIZE_ATERM)
    N = obs.grid_size
    vis = torch.zeros((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64, device="cuda")
    A = torch.as_tensor(synth.aterms_identity(obs.n_intervals, obs.n_stations, obs.aterm_nodes)).cuda()
    G = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
    with pytest.raises(idg_mod.IdgError) as e:
        idg_mod.idg_grid_noalloc(plan.handle, idg_mod._dev_ptr(vis), idg_mod._dev_ptr(A), idg_mod._dev_ptr(G))
    assert e.value.status == 8
    plan.close()
    plain = idg_mod.Plan(obs)
    with pytest.raises(idg_mod.IdgError):
        plain.aterm_weights()
    plain.close()
