"""Stokes-I mode on the GPU (IDG_STOKES_I: one grid / image plane, I = (XX +
YY)/2 of each corrected subgrid image; prediction from an unpolarised model)
against the FP64 oracle, with the tolerances of the 4-plane tests: gridder
relative L2 <= 1e-5, degridder rms / peak <= 1e-5, images taper-weighted."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _setup(idg_mod, oracle_mod, seed=0, flags=0, oflags=0, obs=None, diagonal=None, degrid_channels=0):
    obs = obs or synth.config(2, seed=seed, n_stations=14, n_timesteps=12, n_channels=16)
    rng = np.random.default_rng(seed + 1)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    if diagonal == "all":
        A[..., 1:3] = 0.0
    elif diagonal == "mixed":      # diagonal Jones matrices for every other (interval, station)
        A[::2, ::2, ..., 1:3] = 0.0
        A[1::2, 1::2, ..., 1:3] = 0.0
    vis = synth.random_visibilities(rng, obs).astype(np.complex64)
    plan = idg_mod.Plan(obs, flags=idg_mod.IDG_STOKES_I | flags, degrid_channels=degrid_channels)
    geom = oracle_mod.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                               aterm_nodes=obs.aterm_nodes, flags=oracle_mod.FLAG_STOKES_I | oflags)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    args = (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)
    return obs, A, vis, plan, geom, pl, args


@pytest.mark.parametrize("persistent,diagonal", [(False, None), (True, None), (False, "all"), (True, "mixed")])
def test_stokes_i_grid_and_degrid(idg_mod, oracle_mod, cuda_device, persistent, diagonal):
    """Full-Jones, diagonal and mixed A-terms: with diagonal ones the kernels
    sum only XX and YY (the predicted XY and YX are zero)."""
    import torch
    obs, A, vis, plan, geom, pl, args = _setup(idg_mod, oracle_mod, diagonal=diagonal,
                                                flags=idg_mod.IDG_PERSISTENT if persistent else 0)
    N = obs.grid_size
    assert plan.grid_shape() == (1, N, N) and plan.stats().n_pol == 1
    A_d = torch.as_tensor(A).cuda()
    G = torch.zeros(plan.grid_shape(), dtype=torch.complex128, device="cuda")
    plan.grid(torch.as_tensor(vis).cuda(), A_d, G)
    plan.synchronize()
    G_ref = oracle_mod.grid(*args, vis.astype(np.complex128), A.astype(np.complex128))
    assert G_ref.shape == (1, N, N)
    err = np.linalg.norm(G.cpu().numpy() - G_ref) / np.linalg.norm(G_ref)
    assert err < TOL, err
    rng = np.random.default_rng(9)
    Gr = (rng.standard_normal(G_ref.shape) + 1j * rng.standard_normal(G_ref.shape)) * 1e-3
    V = torch.empty(vis.shape, dtype=torch.complex64, device="cuda")
    plan.degrid(torch.as_tensor(Gr).cuda(), A_d, V)
    plan.synchronize()
    V_ref = oracle_mod.degrid(*args, Gr, A.astype(np.complex128))
    derr = np.sqrt(np.mean(np.abs(V.cpu().numpy() - V_ref) ** 2)) / np.abs(V_ref).max()
    assert derr < TOL, derr
    if diagonal == "all":
        assert not V.cpu().numpy()[..., 1:3].any()
    plan.close()


@pytest.mark.parametrize("channels,diagonal", [(2, "all"), (4, "all"), (4, "mixed")])
def test_stokes_i_degrid_channel_groups(idg_mod, oracle_mod, cuda_device, channels, diagonal):
    """Stokes-I prediction with 2 or 4 channels per degridder lane (rotation
    by the channel-step phasor), on the XX/YY-only path (diagonal A-terms)
    and with items that mix it with full Jones matrices."""
    import torch
    obs, A, vis, plan, geom, pl, args = _setup(idg_mod, oracle_mod, seed=5, diagonal=diagonal,
                                                degrid_channels=channels)
    assert plan.stats().degrid_channels == channels
    rng = np.random.default_rng(10)
    N = obs.grid_size
    Gr = (rng.standard_normal((1, N, N)) + 1j * rng.standard_normal((1, N, N))) * 1e-3
    V = torch.empty(vis.shape, dtype=torch.complex64, device="cuda")
    plan.degrid(torch.as_tensor(Gr).cuda(), torch.as_tensor(A).cuda(), V)
    plan.synchronize()
    V_ref = oracle_mod.degrid(*args, Gr, A.astype(np.complex128))
    derr = np.sqrt(np.mean(np.abs(V.cpu().numpy() - V_ref) ** 2)) / np.abs(V_ref).max()
    assert derr < TOL, derr
    plan.close()


def test_stokes_i_subgrid_images(idg_mod, oracle_mod, cuda_device):
    import torch
    obs, A, vis, plan, geom, pl, args = _setup(idg_mod, oracle_mod, seed=2,
                                                obs=synth.config(1, seed=2, n_stations=10, n_timesteps=8))
    L = obs.subgrid_size
    _, img_ref, uv_ref = oracle_mod.grid(*args, vis.astype(np.complex128), A.astype(np.complex128),
                                         want_subgrids=True)
    vis_d, A_d = torch.as_tensor(vis).cuda(), torch.as_tensor(A).cuda()   # kept alive across the async call
    for stage, ref in ((0, img_ref), (1, uv_ref)):
        out = torch.zeros((pl.subgrids.shape[0], 1, L, L), dtype=torch.complex64, device="cuda")
        idg_mod.idg_subgrid_images(plan.handle, idg_mod._dev_ptr(vis_d), idg_mod._dev_ptr(A_d), stage,
                                   idg_mod._dev_ptr(out))
        plan.synchronize()
        got = out.cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL
    plan.close()


def test_stokes_i_invert_predict_with_w_layers_and_normalisation(idg_mod, oracle_mod, cuda_device):
    """Stokes I combined with w layers and the A-term power normalisation:
    invert and predict against the oracle."""
    import torch
    rng = np.random.default_rng(4)
    enu = synth.stations_uniform_disk(rng, 12, 600.0)
    enu[:, 2] = rng.normal(0.0, 300.0, enu.shape[0])
    obs = synth.make_observation(enu, 12, 2.0, np.linspace(140e6, 170e6, 16), 4, 512, 64, 18, 0.5, name="w-layers")
    obs_, A, vis, plan, geom, pl, args = _setup(
        idg_mod, oracle_mod, seed=5, obs=obs,
        flags=idg_mod.IDG_W_LAYERS | idg_mod.IDG_NORMALIZE_ATERM, oflags=oracle_mod.FLAG_W_LAYERS)
    N = obs.grid_size
    assert plan.grid_shape()[1] == 1 and plan.grid_shape()[0] >= 2
    A_d = torch.as_tensor(A).cuda()
    G = torch.empty(plan.grid_shape(), dtype=torch.complex128, device="cuda")
    I = torch.empty(plan.image_shape(), dtype=torch.complex128, device="cuda")
    plan.invert(torch.as_tensor(vis).cuda(), A_d, G, I)
    plan.synchronize()
    ref = oracle_mod.invert(*args, vis.astype(np.complex128), A.astype(np.complex128), normalize=True)
    Wt = oracle_mod.image_taper(geom)[None]
    err = np.linalg.norm((I.cpu().numpy() - ref) * Wt) / np.linalg.norm(ref * Wt)
    assert err < TOL, err
    img = np.zeros((1, N, N), complex)
    for _ in range(12):
        p, q = rng.integers(N // 2 - N // 3 + 1, N // 2 + N // 3 - 1, 2)
        img[0, q, p] += rng.lognormal()
    V = torch.empty(vis.shape, dtype=torch.complex64, device="cuda")
    plan.predict(torch.as_tensor(img).cuda(), A_d, G, V)
    plan.synchronize()
    V_ref = oracle_mod.predict(*args, img, A.astype(np.complex128))
    derr = np.sqrt(np.mean(np.abs(V.cpu().numpy() - V_ref) ** 2)) / np.abs(V_ref).max()
    assert derr < TOL, derr
    plan.close()
