"""Image-domain wrapper on the GPU (idg_invert / idg_predict, Eq. 11 and
Eq. 12 with the single w = 0 layer) against the FP64 oracle.

Tolerances.  The image is the gridded plane transformed and divided by
L^2 T(l) T(m); by Parseval the taper-weighted image error equals the grid
error, so the invert check is ||(I_gpu - I_ref) T T|| / ||I_ref T T|| <= 1e-5,
the gridder's tolerance.  predict is checked like the degridder (rms error
over the peak visibility <= 1e-5) on a model whose sources lie in the central
1/1.5 of the field, where 1/T^2 stays below the FP32 budget."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _setup(idg_mod, oracle_mod, seed=0, stations=12):
    obs = synth.config(1, seed=seed, n_stations=stations, n_timesteps=8)
    obs.aterm_offsets = np.array([0, 4, 8], np.int32)
    rng = np.random.default_rng(seed)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    vis = synth.random_visibilities(rng, obs)
    plan = idg_mod.Plan(obs)
    geom = oracle_mod.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                               aterm_nodes=obs.aterm_nodes)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    args = (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)
    return obs, A, vis, plan, geom, args


def _model_image(rng, obs, n_src=30):
    """Point sources on image pixels inside the central 1/1.5 of the field."""
    N = obs.grid_size
    img = np.zeros((4, N, N), complex)
    lo, hi = int(N / 2 - N / 3) + 1, int(N / 2 + N / 3) - 1
    for _ in range(n_src):
        p, q = rng.integers(lo, hi, 2)
        s = rng.lognormal(0.0, 1.0)
        img[0, q, p] += s
        img[3, q, p] += s
    return img


def test_invert_matches_oracle(idg_mod, oracle_mod, cuda_device):
    import torch
    obs, A, vis, plan, geom, args = _setup(idg_mod, oracle_mod)
    N = obs.grid_size
    G = torch.empty((4, N, N), dtype=torch.complex128, device="cuda")
    I = torch.empty_like(G)
    vis64 = vis.astype(np.complex64)
    plan.invert(torch.as_tensor(vis64).cuda(), torch.as_tensor(A).cuda(), G, I)
    plan.synchronize()
    ref = oracle_mod.invert(*args, vis64.astype(np.complex128), A.astype(np.complex128))
    W = oracle_mod.image_taper(geom)[None]
    got = I.cpu().numpy()
    err = np.linalg.norm((got - ref) * W) / np.linalg.norm(ref * W)
    assert err < TOL, err
    # the grid argument holds the gridded plane
    G_ref = oracle_mod.grid(*args, vis64.astype(np.complex128), A.astype(np.complex128))
    assert np.linalg.norm(G.cpu().numpy() - G_ref) / np.linalg.norm(G_ref) < TOL
    plan.close()


def test_predict_matches_oracle(idg_mod, oracle_mod, cuda_device):
    import torch
    obs, A, _, plan, geom, args = _setup(idg_mod, oracle_mod, seed=1)
    img = _model_image(np.random.default_rng(2), obs)
    N = obs.grid_size
    G = torch.empty((4, N, N), dtype=torch.complex128, device="cuda")
    V = torch.empty((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64, device="cuda")
    plan.predict(torch.as_tensor(img).cuda(), torch.as_tensor(A).cuda(), G, V)
    plan.synchronize()
    ref = oracle_mod.predict(*args, img, A.astype(np.complex128))
    got = V.cpu().numpy()
    err = np.sqrt(np.mean(np.abs(got - ref) ** 2)) / np.abs(ref).max()
    assert err < TOL, err
    plan.close()


def test_invert_predict_adjoint_on_gpu(idg_mod, oracle_mod, cuda_device):
    import torch
    obs, A, vis, plan, geom, args = _setup(idg_mod, oracle_mod, seed=3)
    img = _model_image(np.random.default_rng(4), obs, 50)
    N = obs.grid_size
    A_d = torch.as_tensor(A).cuda()
    vis_d = torch.as_tensor(vis.astype(np.complex64)).cuda()
    G = torch.empty((4, N, N), dtype=torch.complex128, device="cuda")
    I = torch.empty_like(G)
    V = torch.empty_like(vis_d)
    plan.invert(vis_d, A_d, G, I)
    plan.predict(torch.as_tensor(img).cuda(), A_d, G, V)
    plan.synchronize()
    lhs = complex(torch.vdot(V.reshape(-1).to(torch.complex128), vis_d.reshape(-1).to(torch.complex128)))
    rhs = complex(torch.vdot(torch.as_tensor(img).cuda().reshape(-1), I.reshape(-1)))
    assert abs(lhs - rhs) / abs(rhs) < TOL
    plan.close()


def test_user_taper_is_unsupported(idg_mod, cuda_device):
    import torch
    obs = synth.config(1, seed=0, n_stations=4, n_timesteps=2)
    plan = idg_mod.Plan(obs, taper_user=np.ones(obs.subgrid_size))
    N = obs.grid_size
    G = torch.empty((4, N, N), dtype=torch.complex128, device="cuda")
    vis = torch.zeros((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64, device="cuda")
    A = torch.as_tensor(synth.aterms_identity(obs.n_intervals, obs.n_stations)).cuda()
    with pytest.raises(idg_mod.IdgError) as e:
        plan.invert(vis, A, G, torch.empty_like(G))
    assert e.value.status == 8
    plan.close()
