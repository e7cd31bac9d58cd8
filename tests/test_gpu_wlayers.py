"""w layers on the GPU (IDG_W_LAYERS, Section 2.4 with w-stacking, Eq. 11 and
Eq. 12) against the FP64 oracle: a compact array whose stations sit up to a
few hundred metres apart in height, so |w| spans several layers of 2 w_max.
Tolerances as in the single-layer tests: gridder relative L2 <= 1e-5 over all
layers, degridder rms / peak <= 1e-5, the image taper-weighted (Parseval)."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _obs(seed=0):
    rng = np.random.default_rng(seed)
    enu = synth.stations_uniform_disk(rng, 12, 600.0)
    enu[:, 2] = rng.normal(0.0, 300.0, enu.shape[0])
    return synth.make_observation(enu, 12, 2.0, np.linspace(140e6, 170e6, 16), 4, 512, 64, 18, 0.5, name="w-layers")


def _setup(idg_mod, oracle_mod, seed=0, persistent=False):
    obs = _obs(seed)
    rng = np.random.default_rng(seed + 1)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    vis = synth.random_visibilities(rng, obs)
    flags = idg_mod.IDG_W_LAYERS | (idg_mod.IDG_PERSISTENT if persistent else 0)
    plan = idg_mod.Plan(obs, flags=flags)
    geom = oracle_mod.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                               aterm_nodes=obs.aterm_nodes, flags=oracle_mod.FLAG_W_LAYERS)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    np.testing.assert_array_equal(plan.subgrids(), pl.subgrids)
    np.testing.assert_array_equal(plan.layers(), np.stack([pl.layers, pl.conj], axis=1))
    assert pl.conj.any() and not pl.conj.all()
    assert plan.grid_shape() == oracle_mod.grid_shape(geom, pl) and plan.grid_shape()[0] >= 2
    args = (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)
    return obs, A, vis, plan, geom, pl, args


@pytest.mark.parametrize("persistent", [False, True])
def test_w_layers_grid_and_degrid(idg_mod, oracle_mod, cuda_device, persistent):
    import torch
    obs, A, vis, plan, geom, pl, args = _setup(idg_mod, oracle_mod, persistent=persistent)
    vis64 = vis.astype(np.complex64)
    A_d = torch.as_tensor(A).cuda()
    G = torch.zeros(plan.grid_shape(), dtype=torch.complex128, device="cuda")
    plan.grid(torch.as_tensor(vis64).cuda(), A_d, G)
    plan.synchronize()
    G_ref = oracle_mod.grid(*args, vis64.astype(np.complex128), A.astype(np.complex128))
    err = np.linalg.norm(G.cpu().numpy() - G_ref) / np.linalg.norm(G_ref)
    assert err < TOL, err
    rng = np.random.default_rng(3)
    Gr = (rng.standard_normal(G_ref.shape) + 1j * rng.standard_normal(G_ref.shape)) * 1e-3
    V = torch.empty(vis.shape, dtype=torch.complex64, device="cuda")
    plan.degrid(torch.as_tensor(Gr).cuda(), A_d, V)
    plan.synchronize()
    V_ref = oracle_mod.degrid(*args, Gr, A.astype(np.complex128))
    derr = np.sqrt(np.mean(np.abs(V.cpu().numpy() - V_ref) ** 2)) / np.abs(V_ref).max()
    assert derr < TOL, derr
    plan.close()


def test_w_stacked_invert_and_predict(idg_mod, oracle_mod, cuda_device):
    import torch
    obs, A, vis, plan, geom, pl, args = _setup(idg_mod, oracle_mod, seed=4)
    N = obs.grid_size
    vis64 = vis.astype(np.complex64)
    A_d = torch.as_tensor(A).cuda()
    G = torch.empty(plan.grid_shape(), dtype=torch.complex128, device="cuda")
    I = torch.empty((4, N, N), dtype=torch.complex128, device="cuda")
    plan.invert(torch.as_tensor(vis64).cuda(), A_d, G, I)
    plan.synchronize()
    ref = oracle_mod.invert(*args, vis64.astype(np.complex128), A.astype(np.complex128))
    W = oracle_mod.image_taper(geom)[None]
    err = np.linalg.norm((I.cpu().numpy() - ref) * W) / np.linalg.norm(ref * W)
    assert err < TOL, err
    # predict a point-source model inside the central 1/1.5 of the field
    rng = np.random.default_rng(6)
    img = np.zeros((4, N, N), complex)
    for _ in range(20):
        p, q = rng.integers(N // 2 - N // 3 + 1, N // 2 + N // 3 - 1, 2)
        img[0, q, p] += rng.lognormal()
        img[3, q, p] = img[0, q, p]
    V = torch.empty(vis.shape, dtype=torch.complex64, device="cuda")
    plan.predict(torch.as_tensor(img).cuda(), A_d, G, V)
    plan.synchronize()
    V_ref = oracle_mod.predict(*args, img, A.astype(np.complex128))
    derr = np.sqrt(np.mean(np.abs(V.cpu().numpy() - V_ref) ** 2)) / np.abs(V_ref).max()
    assert derr < TOL, derr
    # adjointness of the pair on the GPU results, in the real inner product
    # (the mirrored rows are conjugated)
    lhs = np.vdot(V.cpu().numpy().astype(np.complex128), vis64.astype(np.complex128)).real
    rhs = np.vdot(img, I.cpu().numpy()).real
    assert abs(lhs - rhs) / abs(rhs) < TOL
    plan.close()
