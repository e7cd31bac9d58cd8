"""GPU parity of the tensor-core gridder and degridder (mac_unit =
IDG_MAC_TENSOR) with the FP64 oracle: the tolerances of the FP32 path
(gridder relative L2 <= 1e-5, degridder rms |V - V_ref| / max |V_ref| <=
1e-5), at every subgrid size, with two segments per degridder item, ragged
tiles and row groups, few-visibility subgrids, 1 to 30 channels, the
persistent queue, Stokes I, w layers (mirrored rows) and the shared
multi-plan launch; plans whose channels are not uniformly spaced or that
normalise the A-term power keep the FP32 gridder."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import synth
from tests.test_gpu_parity import DEGRID_TOL, GRID_TOL, Case, _degrid_err, _random_problem, _rel

pytestmark = pytest.mark.gpu


def _grand(seed, N):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))) * 1e-3


@pytest.mark.parametrize("L,n_ch,n_t", [(32, 17, 13), (64, 7, 11), (96, 24, 9), (128, 13, 7)])
def test_tensor_degrid_matches_oracle(idg_mod, oracle_mod, cuda_device, L, n_ch, n_t):
    """Random full-Jones A-terms over several intervals (items of one and two
    segments, tiles cut by the segment boundary), the oracle's own grid and a
    random grid; the FP32 kernel's error on the same input for reference."""
    obs = synth.config(2, n_stations=9, n_timesteps=n_t, n_channels=n_ch)
    A, vis = _random_problem(1300 + L + n_ch, obs, n_int=3)
    c = Case(idg_mod, oracle_mod, obs, A, vis, L=L, mac_unit=idg_mod.IDG_MAC_TENSOR)
    st = c.plan.stats()
    assert st.mac_unit == idg_mod.IDG_MAC_TENSOR and st.degrid_channels == 1
    f = Case(idg_mod, oracle_mod, obs, A, vis, L=L, mac_unit=idg_mod.IDG_MAC_FP32)
    assert f.plan.stats().mac_unit == idg_mod.IDG_MAC_FP32
    G_ref = c.oracle_grid()
    g_tc, g_fp = _rel(c.gpu_grid(), G_ref), _rel(f.gpu_grid(), G_ref)
    print(f"L={L}: grid relative L2 error tensor {g_tc:.2e}, fp32 {g_fp:.2e}")
    assert g_tc < GRID_TOL
    for Gin in (G_ref, _grand(L, obs.grid_size)):
        V_ref = c.oracle_degrid(Gin)
        e_tc = _degrid_err(c.gpu_degrid(Gin), V_ref)
        e_fp = _degrid_err(f.gpu_degrid(Gin), V_ref)
        print(f"L={L}: degrid rms/peak error tensor {e_tc:.2e}, fp32 {e_fp:.2e}")
        assert e_tc < DEGRID_TOL


@pytest.mark.parametrize("n_ch,n_t,steps", [(1, 1, 1), (3, 3, 3), (5, 4, 2), (4, 8, 4), (3, 7, 2), (17, 2, 1),
                                            (30, 11, 5), (9, 6, 6)])
def test_tensor_degrid_low_occupancy(idg_mod, oracle_mod, cuda_device, n_ch, n_t, steps):
    """Items of 1 to 40 visibilities: those of at most 8 run in the few-lane
    FP32 kernel, the others fill one to three tiles, with and without a
    second segment."""
    obs = synth.config(2, n_stations=9, n_timesteps=n_t, n_channels=n_ch)
    obs.aterm_offsets = np.array(list(range(0, n_t, steps)) + [n_t], np.int32)
    A, vis = _random_problem(1700 + 10 * n_ch + n_t, obs)
    c = Case(idg_mod, oracle_mod, obs, A, vis, mac_unit=idg_mod.IDG_MAC_TENSOR)
    Gin = _grand(n_ch * n_t, obs.grid_size)
    assert _degrid_err(c.gpu_degrid(Gin), c.oracle_degrid(Gin)) < DEGRID_TOL
    assert _rel(c.gpu_grid(), c.oracle_grid()) < GRID_TOL


def _degrid_with(idg_mod, obs, flags, mac, Gin, A):
    import torch
    plan = idg_mod.Plan(obs, flags=flags, mac_unit=mac)
    try:
        V = torch.full((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), 7.0 + 7.0j, dtype=torch.complex64,
                       device="cuda")
        plan.degrid(torch.as_tensor(Gin).cuda(), torch.as_tensor(A).cuda(), V)
        plan.synchronize()
        return V.cpu().numpy()
    finally:
        plan.close()


@pytest.mark.parametrize("diagonal", [None, "mixed"])
def test_tensor_degrid_stokes_i_persistent(idg_mod, oracle_mod, cuda_device, diagonal):
    """Stokes-I prediction (XX = YY = I) through the persistent work queue."""
    from tests import test_gpu_stokes
    obs, A, vis, plan, geom, pl, args = test_gpu_stokes._setup(idg_mod, oracle_mod, seed=5, diagonal=diagonal)
    plan.close()
    rng = np.random.default_rng(11)
    N = obs.grid_size
    Gr = (rng.standard_normal((1, N, N)) + 1j * rng.standard_normal((1, N, N))) * 1e-3
    V = _degrid_with(idg_mod, obs, idg_mod.IDG_STOKES_I | idg_mod.IDG_PERSISTENT, idg_mod.IDG_MAC_TENSOR, Gr, A)
    V_ref = oracle_mod.degrid(*args, Gr, A.astype(np.complex128))
    assert _degrid_err(V, V_ref) < DEGRID_TOL


def test_tensor_degrid_w_layers(idg_mod, oracle_mod, cuda_device):
    """w layers with mirrored rows (the degridder writes V^H of the mirror)."""
    from tests import test_gpu_wlayers
    obs, A, vis, plan, geom, pl, args = test_gpu_wlayers._setup(idg_mod, oracle_mod, seed=2)
    shape = plan.grid_shape()
    plan.close()
    rng = np.random.default_rng(4)
    Gr = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 1e-3
    V = _degrid_with(idg_mod, obs, idg_mod.IDG_W_LAYERS, idg_mod.IDG_MAC_TENSOR, Gr, A)
    V_ref = oracle_mod.degrid(*args, Gr, A.astype(np.complex128))
    assert _degrid_err(V, V_ref) < DEGRID_TOL


def test_tensor_degrid_many_equals_single_calls(idg_mod, cuda_device):
    """Several tensor-core plans in one shared launch give the single-plan
    results; plans of different mac units are refused together."""
    import torch
    obs_list = [synth.config(2, seed=s, n_stations=6 + 2 * s, n_timesteps=9, n_channels=10 + s) for s in range(3)]
    plans, Vs, Gs, As = [], [], [], []
    for s, obs in enumerate(obs_list):
        rng = np.random.default_rng(40 + s)
        plans.append(idg_mod.Plan(obs, mac_unit=idg_mod.IDG_MAC_TENSOR))
        As.append(torch.as_tensor(synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
                                  .astype(np.complex64)).cuda())
        Gs.append(torch.as_tensor(_grand(50 + s, obs.grid_size)).cuda())
        Vs.append(torch.empty((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64,
                              device="cuda"))
    try:
        idg_mod.degrid_many(plans, Gs, As, Vs)
        torch.cuda.synchronize()
        for p, G, A, V in zip(plans, Gs, As, Vs):
            ref = torch.empty_like(V)
            p.degrid(G, A, ref)
            p.synchronize()
            # the same kernel; only the order of the shared-memory adds of the warps' partial sums differs
            d = (V - ref).abs().max().item() / ref.abs().max().item()
            assert d < 1e-6, d
        fp = idg_mod.Plan(obs_list[0], mac_unit=idg_mod.IDG_MAC_FP32)
        try:
            with pytest.raises(idg_mod.IdgError):
                idg_mod.degrid_many([plans[0], fp], Gs[:1] * 2, As[:1] * 2, Vs[:1] * 2)
        finally:
            fp.close()
    finally:
        for p in plans:
            p.close()


def _grid_with(idg_mod, obs, flags, mac, vis, A, shape=None, persistent=False):
    import torch
    plan = idg_mod.Plan(obs, flags=flags | (idg_mod.IDG_PERSISTENT if persistent else 0), mac_unit=mac)
    try:
        G = torch.zeros(shape or plan.grid_shape(), dtype=torch.complex128, device="cuda")
        plan.grid(torch.as_tensor(vis.astype(np.complex64)).cuda(), torch.as_tensor(A).cuda(), G)
        plan.synchronize()
        return G.cpu().numpy()
    finally:
        plan.close()


@pytest.mark.parametrize("persistent", [False, True])
def test_tensor_grid_stokes_i_and_w_layers(idg_mod, oracle_mod, cuda_device, persistent):
    """Stokes-I gridding (plane 0 = (XX + YY) / 2) and w layers with mirrored
    rows, one block per item and the persistent queue."""
    from tests import test_gpu_stokes, test_gpu_wlayers
    obs, A, vis, plan, geom, pl, args = test_gpu_stokes._setup(idg_mod, oracle_mod, seed=7, diagonal="mixed")
    plan.close()
    G = _grid_with(idg_mod, obs, idg_mod.IDG_STOKES_I, idg_mod.IDG_MAC_TENSOR, vis, A, persistent=persistent)
    G_ref = oracle_mod.grid(*args, vis.astype(np.complex64).astype(np.complex128), A.astype(np.complex128))
    assert _rel(G, G_ref) < GRID_TOL
    obs, A, vis, plan, geom, pl, args = test_gpu_wlayers._setup(idg_mod, oracle_mod, seed=3)
    plan.close()
    G = _grid_with(idg_mod, obs, idg_mod.IDG_W_LAYERS, idg_mod.IDG_MAC_TENSOR, vis, A, persistent=persistent)
    G_ref = oracle_mod.grid(*args, vis.astype(np.complex64).astype(np.complex128), A.astype(np.complex128))
    assert _rel(G, G_ref) < GRID_TOL


@pytest.mark.parametrize("case", ["nonuniform", "normalize"])
def test_tensor_plan_keeps_fp32_gridder(idg_mod, oracle_mod, cuda_device, case):
    """Channels not uniformly spaced, or the A-term power normalisation: the
    plan grids with the FP32 kernel (and degrids on the tensor cores)."""
    obs = synth.config(2, n_stations=8, n_timesteps=9, n_channels=11)
    if case == "nonuniform":
        obs.freqs = obs.freqs + np.linspace(0.0, 1.0, obs.n_channels) ** 2 * 2e5
    A, vis = _random_problem(2100, obs, n_int=3)
    flags = idg_mod.IDG_NORMALIZE_ATERM if case == "normalize" else 0
    c = Case(idg_mod, oracle_mod, obs, A, vis, flags=0, mac_unit=idg_mod.IDG_MAC_TENSOR)
    if case == "nonuniform":
        assert _rel(c.gpu_grid(), c.oracle_grid()) < GRID_TOL
    else:
        import torch
        p_t = idg_mod.Plan(obs, flags=flags, mac_unit=idg_mod.IDG_MAC_TENSOR)
        p_f = idg_mod.Plan(obs, flags=flags, mac_unit=idg_mod.IDG_MAC_FP32)
        try:
            Gs = []
            for p in (p_t, p_f):
                G = torch.zeros(p.grid_shape(), dtype=torch.complex128, device="cuda")
                p.grid(c.vis_d, c.A_d, G)
                p.synchronize()
                Gs.append(G)
            assert torch.equal(Gs[0], Gs[1])  # the same FP32 gridder
        finally:
            p_t.close()
            p_f.close()
    Gin = _grand(21, obs.grid_size)
    assert _degrid_err(c.gpu_degrid(Gin), c.oracle_degrid(Gin)) < DEGRID_TOL


def test_tensor_grid_many_equals_single_calls(idg_mod, cuda_device):
    """Tensor-core plans gridded in one shared launch per wave."""
    import torch
    obs_list = [synth.config(2, seed=s, n_stations=6 + 2 * s, n_timesteps=9, n_channels=10 + s) for s in range(3)]
    plans, Vs, Gs, As = [], [], [], []
    for s, obs in enumerate(obs_list):
        rng = np.random.default_rng(60 + s)
        plans.append(idg_mod.Plan(obs, mac_unit=idg_mod.IDG_MAC_TENSOR))
        As.append(torch.as_tensor(synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
                                  .astype(np.complex64)).cuda())
        Vs.append(torch.as_tensor(synth.random_visibilities(rng, obs).astype(np.complex64)).cuda())
        Gs.append(torch.zeros((4, obs.grid_size, obs.grid_size), dtype=torch.complex128, device="cuda"))
    try:
        idg_mod.grid_many(plans, Vs, As, Gs)
        torch.cuda.synchronize()
        for p, V, A, G in zip(plans, Vs, As, Gs):
            ref = torch.zeros_like(G)
            p.grid(V, A, ref)
            p.synchronize()
            err = float(torch.linalg.vector_norm(G - ref) / torch.linalg.vector_norm(ref))
            assert err < 1e-12, err
    finally:
        for p in plans:
            p.close()
