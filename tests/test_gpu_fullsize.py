"""Full-size parity on the MWA-like workload, in the launch configuration
bench.py times (default plan: batches of 1 GiB of subgrid images), and the
mixed-precision report with a 1000-source degrid -> grid round trip.

At full size the oracle checks sampled outputs it can compute one subgrid at
a time (degridded visibilities of a seeded, occupancy-stratified sample of
subgrids), and the full grid element by element on a baseline sample: the
gridder is linear, so gridding the whole observation with every visibility
outside the sampled baselines set to zero (all 8128 baselines planned and
launched, in the bench's batches) gives exactly the grid of the sampled
baselines, which the oracle computes on that sub-observation.  Identities
that hold at any size add the DC invariant, the adjoint identity, and
Stokes-I mode against the four-correlation path."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import parallel, synth
from tests import _brute

pytestmark = pytest.mark.gpu

GRID_TOL = 1e-5
DEGRID_TOL = 1e-5


def _subplan(oracle_mod, full, idx):
    idx = np.sort(np.asarray(idx))
    remap = {int(o): n for n, o in enumerate(idx)}
    keep = np.isin(full.segments[:, 0], idx)
    segs = full.segments[keep].copy()
    segs[:, 0] = [remap[int(s)] for s in segs[:, 0]]
    return oracle_mod.Plan(full.subgrids[idx].copy(), segs)


def _stratified(rng, counts, n):
    """n subgrid indices spread over the occupancy distribution."""
    order = np.argsort(counts, kind="stable")
    picks = [order[int(q)] for q in np.linspace(0, len(order) - 1, n)]
    extra = rng.choice(len(order), size=n // 2, replace=False)
    return np.unique(np.concatenate([picks, extra]))


@pytest.fixture(scope="module")
def mwa_full(idg_mod, oracle_mod, cuda_device):
    import torch
    obs = synth.config(2, seed=0)
    rng = np.random.default_rng(0)
    model = synth.beam_screen_model(rng, rms_rad=2.0)
    A = synth.aterms_beam_screen(obs, model)
    vis = synth.random_visibilities(rng, obs)
    plan = idg_mod.Plan(obs)
    geom = oracle_mod.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size)
    ref_plan = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    yield dict(obs=obs, A=A, vis=vis, plan=plan, geom=geom, ref_plan=ref_plan,
               A_d=torch.as_tensor(A).cuda(), vis_d=torch.as_tensor(vis).cuda())
    plan.close()


def test_full_size_plan_is_bit_exact(mwa_full):
    np.testing.assert_array_equal(mwa_full["plan"].subgrids(), mwa_full["ref_plan"].subgrids)
    np.testing.assert_array_equal(mwa_full["plan"].segments(), mwa_full["ref_plan"].segments)
    st = mwa_full["plan"].stats()
    assert st.n_batches > 1 and st.n_subgrids == mwa_full["ref_plan"].subgrids.shape[0]


def test_full_size_degrid_sampled_subgrids(mwa_full, oracle_mod):
    import torch
    obs, plan = mwa_full["obs"], mwa_full["plan"]
    N = obs.grid_size
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    G_d = torch.randn((4, N, N), dtype=torch.complex128, device="cuda", generator=g)
    V_d = torch.empty_like(mwa_full["vis_d"])
    plan.degrid(G_d, mwa_full["A_d"], V_d)
    plan.synchronize()
    V = V_d.cpu().numpy()
    G = G_d.cpu().numpy()
    full = mwa_full["ref_plan"]
    counts = (full.subgrids[:, 2] - full.subgrids[:, 1]) * (full.subgrids[:, 4] - full.subgrids[:, 3])
    idx = _stratified(np.random.default_rng(11), counts, 16)
    sub = _subplan(oracle_mod, full, idx)
    V_ref = oracle_mod.degrid(mwa_full["geom"], obs.n_stations, obs.baselines, obs.uvw, obs.freqs,
                              obs.aterm_offsets, sub, G, mwa_full["A"].astype(np.complex128))
    mask = np.zeros(V.shape[:3], bool)
    for b, t0, t1, c0, c1, *_ in full.subgrids[idx]:
        mask[b, t0:t1, c0:c1] = True
    got, ref = V[mask], V_ref[mask]
    err = np.sqrt(np.mean(np.abs(got - ref) ** 2)) / np.abs(ref).max()
    assert err < DEGRID_TOL, err


def _baseline_sample(full, n=16, seed=21):
    """Baselines of an occupancy-stratified seeded sample of subgrids."""
    counts = (full.subgrids[:, 2] - full.subgrids[:, 1]) * (full.subgrids[:, 4] - full.subgrids[:, 3])
    idx = _stratified(np.random.default_rng(seed), counts, n)
    return np.unique(full.subgrids[idx, 0])


def _grid_of_baselines(plan, vis_d, A_d, bls, N):
    """Full-size grid of the whole plan with the visibilities of every baseline
    outside `bls` zeroed: by linearity, the grid of `bls` alone."""
    import torch
    keep = torch.zeros(vis_d.shape[0], dtype=torch.bool, device=vis_d.device)
    keep[torch.as_tensor(bls, device=vis_d.device)] = True
    vis_s = torch.where(keep[:, None, None, None], vis_d, torch.zeros((), dtype=vis_d.dtype, device=vis_d.device))
    G_d = torch.zeros((4, N, N), dtype=torch.complex128, device=vis_d.device)
    plan.grid(vis_s, A_d, G_d)
    plan.synchronize()
    return G_d


def test_full_size_grid_of_sampled_baselines_elementwise(mwa_full, oracle_mod):
    """Element-wise grid parity at full size: the whole MWA-like plan in the
    bench's launch configuration, visibilities kept on a stratified sample
    of baselines (short to long), against the oracle's grid of those
    baselines over all 4 x 4096^2 cells."""
    obs, plan = mwa_full["obs"], mwa_full["plan"]
    N = obs.grid_size
    bls = _baseline_sample(mwa_full["ref_plan"])
    assert len(bls) >= 8
    G = _grid_of_baselines(plan, mwa_full["vis_d"], mwa_full["A_d"], bls, N).cpu().numpy()
    sub = parallel.sub_observation(obs, bls)
    ref_plan = oracle_mod.plan(mwa_full["geom"], sub.uvw, obs.freqs, obs.aterm_offsets)
    G_ref = oracle_mod.grid(mwa_full["geom"], obs.n_stations, sub.baselines, sub.uvw, obs.freqs, obs.aterm_offsets,
                            ref_plan, mwa_full["vis"][bls].astype(np.complex128), mwa_full["A"].astype(np.complex128))
    err = float(np.linalg.norm((G - G_ref).ravel()) / np.linalg.norm(G_ref.ravel()))
    print(f"full-size grid of {len(bls)} sampled baselines: relative L2 {err:.2e}")
    assert err < GRID_TOL, err
    # nothing leaks outside the sampled baselines' footprints
    assert np.count_nonzero(G_ref) == np.count_nonzero(G)


def test_full_size_grid_fp32_gridder_sampled_baselines(mwa_full, idg_mod, oracle_mod):
    """The same element-wise check with the FP32-pipe gridder (mac_unit =
    IDG_MAC_TENSOR_DEGRID) gridding the whole plan; the library's default
    plan above grids on the tensor cores."""
    obs = mwa_full["obs"]
    N = obs.grid_size
    assert mwa_full["plan"].stats().mac_unit == idg_mod.IDG_MAC_TENSOR
    plan = idg_mod.Plan(obs, mac_unit=idg_mod.IDG_MAC_TENSOR_DEGRID)
    try:
        assert plan.stats().mac_unit == idg_mod.IDG_MAC_TENSOR_DEGRID
        bls = _baseline_sample(mwa_full["ref_plan"], seed=23)
        G = _grid_of_baselines(plan, mwa_full["vis_d"], mwa_full["A_d"], bls, N).cpu().numpy()
    finally:
        plan.close()
    sub = parallel.sub_observation(obs, bls)
    ref_plan = oracle_mod.plan(mwa_full["geom"], sub.uvw, obs.freqs, obs.aterm_offsets)
    G_ref = oracle_mod.grid(mwa_full["geom"], obs.n_stations, sub.baselines, sub.uvw, obs.freqs, obs.aterm_offsets,
                            ref_plan, mwa_full["vis"][bls].astype(np.complex128), mwa_full["A"].astype(np.complex128))
    err = float(np.linalg.norm((G - G_ref).ravel()) / np.linalg.norm(G_ref.ravel()))
    print(f"full-size FP32-gridder grid of {len(bls)} sampled baselines: relative L2 {err:.2e}")
    assert err < GRID_TOL, err


def test_full_size_grid_identities(mwa_full):
    """DC invariant and adjoint identity on the full MWA-like workload."""
    import torch
    obs, plan, A = mwa_full["obs"], mwa_full["plan"], mwa_full["A"]
    N, L = obs.grid_size, obs.subgrid_size
    G_d = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
    plan.grid(mwa_full["vis_d"], mwa_full["A_d"], G_d)
    plan.synchronize()
    # DC invariant: sum G = L^2 T(0)^2 sum_seg A_p(0)^H (sum V) A_q(0), T(0) = 1
    vis = mwa_full["vis"].astype(np.complex128)
    full = mwa_full["ref_plan"]
    c = obs.aterm_nodes // 2
    Ac = A[:, :, c, c].astype(np.complex128).reshape(A.shape[0], A.shape[1], 2, 2)
    # per (baseline, timestep) sums over channel ranges via cumulative sums
    csum = np.concatenate([np.zeros(vis.shape[:2] + (1, 4), complex), np.cumsum(vis, axis=2)], axis=2)
    want = np.zeros((2, 2), complex)
    for (s, a, tb, te) in full.segments:
        b, _, _, c0, c1 = full.subgrids[s, :5]
        S = (csum[b, tb:te, c1] - csum[b, tb:te, c0]).sum(axis=0).reshape(2, 2)
        p, q = obs.baselines[b]
        want += Ac[a, p].conj().T @ S @ Ac[a, q]
    got = G_d.sum(dim=(1, 2)).cpu().numpy().reshape(2, 2)
    assert np.abs(got - L * L * want).max() / np.abs(L * L * want).max() < GRID_TOL
    # adjoint identity with a random grid
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    R = torch.randn((4, N, N), dtype=torch.complex128, device="cuda", generator=g)
    V_d = torch.empty_like(mwa_full["vis_d"])
    plan.degrid(R, mwa_full["A_d"], V_d)
    plan.synchronize()
    lhs = torch.vdot(V_d.reshape(-1).to(torch.complex128), mwa_full["vis_d"].reshape(-1).to(torch.complex128))
    rhs = torch.vdot(R.reshape(-1), G_d.reshape(-1))
    assert abs(complex(lhs) - complex(rhs)) / abs(complex(rhs)) < GRID_TOL


def test_full_size_stokes_i_against_four_correlations(mwa_full, idg_mod):
    """Stokes-I mode (one grid plane) on the full workload, against the
    four-correlation path of the same observation through identities that
    hold at any size: the I grid is (G_XX + G_YY)/2 of the four-plane grid
    (subgrid FFT and adder are linear), and the visibilities predicted from a
    model I plane equal the four-plane prediction of the model XX = YY = I,
    XY = YX = 0; the beam x screen A-terms are diagonal, so the predicted XY
    and YX are exactly zero."""
    import torch
    obs, A_d, vis_d = mwa_full["obs"], mwa_full["A_d"], mwa_full["vis_d"]
    N = obs.grid_size
    plan4 = mwa_full["plan"]
    plan1 = idg_mod.Plan(obs, flags=idg_mod.IDG_STOKES_I)
    try:
        assert plan1.grid_shape() == (1, N, N)
        G4 = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
        plan4.grid(vis_d, A_d, G4)
        plan4.synchronize()
        GI = torch.zeros((1, N, N), dtype=torch.complex128, device="cuda")
        plan1.grid(vis_d, A_d, GI)
        plan1.synchronize()
        want = 0.5 * (G4[0] + G4[3])
        err = float(torch.linalg.vector_norm(GI[0] - want) / torch.linalg.vector_norm(want))
        assert err < GRID_TOL, err
        del G4, GI, want
        g = torch.Generator(device="cuda")
        g.manual_seed(13)
        I = torch.randn((1, N, N), dtype=torch.complex128, device="cuda", generator=g)
        Gm = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
        Gm[0] = I[0]
        Gm[3] = I[0]
        V4 = torch.empty_like(vis_d)
        VI = torch.empty_like(vis_d)
        plan4.degrid(Gm, A_d, V4)
        plan4.synchronize()
        plan1.degrid(I, A_d, VI)
        plan1.synchronize()
        d = (VI - V4).to(torch.complex128)
        err = float(torch.sqrt(torch.mean(d.abs() ** 2)) / V4.abs().max())
        assert err < DEGRID_TOL, err
        assert not bool(VI[..., 1:3].any())
    finally:
        plan1.close()


def _model_grid(obs, sky, beta):
    """Model grid of a point-source sky divided by the taper:
    sum_s S_s / (T(l) T(m)) e^{-2 pi i (u l + v m)} in XX and YY."""
    import scipy.special
    N, fov = obs.grid_size, obs.image_size
    T = lambda x: scipy.special.i0(beta * np.sqrt(1 - (2 * x / fov) ** 2)) / scipy.special.i0(beta)
    u = (np.arange(N) - N // 2) / fov
    ex = np.exp(-2j * np.pi * np.outer(u, sky.l))
    ey = np.exp(-2j * np.pi * np.outer(u, sky.m))
    G = np.zeros((4, N, N), complex)
    G[0] = (ey * (sky.flux / (T(sky.l) * T(sky.m)))) @ ex.T
    G[3] = G[0]
    return G


def _round_trip_full_array(idg_mod, oracle_mod, obs, A, G_model, beta):
    """Workload 3 on the whole array: degrid the model (every visibility),
    grid the result; errors against the oracle on a stratified sample of
    baselines (degrid: those baselines' visibilities; grid: the full-size grid
    of the GPU visibilities kept on those baselines, by linearity)."""
    import torch
    N, L = obs.grid_size, obs.subgrid_size
    plan = idg_mod.Plan(obs, taper_beta=beta)
    try:
        geom = oracle_mod.Geometry(N, L, obs.kernel_padding, obs.image_size, taper_beta=beta)
        full = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
        bls = _baseline_sample(full, seed=33)
        sub = parallel.sub_observation(obs, bls)
        sub_plan = oracle_mod.plan(geom, sub.uvw, obs.freqs, obs.aterm_offsets)
        A_d = torch.as_tensor(A).cuda()
        V_d = torch.empty((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64,
                          device="cuda")
        plan.degrid(torch.as_tensor(G_model).cuda(), A_d, V_d)
        plan.synchronize()
        G = _grid_of_baselines(plan, V_d, A_d, bls, N).cpu().numpy()
        V_s = V_d[torch.as_tensor(bls, device="cuda")].cpu().numpy()
        args = (geom, obs.n_stations, sub.baselines, sub.uvw, obs.freqs, obs.aterm_offsets, sub_plan)
        V_ref = oracle_mod.degrid(*args, G_model, A.astype(np.complex128))
        G_ref = oracle_mod.grid(*args, V_s.astype(np.complex128), A.astype(np.complex128))
        deg_err = float(np.sqrt(np.mean(np.abs(V_s - V_ref) ** 2)) / np.abs(V_ref).max())
        grid_err = float(np.linalg.norm((G - G_ref).ravel()) / np.linalg.norm(G_ref.ravel()))
        return deg_err, grid_err, len(bls)
    finally:
        plan.close()


def test_mixed_precision_round_trip_full_array(idg_mod, oracle_mod, cuda_device):
    """Workload 3 at full size (128 stations, 10.9 M visibilities, 4096^2):
    FP32 phasors with FP64 subgrid offsets against the FP64 oracle on a
    1000-source model, model grid -> degrid -> grid, in the bench's launch
    configuration.  Asserted at the default taper beta = 0.35 pi P; the
    same round trip at beta = pi P / 2 is recorded (printed), not asserted:
    the model divided by that steeper taper carries a dynamic range 1/T^2
    about 60 times larger, which FP32 phasor sums pass on as error."""
    obs = synth.config(3, seed=0)
    assert obs.n_stations == 128 and obs.n_vis == 10924032
    rng = np.random.default_rng(3)
    model = synth.beam_screen_model(rng, rms_rad=2.0)
    A = synth.aterms_beam_screen(obs, model)
    sky = synth.point_sources(rng, 1000, 0.16)
    results = {}
    for name, beta in (("0.35 pi P", 0.35 * np.pi * obs.kernel_padding), ("pi P / 2", 0.5 * np.pi * obs.kernel_padding)):
        G_model = _model_grid(obs, sky, beta)
        results[name] = _round_trip_full_array(idg_mod, oracle_mod, obs, A, G_model, beta)
        d, g, nb = results[name]
        print(f"mixed precision, full array, beta = {name}: degrid rms/peak {d:.2e}, grid rel {g:.2e} "
              f"({nb} sampled baselines)")
    d, g, _ = results["0.35 pi P"]
    assert d < DEGRID_TOL and g < GRID_TOL, results


def test_mixed_precision_round_trip(idg_mod, oracle_mod, cuda_device):
    """Workload 3 on 16 of its stations, every output compared: FP32 phasors
    with FP64 subgrid offsets against the FP64 oracle, on a 1000-source
    model: model grid -> degrid -> grid."""
    import torch
    obs = synth.config(3, seed=0, n_stations=16)
    rng = np.random.default_rng(3)
    model = synth.beam_screen_model(rng, rms_rad=2.0)
    A = synth.aterms_beam_screen(obs, model)
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    sky = synth.point_sources(rng, 1000, 0.16)
    # model image / T transformed to the grid: sum_s S_s/(T(l)T(m)) e^{-2 pi i (u l + v m)}
    beta = oracle_mod.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size).beta
    import scipy.special
    T = lambda x: scipy.special.i0(beta * np.sqrt(1 - (2 * x / fov) ** 2)) / scipy.special.i0(beta)
    u = (np.arange(N) - N // 2) / fov
    ex = np.exp(-2j * np.pi * np.outer(u, sky.l))
    ey = np.exp(-2j * np.pi * np.outer(u, sky.m))
    G_model = np.zeros((4, N, N), complex)
    w = sky.flux / (T(sky.l) * T(sky.m))
    G_model[0] = (ey * w) @ ex.T
    G_model[3] = G_model[0]
    plan = idg_mod.Plan(obs)
    geom = oracle_mod.Geometry(obs.grid_size, L, obs.kernel_padding, fov)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    args = (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)
    A_d = torch.as_tensor(A).cuda()
    V_d = torch.empty((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64, device="cuda")
    plan.degrid(torch.as_tensor(G_model).cuda(), A_d, V_d)
    G_d = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
    plan.grid(V_d, A_d, G_d)
    plan.synchronize()
    V_gpu, G_gpu = V_d.cpu().numpy(), G_d.cpu().numpy()
    V_ref = oracle_mod.degrid(*args, G_model, A.astype(np.complex128))
    G_ref = oracle_mod.grid(*args, V_gpu.astype(np.complex128), A.astype(np.complex128))
    deg_err = np.sqrt(np.mean(np.abs(V_gpu - V_ref) ** 2)) / np.abs(V_ref).max()
    grid_err = np.linalg.norm(G_gpu - G_ref) / np.linalg.norm(G_ref)
    print(f"mixed precision: degrid rms/peak {deg_err:.2e}, grid rel {grid_err:.2e}")
    assert deg_err < DEGRID_TOL and grid_err < GRID_TOL
    plan.close()
