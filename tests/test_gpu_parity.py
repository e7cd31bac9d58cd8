"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (FP32 path against the FP64 oracle):
  gridder   ||G_gpu - G_oracle||_2 / ||G_oracle||_2 <= 1e-5 over all 4 planes
  degridder rms_k |V_gpu - V_oracle| / max_k |V_oracle| <= 1e-5
  plans     bit-exact
"""
import numpy as np
import pytest

from paper_2502_17789_gb300 import synth
from tests import _brute

pytestmark = pytest.mark.gpu

GRID_TOL = 1e-5
DEGRID_TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _degrid_err(v, ref):
    return float(np.sqrt(np.mean(np.abs(v - ref) ** 2)) / np.abs(ref).max())


def _oracle_geom(oracle_mod, obs, L, flags):
    f = 0
    if flags & 1:
        f |= oracle_mod.FLAG_DROP
    if flags & 2:
        f |= oracle_mod.FLAG_SPLIT_INTERVALS
    return oracle_mod.Geometry(obs.grid_size, L, obs.kernel_padding, obs.image_size, aterm_nodes=obs.aterm_nodes,
                               flags=f)


class Case:
    def __init__(self, idg_mod, oracle_mod, obs, A, vis, L=None, flags=0, degrid_channels=0, mac_unit=0):
        import torch
        self.obs, self.L = obs, L or obs.subgrid_size
        self.plan = idg_mod.Plan(obs, subgrid_size=self.L, flags=flags, degrid_channels=degrid_channels,
                                 mac_unit=mac_unit)
        self.geom = _oracle_geom(oracle_mod, obs, self.L, flags)
        self.ref_plan = oracle_mod.plan(self.geom, obs.uvw, obs.freqs, obs.aterm_offsets)
        np.testing.assert_array_equal(self.plan.subgrids(), self.ref_plan.subgrids)
        np.testing.assert_array_equal(self.plan.segments(), self.ref_plan.segments)
        self.A = A.astype(np.complex64)
        self.vis = vis.astype(np.complex64)
        self.A_d = torch.as_tensor(self.A).cuda()
        self.vis_d = torch.as_tensor(self.vis).cuda()
        self.oracle = oracle_mod

    def args(self):
        o = self.obs
        return (self.geom, o.n_stations, o.baselines, o.uvw, o.freqs, o.aterm_offsets, self.ref_plan)

    def gpu_grid(self, base=None):
        import torch
        N = self.obs.grid_size
        G = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda") if base is None else \
            torch.as_tensor(base).cuda()
        self.plan.grid(self.vis_d, self.A_d, G)
        self.plan.synchronize()
        return G.cpu().numpy()

    def gpu_degrid(self, G):
        import torch
        out = torch.full(self.vis.shape, 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
        self.plan.degrid(torch.as_tensor(G).cuda(), self.A_d, out)
        self.plan.synchronize()
        return out.cpu().numpy()

    def oracle_grid(self, **kw):
        return self.oracle.grid(*self.args(), self.vis.astype(np.complex128), self.A.astype(np.complex128), **kw)

    def oracle_degrid(self, G):
        return self.oracle.degrid(*self.args(), G, self.A.astype(np.complex128))


def _random_problem(seed, obs, n_int=None, identity=False):
    rng = np.random.default_rng(seed)
    if n_int is not None:
        steps = max(1, obs.n_timesteps // n_int)
        obs.aterm_offsets = np.array(sorted(set(list(range(0, obs.n_timesteps, steps)) + [obs.n_timesteps])), np.int32)
    A = synth.aterms_identity(obs.n_intervals, obs.n_stations) if identity else \
        synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    vis = synth.random_visibilities(rng, obs)
    return A, vis


# ------------------------------------------------------------------ stage parity

@pytest.mark.parametrize("mac", ["default", "fp32_gridder"])
@pytest.mark.parametrize("L", [32, 64, 96, 128])
def test_subgrid_images_match_oracle(idg_mod, oracle_mod, cuda_device, L, mac):
    """Gridder output per subgrid, before (stage 0) and after (stage 1) the
    FFT, with the default (tensor-core) gridder and the FP32-pipe one."""
    obs = synth.config(2, n_stations=6, n_timesteps=9, n_channels=11)
    A, vis = _random_problem(L, obs, n_int=3)
    c = Case(idg_mod, oracle_mod, obs, A, vis, L=L,
             mac_unit=idg_mod.IDG_MAC_TENSOR_DEGRID if mac == "fp32_gridder" else 0)
    _, img, uv = c.oracle_grid(want_subgrids=True)
    import torch
    for stage, ref in ((0, img), (1, uv)):
        got = c.plan.subgrid_images(c.vis_d, c.A_d, stage)
        c.plan.synchronize()
        got = got.cpu().numpy()
        assert _rel(got, ref) < GRID_TOL, (stage, _rel(got, ref))


# ------------------------------------------------------------------ grid / degrid parity

def test_small_workload_full_grid_and_degrid(idg_mod, oracle_mod, cuda_device):
    """Workload 1 at full size: 32 stations, 16 x 8 s, 8 channels, 512^2 grid,
    L = 32, identity A-terms, point-source sky plus noise."""
    obs = synth.config(1, seed=0)
    rng = np.random.default_rng(0)
    sky = synth.point_sources(rng, 20, 0.0873)
    vis = synth.simulate_visibilities(obs, sky, noise_sigma=0.1, rng=rng)
    A = synth.aterms_identity(obs.n_intervals, obs.n_stations)
    c = Case(idg_mod, oracle_mod, obs, A, vis)
    G_ref = c.oracle_grid()
    G = c.gpu_grid()
    assert _rel(G, G_ref) < GRID_TOL
    V_ref = c.oracle_degrid(G_ref)
    V = c.gpu_degrid(G_ref)
    assert _degrid_err(V, V_ref) < DEGRID_TOL


@pytest.mark.parametrize("mac", ["default", "fp32_gridder"])
@pytest.mark.parametrize("L,split", [(32, False), (64, True), (96, False), (96, True), (128, False)])
def test_reduced_mwa_like_random_aterms(idg_mod, oracle_mod, cuda_device, L, split, mac):
    """Random full-Jones A-terms, several intervals, ragged chunk tails; the
    default (tensor-core) kernels and the FP32-pipe gridder."""
    obs = synth.config(2, n_stations=10, n_timesteps=13, n_channels=17)
    A, vis = _random_problem(100 + L, obs, n_int=4)
    c = Case(idg_mod, oracle_mod, obs, A, vis, L=L, flags=2 if split else 0,
             mac_unit=idg_mod.IDG_MAC_TENSOR_DEGRID if mac == "fp32_gridder" else 0)
    G_ref = c.oracle_grid()
    assert _rel(c.gpu_grid(), G_ref) < GRID_TOL
    rng = np.random.default_rng(L)
    N = obs.grid_size
    Grand = (rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))) * 1e-3
    for Gin in (G_ref, Grand):
        V_ref = c.oracle_degrid(Gin)
        assert _degrid_err(c.gpu_degrid(Gin), V_ref) < DEGRID_TOL


@pytest.mark.parametrize("channels", [1, 2, 4])
@pytest.mark.parametrize("L,n_ch", [(32, 17), (64, 7), (96, 24), (128, 13)])
def test_degrid_channel_groups(idg_mod, oracle_mod, cuda_device, channels, L, n_ch):
    """Degridder lanes of 1, 2 or 4 channels (the first by sine and cosine,
    the rest by rotation with the channel-step phasor): ragged and balanced
    groups (17 channels in groups of 4 are 5 groups of 3 or 4), two segments
    per work item, one block per item and the persistent queue."""
    import torch
    obs = synth.config(2, n_stations=8, n_timesteps=11, n_channels=n_ch)
    A, vis = _random_problem(900 + L + n_ch, obs, n_int=3)
    rng = np.random.default_rng(L)
    N = obs.grid_size
    Grand = (rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))) * 1e-3
    c = Case(idg_mod, oracle_mod, obs, A, vis, L=L, degrid_channels=channels, mac_unit=idg_mod.IDG_MAC_FP32)
    assert c.plan.stats().degrid_channels == channels
    V_ref = c.oracle_degrid(Grand)
    assert _degrid_err(c.gpu_degrid(Grand), V_ref) < DEGRID_TOL
    pp = idg_mod.Plan(obs, subgrid_size=L, flags=idg_mod.IDG_PERSISTENT, degrid_channels=channels,
                      mac_unit=idg_mod.IDG_MAC_FP32)
    try:
        V = torch.full(c.vis.shape, 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
        pp.degrid(torch.as_tensor(Grand).cuda(), c.A_d, V)
        pp.synchronize()
        assert _degrid_err(V.cpu().numpy(), V_ref) < DEGRID_TOL
    finally:
        pp.close()


@pytest.mark.parametrize("channels", [1, 2, 4])
@pytest.mark.parametrize("n_ch,n_t,steps", [(1, 1, 1), (1, 3, 1), (2, 2, 1), (3, 3, 3), (5, 4, 2), (4, 8, 4)])
def test_degrid_low_occupancy(idg_mod, oracle_mod, cuda_device, channels, n_ch, n_t, steps):
    """Work items of few lanes (1 to 16: subgrids of a few visibilities,
    Section 3.2) spread each visibility's pixels over R = 32 / 2^ceil(log2
    lanes) lanes of a warp and add the partial sums with shuffles; one or
    two segments per item."""
    obs = synth.config(2, n_stations=9, n_timesteps=n_t, n_channels=n_ch)
    obs.aterm_offsets = np.array(list(range(0, n_t, steps)) + [n_t], np.int32)
    A, vis = _random_problem(700 + 10 * n_ch + n_t, obs)
    rng = np.random.default_rng(n_ch * n_t)
    N = obs.grid_size
    Grand = (rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))) * 1e-3
    c = Case(idg_mod, oracle_mod, obs, A, vis, degrid_channels=channels, mac_unit=idg_mod.IDG_MAC_FP32)
    V_ref = c.oracle_degrid(Grand)
    assert _degrid_err(c.gpu_degrid(Grand), V_ref) < DEGRID_TOL
    assert _rel(c.gpu_grid(), c.oracle_grid()) < GRID_TOL


@pytest.mark.parametrize("chunk", [32, 64])
def test_grid_chunk_sizes(idg_mod, oracle_mod, cuda_device, chunk):
    """Gridder record chunks other than the default (the autotuner's choice):
    chunks that end inside a segment, ragged chunk tails, one block per item
    and the persistent queue."""
    import torch
    obs = synth.config(2, n_stations=10, n_timesteps=13, n_channels=17)
    A, vis = _random_problem(400 + chunk, obs, n_int=4)
    G_ref = oracle_mod.grid(*Case(idg_mod, oracle_mod, obs, A, vis).args(), vis.astype(np.complex64).astype(np.complex128),
                            A.astype(np.complex64).astype(np.complex128))
    for flags in (0, idg_mod.IDG_PERSISTENT):
        plan = idg_mod.Plan(obs, flags=flags, grid_chunk=chunk, mac_unit=idg_mod.IDG_MAC_TENSOR_DEGRID)
        try:
            assert plan.stats().grid_chunk == chunk
            G = torch.zeros((4, obs.grid_size, obs.grid_size), dtype=torch.complex128, device="cuda")
            plan.grid(torch.as_tensor(vis.astype(np.complex64)).cuda(), torch.as_tensor(A.astype(np.complex64)).cuda(), G)
            plan.synchronize()
            assert _rel(G.cpu().numpy(), G_ref) < GRID_TOL
        finally:
            plan.close()


def test_grid_accumulates_into_existing_grid(idg_mod, oracle_mod, cuda_device):
    obs = synth.config(1, n_stations=8)
    A, vis = _random_problem(3, obs, n_int=2)
    c = Case(idg_mod, oracle_mod, obs, A, vis)
    rng = np.random.default_rng(1)
    N = obs.grid_size
    base = rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))
    G = c.gpu_grid(base)
    G_ref = c.oracle_grid()
    assert _rel(G - base, G_ref) < GRID_TOL


def test_dropped_subgrids(idg_mod, oracle_mod, cuda_device):
    obs = _brute.tiny_observation(seed=4, n_st=8, N=128, L=32, P=12, fov=0.3)
    u, v, _ = _brute.uvw_lambda(obs)
    reach = np.abs(np.stack([u, v])).max(axis=(0, 2, 3)) * obs.image_size
    obs.uvw = obs.uvw * (1.2 * (obs.grid_size / 2 - obs.subgrid_size / 2) / np.median(reach))
    obs.uvw[..., 2] = 0.0
    A, vis = _random_problem(9, obs)
    c = Case(idg_mod, oracle_mod, obs, A, vis, flags=1)
    assert c.plan.stats().n_subgrids_dropped > 0
    G_ref = c.oracle_grid()
    assert _rel(c.gpu_grid(), G_ref) < GRID_TOL
    V = c.gpu_degrid(G_ref)
    V_ref = c.oracle_degrid(G_ref)
    assert _degrid_err(V, V_ref) < DEGRID_TOL
    dropped = np.zeros(V.shape[:3], bool)
    for row in c.ref_plan.subgrids:
        if row[7]:
            dropped[row[0], row[1]:row[2], row[3]:row[4]] = True
    assert np.all(V[dropped] == 0)


def test_single_visibility_and_empty(idg_mod, oracle_mod, cuda_device):
    import torch
    obs = _brute.tiny_observation(seed=2, n_st=2, n_t=1, n_ch=1, N=64, L=32, P=12, fov=0.3)
    A, vis = _random_problem(5, obs)
    c = Case(idg_mod, oracle_mod, obs, A, vis)
    assert _rel(c.gpu_grid(), c.oracle_grid()) < GRID_TOL
    empty = _brute.tiny_observation(seed=2, n_st=3, n_t=0, N=64, L=32, P=12, fov=0.3)
    plan = idg_mod.Plan(empty)
    G = torch.ones((4, 64, 64), dtype=torch.complex128, device="cuda")
    v = torch.zeros((3, 0, 4, 4), dtype=torch.complex64, device="cuda")
    Aq = torch.as_tensor(synth.aterms_identity(1, 3)).cuda()
    vbuf = torch.zeros(16, dtype=torch.complex64, device="cuda")  # a valid pointer for a zero-size array
    plan.grid(vbuf, Aq, G)
    plan.degrid(G, Aq, vbuf)
    torch.cuda.synchronize()
    assert torch.all(G == 1)
    del v


def test_adjoint_identity_gpu(idg_mod, oracle_mod, cuda_device):
    obs = synth.config(2, n_stations=12, n_timesteps=10, n_channels=24)
    A, vis = _random_problem(21, obs, n_int=3)
    c = Case(idg_mod, oracle_mod, obs, A, vis)
    rng = np.random.default_rng(2)
    N = obs.grid_size
    G = rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))
    lhs = np.vdot(c.gpu_degrid(G).astype(np.complex128), vis.astype(np.complex128))
    rhs = np.vdot(G, c.gpu_grid())
    assert abs(lhs - rhs) / abs(rhs) < 1e-5


def test_invalid_arguments_return_status(idg_mod, cuda_device):
    import ctypes
    obs = synth.config(1, n_stations=4)
    plan = idg_mod.Plan(obs)
    lib = idg_mod.load()
    assert lib.idg_grid(plan.handle, None, None, None) == 1
    assert lib.idg_degrid(None, None, None, None) == 1
    assert "NULL" in idg_mod.idg_last_error(None)
    assert lib.idg_subgrid_images(plan.handle, ctypes.c_void_p(16), ctypes.c_void_p(16), 5, ctypes.c_void_p(16)) == 1


def test_persistent_queue_and_graph_replay(idg_mod, oracle_mod, cuda_device):
    """The batched forms (persistent work-queue launches, CUDA-graph replay of
    a whole call) give the oracle's result, on a plan with several batches."""
    import os
    import torch
    obs = synth.config(2, n_stations=14, n_timesteps=16, n_channels=24)
    A, vis = _random_problem(31, obs, n_int=4)
    os.environ["IDG_SCRATCH_BYTES"] = str(64 * 4 * 96 * 96 * 8)  # 64 subgrids per batch
    try:
        c = Case(idg_mod, oracle_mod, obs, A, vis)
        stream = torch.cuda.Stream()
        pp = idg_mod.Plan(obs, flags=idg_mod.IDG_PERSISTENT, stream=stream.cuda_stream)
    finally:
        del os.environ["IDG_SCRATCH_BYTES"]
    assert pp.stats().n_batches > 1
    G_ref = c.oracle_grid()
    N = obs.grid_size
    rng = np.random.default_rng(3)
    Gin = rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))
    V_ref = c.oracle_degrid(Gin)
    Gin_d = torch.as_tensor(Gin).cuda()
    with torch.cuda.stream(stream):
        for use_graph in (False, True, True):
            G = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
            V = torch.full(vis.shape, 7.0, dtype=torch.complex64, device="cuda")
            if use_graph:
                pp.grid_graph(c.vis_d, c.A_d, G)
                pp.degrid_graph(Gin_d, c.A_d, V)
            else:
                pp.grid(c.vis_d, c.A_d, G)
                pp.degrid(Gin_d, c.A_d, V)
            pp.synchronize()
            assert _rel(G.cpu().numpy(), G_ref) < GRID_TOL
            assert _degrid_err(V.cpu().numpy(), V_ref) < DEGRID_TOL
        # graph replay with the same buffers accumulates again into G
        pp.grid_graph(c.vis_d, c.A_d, G)
        pp.synchronize()
        assert _rel(G.cpu().numpy(), 2 * G_ref) < GRID_TOL
    pp.close()


def test_graph_needs_a_stream(idg_mod, cuda_device):
    import torch
    obs = synth.config(1, n_stations=4)
    plan = idg_mod.Plan(obs, stream=0)
    v = torch.zeros((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), dtype=torch.complex64, device="cuda")
    A = torch.as_tensor(synth.aterms_identity(1, obs.n_stations)).cuda()
    G = torch.zeros((4, obs.grid_size, obs.grid_size), dtype=torch.complex128, device="cuda")
    with pytest.raises(idg_mod.IdgError) as e:
        plan.grid_graph(v, A, G)
    assert e.value.status == 1


@pytest.mark.parametrize("L", [64, 96])
def test_diagonal_and_mixed_aterms(idg_mod, oracle_mod, cuda_device, L):
    """A-terms whose off-diagonal entries are all zero take the diagonal
    epilogue (Section 3.3 with diagonal Jones matrices); stations and intervals
    that mix diagonal and full Jones matrices must give the same result as the
    full product."""
    obs = synth.config(2, n_stations=9, n_timesteps=12, n_channels=13)
    A, vis = _random_problem(300 + L, obs, n_int=3)
    A[..., 1] = 0
    A[..., 2] = 0
    N = obs.grid_size
    rng = np.random.default_rng(L)
    Grand = (rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))) * 1e-3
    mixed = A.copy()
    full = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    mixed[0, ::2] = full[0, ::2]          # interval 0: even stations full Jones
    mixed[2, 4] = full[2, 4]              # one station of interval 2
    mixed[1, 3, 4, 4, 1] = 1e-3           # a single off-diagonal node entry
    for Acase in (A, mixed):
        c = Case(idg_mod, oracle_mod, obs, Acase, vis, L=L)
        assert _rel(c.gpu_grid(), c.oracle_grid()) < GRID_TOL
        assert _degrid_err(c.gpu_degrid(Grand), c.oracle_degrid(Grand)) < DEGRID_TOL


@pytest.mark.parametrize("spacing", ["random", "uniform_then_jump", "single"])
def test_channel_spacing(idg_mod, oracle_mod, cuda_device, spacing):
    """The gridder rotates phasors along runs of channels with a constant
    frequency step (phi is linear in frequency, Eq. 7); non-uniform steps,
    a change of step within a row and single-channel rows must take the
    direct evaluation and still match the oracle."""
    rng = np.random.default_rng(11)
    enu = synth.stations_uniform_disk(rng, 9, 3000.0)
    if spacing == "random":
        freqs = 140e6 + np.cumsum(rng.uniform(0.8e6, 1.6e6, 19))
    elif spacing == "uniform_then_jump":
        freqs = np.concatenate([140e6 + 1.25e6 * np.arange(11), 160e6 + 0.9e6 * np.arange(9)])
    else:
        freqs = np.array([150e6])
    obs = synth.make_observation(enu, 12, 2.0, freqs, 4, 4096, 96, 18, 0.5, name="spacing")
    A, vis = _random_problem(5, obs)
    N = obs.grid_size
    Grand = (rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))) * 1e-3
    c = Case(idg_mod, oracle_mod, obs, A, vis)
    # the degridder's channel groups need one frequency step along the band
    assert c.plan.stats().degrid_channels == 1
    c4 = idg_mod.Plan(obs, degrid_channels=4)
    assert c4.stats().degrid_channels == (1 if spacing != "single" else 4)
    c4.close()
    assert _rel(c.gpu_grid(), c.oracle_grid()) < GRID_TOL
    assert _degrid_err(c.gpu_degrid(Grand), c.oracle_degrid(Grand)) < DEGRID_TOL


def test_bounded_wait_reports_timeout(idg_mod, oracle_mod, cuda_device):
    """A device wait that nothing completes gives up after its limit (20 ms
    here), the host reads IDG_ERR_TIMEOUT from the plan's status word, the
    word is cleared, and the plan keeps working."""
    obs = synth.config(1, n_stations=6, n_timesteps=4)
    A, vis = _random_problem(3, obs)
    c = Case(idg_mod, oracle_mod, obs, A, vis)
    c.plan.wait_selftest(20000)
    with pytest.raises(idg_mod.IdgError) as e:
        c.plan.synchronize()
    assert e.value.status == 7
    c.plan.synchronize()
    assert _rel(c.gpu_grid(), c.oracle_grid()) < GRID_TOL
    with pytest.raises(idg_mod.IdgError) as e:
        c.plan.wait_selftest(0)
    assert e.value.status == 1


def _small_obs(rng, L, nodes=9, n_t=10, n_ch=12):
    enu = synth.stations_uniform_disk(rng, 8, 3000.0)
    return synth.make_observation(enu, n_t, 2.0, np.linspace(140e6, 170e6, n_ch), 4, 4096, L, 18, 0.5,
                                  aterm_nodes=nodes, name="small")


@pytest.mark.parametrize("nodes,L", [(5, 64), (13, 96), (2, 128)])
def test_aterm_node_counts(idg_mod, oracle_mod, cuda_device, nodes, L):
    """A-term sampling grids other than 9 x 9 (Section 3.3 interpolation)."""
    rng = np.random.default_rng(nodes)
    obs = _small_obs(rng, L, nodes)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, nodes)
    vis = synth.random_visibilities(rng, obs)
    N = obs.grid_size
    Grand = (rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))) * 1e-3
    c = Case(idg_mod, oracle_mod, obs, A, vis)
    assert _rel(c.gpu_grid(), c.oracle_grid()) < GRID_TOL
    assert _degrid_err(c.gpu_degrid(Grand), c.oracle_degrid(Grand)) < DEGRID_TOL


def test_plans_with_different_node_counts_coexist(idg_mod, oracle_mod, cuda_device):
    """A plan made after another with more A-term nodes must not shrink the
    kernels' shared-memory limit below what the first plan needs."""
    rng = np.random.default_rng(21)
    big = _small_obs(rng, 96, 17)
    A_big = synth.aterms_random(rng, big.n_intervals, big.n_stations, 17)
    vis = synth.random_visibilities(rng, big)
    c_big = Case(idg_mod, oracle_mod, big, A_big, vis)
    small = _small_obs(rng, 96, 3)
    c_small = Case(idg_mod, oracle_mod, small, synth.aterms_random(rng, small.n_intervals, small.n_stations, 3),
                   synth.random_visibilities(rng, small))
    N = big.grid_size
    Grand = (rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))) * 1e-3
    assert _degrid_err(c_big.gpu_degrid(Grand), c_big.oracle_degrid(Grand)) < DEGRID_TOL
    assert _degrid_err(c_small.gpu_degrid(Grand), c_small.oracle_degrid(Grand)) < DEGRID_TOL


def test_user_taper(idg_mod, oracle_mod, cuda_device):
    """IDG_TAPER_USER: the caller's taper samples replace the Kaiser-Bessel taper."""
    import torch
    rng = np.random.default_rng(5)
    obs = _small_obs(rng, 64)
    L = obs.subgrid_size
    x = (np.arange(L) - L / 2) / L
    taper = 0.54 + 0.46 * np.cos(2 * np.pi * x)          # a Hamming-like window, positive everywhere
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes)
    vis = synth.random_visibilities(rng, obs)
    plan = idg_mod.Plan(obs, taper_user=taper)
    geom = oracle_mod.Geometry(obs.grid_size, L, obs.kernel_padding, obs.image_size, taper_kind=1, taper_user=taper,
                               aterm_nodes=obs.aterm_nodes)
    ref_plan = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    args = (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, ref_plan)
    N = obs.grid_size
    G = torch.zeros((4, N, N), dtype=torch.complex128, device="cuda")
    plan.grid(torch.as_tensor(vis.astype(np.complex64)).cuda(), torch.as_tensor(A).cuda(), G)
    plan.synchronize()
    G_ref = oracle_mod.grid(*args, vis.astype(np.complex64).astype(np.complex128), A.astype(np.complex128))
    assert _rel(G.cpu().numpy(), G_ref) < GRID_TOL
    V = torch.empty(vis.shape, dtype=torch.complex64, device="cuda")
    plan.degrid(torch.as_tensor(G_ref).cuda(), torch.as_tensor(A).cuda(), V)
    plan.synchronize()
    V_ref = oracle_mod.degrid(*args, G_ref, A.astype(np.complex128))
    assert _degrid_err(V.cpu().numpy(), V_ref) < DEGRID_TOL
    plan.close()
