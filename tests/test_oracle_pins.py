"""Pins for the FP64 oracle: each test checks it against something other than
itself -- a library routine, a closed form, an exact identity of the method,
a hand-worked example or a textbook brute force (tests/_brute.py)."""
import json
import os

import numpy as np
import pytest
import scipy.special

from paper_2502_17789_gb300 import synth
from tests import _brute

HERE = os.path.dirname(os.path.abspath(__file__))


def _geom(oracle_mod, obs, flags=0, beta=None):
    return oracle_mod.Geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                               taper_beta=beta, aterm_nodes=obs.aterm_nodes, flags=flags)


def _tiny(seed=0, height=15.0, **kw):
    obs = _brute.tiny_observation(seed=seed, **kw)
    rng = np.random.default_rng(seed + 100)
    obs.enu[:, 2] = rng.normal(0.0, height, obs.enu.shape[0])
    hours = obs.times * synth.EARTH_ROTATION
    obs.uvw = synth.uvw_tracks(obs.enu, obs.baselines, hours)
    return obs


def _relerr(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


# ---------------------------------------------------------------- taper / DFT / interpolation

def test_bessel_i0_matches_scipy(oracle_mod):
    for x in [0.0, 0.3, 1.0, 5.0, 9.42, 18.8, 28.27, 40.0]:
        assert oracle_mod.bessel_i0(x) == pytest.approx(float(scipy.special.i0(x)), rel=1e-14)


@pytest.mark.parametrize("L,P", [(16, 6), (32, 12), (96, 18)])
def test_taper_matches_scipy_kaiser_bessel(oracle_mod, L, P):
    beta = np.pi * P / 2
    T = oracle_mod.taper(L, beta)
    np.testing.assert_allclose(T, _brute.kb_taper(L, beta), rtol=1e-13, atol=1e-300)
    assert T[L // 2] == 1.0  # T(0) = 1


@pytest.mark.parametrize("L", [6, 16, 32])
def test_dft2_matches_numpy_fft(oracle_mod, L):
    rng = np.random.default_rng(L)
    X = rng.standard_normal((3, L, L)) + 1j * rng.standard_normal((3, L, L))
    s = (-1.0) ** (np.arange(L)[:, None] + np.arange(L)[None, :])
    # centred kernel e^{-2 pi i (x-L/2)(i-L/2)/L} = (-1)^{x+i+L/2} e^{-2 pi i x i / L}; the
    # (-1)^{L/2} factors of the two axes cancel.
    fwd = s * np.fft.fft2(s * X)
    inv = s * np.fft.ifft2(s * X) * L * L
    np.testing.assert_allclose(oracle_mod.dft2(X, -1), fwd, rtol=0, atol=1e-11 * np.abs(fwd).max())
    np.testing.assert_allclose(oracle_mod.dft2(X, +1), inv, rtol=0, atol=1e-11 * np.abs(inv).max())


def test_aterm_interp_nodes_and_linear_fields(oracle_mod):
    nodes, L, fov = 9, 32, 0.4
    rng = np.random.default_rng(1)
    A = rng.standard_normal((nodes, nodes, 4)) + 1j * rng.standard_normal((nodes, nodes, 4))
    out = oracle_mod.aterm_interp(A, L)
    # pixel i sits on node a when (nodes-1) i / L = a, i.e. i = 4a for L=32
    for a in range(8):
        for b in range(8):
            np.testing.assert_allclose(out[4 * b, 4 * a], A[b, a], rtol=1e-14)
    # a field linear in (l, m) is reproduced exactly between nodes
    c = -0.5 * fov + fov * np.arange(nodes) / (nodes - 1)
    lin = (0.3 + 1.7j) * c[None, :, None] + (2.1 - 0.4j) * c[:, None, None] + np.array([1, 2j, 3, 4j])
    out = oracle_mod.aterm_interp(lin, L)
    pix = (np.arange(L) - L // 2) * fov / L
    expect = (0.3 + 1.7j) * pix[None, :, None] + (2.1 - 0.4j) * pix[:, None, None] + np.array([1, 2j, 3, 4j])
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- planner

def _golden():
    with open(os.path.join(HERE, "golden", "planner_handworked.json")) as f:
        return json.load(f)


def _golden_obs(gd, n_t=5, steps_per_interval=3):
    c = synth.SPEED_OF_LIGHT
    g = gd["geometry"]
    ch = gd["channels"]
    freqs = ch["f0"] + ch["df"] * np.arange(ch["n"])
    uvw = np.zeros((2, n_t, 3))
    uvw[0, :, 0] = 2.9 * c / 1e6
    uvw[1, :, 1] = -3.9 * c / 1e6
    offs = np.array([0, steps_per_interval, n_t], np.int32)
    return g, uvw, freqs, offs


def test_plan_handworked_golden(oracle_mod):
    gd = _golden()
    g, uvw, freqs, offs = _golden_obs(gd)
    geom = oracle_mod.Geometry(g["N"], g["L"], g["P"], g["fov"])
    pl = oracle_mod.plan(geom, uvw, freqs, offs)
    np.testing.assert_array_equal(pl.subgrids, np.array(gd["expected_merged"], np.int32))
    # two segments per subgrid: intervals [0,3) and [3,5)
    assert pl.segments.shape[0] == 2 * pl.subgrids.shape[0]
    for s in range(pl.subgrids.shape[0]):
        segs = pl.segments[pl.segments[:, 0] == s]
        np.testing.assert_array_equal(segs[:, 1:], [[0, 0, 3], [1, 3, 5]])
    geom.flags = oracle_mod.FLAG_SPLIT_INTERVALS
    pl = oracle_mod.plan(geom, uvw, freqs, offs)
    assert int((pl.subgrids[:, 0] == 0).sum()) == gd["expected_split_counts"]["baseline0"]
    assert int((pl.subgrids[:, 0] == 1).sum()) == gd["expected_split_counts"]["baseline1"]
    assert pl.segments.shape[0] == pl.subgrids.shape[0]
    # time case
    tc = gd["time_case"]
    n_t = tc["n_t"]
    uvw = np.zeros((1, n_t, 3))
    uvw[0, :, 0] = (tc["xi0"] - g["N"] / 2 + tc["step"] * np.arange(n_t)) * synth.SPEED_OF_LIGHT / tc["f0"]
    geom = oracle_mod.Geometry(g["N"], g["L"], g["P"], g["fov"])
    pl = oracle_mod.plan(geom, uvw, np.array([tc["f0"]]), np.array([0, n_t], np.int32))
    np.testing.assert_array_equal(pl.subgrids, np.array(tc["expected"], np.int32))


def _shrink_case_uvw(gd):
    sc = gd["shrink_case"]
    xi = np.array(sc["xi"])
    uvw = np.zeros((1, xi.size, 3))
    uvw[0, :, 0] = (xi - gd["geometry"]["N"] / 2) * synth.SPEED_OF_LIGHT / sc["f0"]
    return uvw, np.array([sc["f0"]]), np.array([0, xi.size], np.int32)


def test_plan_shrink_golden(oracle_mod):
    """The final shrink of a time run (Section 3.1 checks only the corners
    while growing): a track whose corners with the first row all fit but
    whose rows 2 and 3 are 23 pixels apart; the hand-worked split is [0,3)
    and [3,6), so a shrink one row short or one row too far fails."""
    gd = _golden()
    g = gd["geometry"]
    uvw, freqs, offs = _shrink_case_uvw(gd)
    pl = oracle_mod.plan(oracle_mod.Geometry(g["N"], g["L"], g["P"], g["fov"]), uvw, freqs, offs)
    np.testing.assert_array_equal(pl.subgrids, np.array(gd["shrink_case"]["expected"], np.int32))


def _check_plan_invariants(obs, pl, split):
    N, L, P, fov = obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size
    u, v, _ = _brute.uvw_lambda(obs)
    xi = u * fov + N // 2
    eta = v * fov + N // 2
    count = np.zeros((obs.n_baselines, obs.n_timesteps, obs.n_channels), int)
    offs = obs.aterm_offsets
    for s, (b, t0, t1, c0, c1, x0, y0, dropped) in enumerate(pl.subgrids):
        assert t1 > t0 and c1 > c0
        count[b, t0:t1, c0:c1] += 1
        if not dropped:
            xs, ys = xi[b, t0:t1, c0:c1], eta[b, t0:t1, c0:c1]
            assert (xs - x0).min() >= P / 2 and (xs - x0).max() <= L - 1 - P / 2
            assert (ys - y0).min() >= P / 2 and (ys - y0).max() <= L - 1 - P / 2
            assert 0 <= x0 <= N - L and 0 <= y0 <= N - L
        segs = pl.segments[pl.segments[:, 0] == s]
        assert segs.shape[0] >= 1
        assert segs[0, 2] == t0 and segs[-1, 3] == t1
        for (_, a, tb, te) in segs:
            assert offs[a] <= tb < te <= offs[a + 1]
        assert np.all(segs[1:, 2] == segs[:-1, 3])
        if split:
            assert segs.shape[0] == 1
    assert np.all(count == 1), "every visibility belongs to exactly one subgrid"


@pytest.mark.parametrize("split", [False, True])
def test_plan_invariants_small(oracle_mod, split):
    obs = synth.config(1)
    obs.aterm_offsets = np.array([0, 5, 11, 16], np.int32)
    geom = _geom(oracle_mod, obs, flags=oracle_mod.FLAG_SPLIT_INTERVALS if split else 0)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    _check_plan_invariants(obs, pl, split)


def test_plan_invariants_mwa_like_reduced(oracle_mod):
    obs = synth.config(2, n_stations=24, n_timesteps=12)
    pl = oracle_mod.plan(_geom(oracle_mod, obs), obs.uvw, obs.freqs, obs.aterm_offsets)
    _check_plan_invariants(obs, pl, False)
    assert pl.subgrids.shape[0] > obs.n_baselines  # long baselines split along channels


def test_plan_error_codes(oracle_mod):
    obs = _tiny()
    geom = _geom(oracle_mod, obs)
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.plan(geom, obs.uvw, obs.freqs[::-1].copy(), obs.aterm_offsets)
    assert e.value.code == 2
    u, v, _ = _brute.uvw_lambda(obs)
    reach = np.abs(np.stack([u, v])).max(axis=(0, 2, 3)) * obs.image_size  # pixels from centre, per baseline
    limit = obs.grid_size / 2 - obs.subgrid_size / 2
    big = obs.uvw * (1.2 * limit / np.median(reach))  # pushes the longer baselines off the 64-pixel grid
    big[..., 2] = 0.0
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.plan(geom, big, obs.freqs, obs.aterm_offsets)
    assert e.value.code == 3
    geom.flags = oracle_mod.FLAG_DROP
    pl = oracle_mod.plan(geom, big, obs.freqs, obs.aterm_offsets)
    assert pl.subgrids[:, 7].sum() > 0 and pl.subgrids[:, 7].sum() < pl.subgrids.shape[0]
    geom.flags = 0
    wbig = obs.uvw.copy()
    wbig[..., 2] = 500.0
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.plan(geom, wbig, obs.freqs, obs.aterm_offsets)
    assert e.value.code == 4


# ---------------------------------------------------------------- gridding / degridding

def _problem(oracle_mod, seed=0, n_int=2, n_t=4, split=False, **kw):
    obs = _tiny(seed=seed, n_t=n_t, steps_per_interval=max(1, n_t // n_int), **kw)
    rng = np.random.default_rng(seed + 7)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes).astype(np.complex128)
    vis = synth.random_visibilities(rng, obs).astype(np.complex128)
    geom = _geom(oracle_mod, obs, flags=oracle_mod.FLAG_SPLIT_INTERVALS if split else 0)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    return obs, geom, pl, A, vis


def _grid(oracle_mod, obs, geom, pl, vis, A, **kw):
    return oracle_mod.grid(geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl,
                           vis, A, **kw)


def _degrid(oracle_mod, obs, geom, pl, G, A):
    return oracle_mod.degrid(geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl,
                             G, A)


@pytest.mark.parametrize("split", [False, True])
def test_grid_image_equals_direct_dft_at_coarse_points(oracle_mod, split):
    """At l_i = (i - L/2) FOV/L the dirty image of the master grid is exactly
    L^2 T_i T_j times the adjoint of the discrete measurement equation (Eq. 1)
    with A-terms: the L-point subgrid transform reproduces every sample point
    of the subgrid image, so no aliasing term enters."""
    obs, geom, pl, A, vis = _problem(oracle_mod, split=split)
    G = _grid(oracle_mod, obs, geom, pl, vis, A)
    L, fov = obs.subgrid_size, obs.image_size
    T = _brute.kb_taper(L, geom.beta)
    worst = 0.0
    for (i, j) in [(8, 8), (3, 11), (12, 2), (0, 5), (15, 15), (6, 9)]:
        l, m = (i - L // 2) * fov / L, (j - L // 2) * fov / L
        got = _brute.image_from_grid(G, fov, l, m)
        want = L * L * T[i] * T[j] * _brute.dft_image(obs, vis, A, l, m)
        worst = max(worst, np.abs(got - want).max() / np.abs(want).max())
    assert worst < 1e-9


def test_degrid_point_source_equals_measurement_equation(oracle_mod):
    """Degridding the Fourier transform of a point source sitting on a coarse
    image point gives Eq. 1 exactly, times L^2 T_i T_j."""
    obs, geom, pl, A, _ = _problem(oracle_mod, seed=3)
    L, fov, N = obs.subgrid_size, obs.image_size, obs.grid_size
    T = _brute.kb_taper(L, geom.beta)
    B = np.array([[1.3, 0.2 - 0.1j], [0.2 + 0.1j, 0.7]])
    for (i0, j0) in [(8, 8), (5, 10), (11, 4)]:
        l, m = (i0 - L // 2) * fov / L, (j0 - L // 2) * fov / L
        G = _brute.point_source_grid(N, fov, l, m, B)
        V = _degrid(oracle_mod, obs, geom, pl, G, A)
        want = L * L * T[i0] * T[j0] * _brute.measurement_equation(obs, A, l, m, B)
        assert _relerr(V, want) < 1e-10


def test_dc_invariant_with_aterms(oracle_mod):
    """sum_{x,y} G = L^2 T(0)^2 sum_segments A_p(0,0)^H (sum_k V_k) A_q(0,0):
    only the centre pixel survives the sum, where the phase is zero."""
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=5, n_int=3, n_t=6)
    G = _grid(oracle_mod, obs, geom, pl, vis, A)
    L = obs.subgrid_size
    c = obs.aterm_nodes // 2
    want = np.zeros((2, 2), complex)
    for (s, a, tb, te) in pl.segments:
        b, _, _, c0, c1 = pl.subgrids[s, :5]
        p, q = obs.baselines[b]
        S = vis[b, tb:te, c0:c1].sum(axis=(0, 1)).reshape(2, 2)
        want += A[a, p, c, c].reshape(2, 2).conj().T @ S @ A[a, q, c, c].reshape(2, 2)
    got = G.sum(axis=(1, 2)).reshape(2, 2)
    assert _relerr(got, L * L * want) < 1e-12


def test_point_source_at_phase_centre(oracle_mod):
    obs = _tiny(seed=2)
    A = synth.aterms_identity(obs.n_intervals, obs.n_stations).astype(np.complex128)
    geom = _geom(oracle_mod, obs)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    L = obs.subgrid_size
    S = 2.5
    vis = np.zeros((obs.n_baselines, obs.n_timesteps, obs.n_channels, 4), complex)
    vis[..., 0] = S
    vis[..., 3] = S
    G = _grid(oracle_mod, obs, geom, pl, vis, A)
    tot = G.sum(axis=(1, 2))
    np.testing.assert_allclose(tot, [L * L * S * obs.n_vis, 0, 0, L * L * S * obs.n_vis], rtol=1e-13, atol=1e-9)
    Gc = np.zeros((4, obs.grid_size, obs.grid_size), complex)
    Gc[0] = S
    Gc[3] = S
    V = _degrid(oracle_mod, obs, geom, pl, Gc, A)
    want = np.zeros_like(V)
    want[..., 0] = L * L * S
    want[..., 3] = L * L * S
    np.testing.assert_allclose(V, want, rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("split", [False, True])
def test_adjoint_identity(oracle_mod, split):
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=11, split=split)
    rng = np.random.default_rng(4)
    N = obs.grid_size
    G = rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))
    lhs = np.vdot(_degrid(oracle_mod, obs, geom, pl, G, A), vis)
    rhs = np.vdot(G, _grid(oracle_mod, obs, geom, pl, vis, A))
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_convolutional_gridding_closed_form(oracle_mod):
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=13, n_st=3, n_t=2, n_ch=2)
    G = _grid(oracle_mod, obs, geom, pl, vis, A)
    T = _brute.kb_taper(obs.subgrid_size, geom.beta)
    Gc = _brute.convolutional_grid(obs, pl, vis.astype(np.complex128), A, T)
    assert _relerr(G, Gc) < 1e-12


def test_linearity(oracle_mod):
    obs, geom, pl, A, v1 = _problem(oracle_mod, seed=17)
    v2 = synth.random_visibilities(np.random.default_rng(99), obs).astype(np.complex128)
    a, b = 0.7 - 1.1j, -2.0 + 0.3j
    lhs = _grid(oracle_mod, obs, geom, pl, a * v1 + b * v2, A)
    rhs = a * _grid(oracle_mod, obs, geom, pl, v1, A) + b * _grid(oracle_mod, obs, geom, pl, v2, A)
    assert _relerr(lhs, rhs) < 1e-13


def test_subgrid_images_match_grid(oracle_mod):
    """The exported pre-FFT subgrid images transform and add up to the grid."""
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=19)
    G, img, uv = _grid(oracle_mod, obs, geom, pl, vis, A, want_subgrids=True)
    np.testing.assert_allclose(uv, oracle_mod.dft2(img, -1), rtol=0, atol=1e-10 * np.abs(uv).max())
    L = obs.subgrid_size
    G2 = np.zeros_like(G)
    for s, row in enumerate(pl.subgrids):
        x0, y0 = row[5], row[6]
        G2[:, y0:y0 + L, x0:x0 + L] += uv[s]
    assert _relerr(G, G2) < 1e-14


def test_degrid_off_grid_sources_within_aliasing_bound(oracle_mod):
    """Point sources anywhere in the central 1/1.5 of the field (not on the
    coarse grid): the oracle's degridded model, transformed with 1/T, agrees
    with Eq. 1 to the taper kernel's aliasing level, 1e-7 at P = 18 with the
    default beta = 0.35 pi P (measured with this oracle at P = 18: 1.6e-6 at
    beta = 16, 9.7e-8 at 20, 5.2e-9 at 24)."""
    obs = _tiny(seed=8, n_st=5, n_t=4, n_ch=3, N=1024, L=96, P=18, fov=0.5, diameter=400.0)
    geom = _geom(oracle_mod, obs)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    A = synth.aterms_identity(obs.n_intervals, obs.n_stations).astype(np.complex128)
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    T = lambda x: scipy.special.i0(geom.beta * np.sqrt(1 - (2 * x / fov) ** 2)) / scipy.special.i0(geom.beta)
    u = (np.arange(N) - N // 2) / fov
    for (l, m) in [(0.1113, -0.0719), (-0.16, 0.155), (0.0533, 0.1499)]:
        G = np.zeros((4, N, N), complex)
        G[0] = np.outer(np.exp(-2j * np.pi * u * m), np.exp(-2j * np.pi * u * l)) / (T(l) * T(m))
        G[3] = G[0]
        V = _degrid(oracle_mod, obs, geom, pl, G, A)
        want = L * L * _brute.measurement_equation(obs, A, l, m, np.eye(2))
        assert np.abs(V - want).max() / np.abs(want).max() < 1e-6


# ---------------------------------------------------------------- image-domain wrapper (Eq. 11, Eq. 12)

def _wrapper_args(obs, geom, pl):
    return (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)


def test_invert_equals_direct_adjoint_on_the_subgrid_lattice(oracle_mod):
    """On image pixels that coincide with subgrid pixel positions
    (p - N/2 = (N/L)(i - L/2)) the dirty image is exactly the adjoint of
    Eq. 1 with A-terms: the gridder's L^2 T_i T_j is divided out by the same
    taper values.  The check is a direct sum over the visibilities."""
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=5)
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    img = oracle_mod.invert(*_wrapper_args(obs, geom, pl), vis, A)
    r = N // L
    worst = 0.0
    for (i, j) in [(8, 8), (3, 11), (12, 2), (5, 7), (9, 14)]:
        p, q = N // 2 + r * (i - L // 2), N // 2 + r * (j - L // 2)
        l, m = (p - N // 2) * fov / N, (q - N // 2) * fov / N
        want = _brute.dft_image(obs, vis, A, l, m).reshape(4)
        worst = max(worst, np.abs(img[:, q, p] - want).max() / np.abs(want).max())
    assert worst < 1e-9


def test_predict_of_a_lattice_point_source_is_the_measurement_equation(oracle_mod):
    """predict() of an image holding brightness B on one lattice pixel gives
    Eq. 1 for a point source there, exactly."""
    obs, geom, pl, A, _ = _problem(oracle_mod, seed=6)
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    r = N // L
    B = np.array([[0.9, 0.1 + 0.3j], [0.1 - 0.3j, 1.4]])
    for (i, j) in [(8, 8), (4, 10), (11, 5)]:
        p, q = N // 2 + r * (i - L // 2), N // 2 + r * (j - L // 2)
        img = np.zeros((4, N, N), complex)
        img[:, q, p] = B.reshape(4)
        V = oracle_mod.predict(*_wrapper_args(obs, geom, pl), img, A)
        l, m = (p - N // 2) * fov / N, (q - N // 2) * fov / N
        want = _brute.measurement_equation(obs, A, l, m, B)
        assert _relerr(V, want) < 1e-10


def test_predict_is_the_adjoint_of_invert(oracle_mod):
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=7)
    N = obs.grid_size
    rng = np.random.default_rng(3)
    img = rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))
    lhs = np.vdot(oracle_mod.predict(*_wrapper_args(obs, geom, pl), img, A), vis)
    rhs = np.vdot(img, oracle_mod.invert(*_wrapper_args(obs, geom, pl), vis, A))
    assert abs(lhs - rhs) / abs(rhs) < 1e-11


def test_invert_off_lattice_within_aliasing_bound(oracle_mod):
    """Anywhere in the central 1/1.5 of the field the dirty image agrees with
    the direct adjoint of Eq. 1 to the taper kernel's aliasing level (P = 18,
    default beta)."""
    obs = _tiny(seed=9, n_st=5, n_t=4, n_ch=3, N=1024, L=96, P=18, fov=0.5, diameter=400.0)
    geom = _geom(oracle_mod, obs)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    A = synth.aterms_identity(obs.n_intervals, obs.n_stations).astype(np.complex128)
    rng = np.random.default_rng(4)
    vis = rng.standard_normal(obs.uvw.shape[:2] + (obs.n_channels, 4)) \
        + 1j * rng.standard_normal(obs.uvw.shape[:2] + (obs.n_channels, 4))
    img = oracle_mod.invert(*_wrapper_args(obs, geom, pl), vis, A)
    N, fov = obs.grid_size, obs.image_size
    scale = np.abs(vis).sum()
    for (p, q) in [(611, 433), (371, 660), (512, 301), (689, 689)]:
        l, m = (p - N // 2) * fov / N, (q - N // 2) * fov / N
        want = _brute.dft_image(obs, vis, A, l, m).reshape(4)
        assert np.abs(img[:, q, p] - want).max() / scale < 1e-6


# ---------------------------------------------------------------- w layers (Section 2.4, Eq. 11, Eq. 12)

def _layered_problem(oracle_mod, seed=0, height=400.0, n_t=6, **kw):
    """A strongly non-coplanar array: |w| well beyond w_max, so w0 = 0 alone
    is rejected and the visibilities spread over several w layers."""
    obs = _tiny(seed=seed, height=height, n_t=n_t, steps_per_interval=3, **kw)
    rng = np.random.default_rng(seed + 11)
    A = synth.aterms_random(rng, obs.n_intervals, obs.n_stations, obs.aterm_nodes).astype(np.complex128)
    vis = synth.random_visibilities(rng, obs).astype(np.complex128)
    geom = _geom(oracle_mod, obs, flags=oracle_mod.FLAG_W_LAYERS)
    pl = oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)
    return obs, geom, pl, A, vis


def _w_prime(obs):
    """Per (baseline, timestep): the side (True = mirrored, w < 0) and the
    gridded coordinates (u', v', w') = sign * (u, v, w) in wavelengths."""
    u, v, w = _brute.uvw_lambda(obs)
    neg = obs.uvw[..., 2] < 0.0
    sgn = np.where(neg, -1.0, 1.0)[..., None]
    return neg, sgn * u, sgn * v, sgn * w


def test_w_layers_plan_invariants(oracle_mod):
    """Section 2.4: rows with w < 0 are mirrored, every gridded w' >= 0 sits
    within w_max of its subgrid's layer w0 = (2k+1) w_max, a subgrid holds one
    layer and one side, and the mirrored members lie inside their subgrid at
    their mirrored (u', v') pixel coordinates."""
    obs, geom, pl, _, _ = _layered_problem(oracle_mod)
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.plan(_geom(oracle_mod, obs), obs.uvw, obs.freqs, obs.aterm_offsets)
    assert e.value.code == 4
    assert pl.k_range[1] >= 2
    # w_max from the fringe limit of the Section 2.4 footnote, independently
    r2 = 0.5 * obs.image_size ** 2
    w_max = (obs.kernel_padding / 2 - 1) / (np.sqrt(r2 / (1 - r2)) * obs.image_size)
    assert pl.w_step == pytest.approx(2 * w_max, rel=1e-14)
    neg, u2, v2, w2 = _w_prime(obs)
    assert neg.any() and (~neg).any(), "the problem needs rows on both sides"
    N, L, P, fov = obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size
    count = np.zeros((obs.n_baselines, obs.n_timesteps, obs.n_channels), int)
    for s, (b, t0, t1, c0, c1, x0, y0, dropped) in enumerate(pl.subgrids):
        count[b, t0:t1, c0:c1] += 1
        assert np.all(neg[b, t0:t1] == bool(pl.conj[s])), "one side per subgrid"
        w0 = (2 * pl.layers[s] + 1) * w_max
        assert pl.layers[s] >= 0
        assert np.abs(w2[b, t0:t1, c0:c1] - w0).max() <= w_max * (1 + 1e-12)
        xs = u2[b, t0:t1, c0:c1] * fov + N // 2
        ys = v2[b, t0:t1, c0:c1] * fov + N // 2
        assert (xs - x0).min() >= P / 2 and (xs - x0).max() <= L - 1 - P / 2
        assert (ys - y0).min() >= P / 2 and (ys - y0).max() <= L - 1 - P / 2
    assert np.all(count == 1), "every visibility belongs to exactly one subgrid"


def test_w_layers_of_a_coplanar_array_are_one_layer_at_w_max(oracle_mod):
    """A nearly coplanar array has every |w| < 2 w_max: all subgrids fall in
    the first layer of the paper's set, w0 = w_max, on either side."""
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=2)
    g2 = _geom(oracle_mod, obs, flags=oracle_mod.FLAG_W_LAYERS)
    p2 = oracle_mod.plan(g2, obs.uvw, obs.freqs, obs.aterm_offsets)
    assert np.all(p2.layers == 0) and p2.k_range == (0, 1)
    neg, *_ = _w_prime(obs)
    assert neg.any() and (~neg).any()
    assert p2.w0(0) == pytest.approx(0.5 * p2.w_step)
    G2 = oracle_mod.grid(g2, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, p2, vis, A)
    assert G2.shape == (1, 4, obs.grid_size, obs.grid_size)


def _herm(img):
    """Hermitian part (B + B^H)/2 of a [4][...] image of 2x2 matrices."""
    m = np.moveaxis(np.asarray(img).reshape((2, 2) + np.shape(img)[1:]), (0, 1), (-2, -1))
    h = 0.5 * (m + np.conj(np.swapaxes(m, -1, -2)))
    return np.moveaxis(h, (-2, -1), (0, 1)).reshape(np.shape(img))


def test_w_stacked_invert_equals_direct_adjoint_on_the_lattice(oracle_mod):
    """With w layers the dirty image on the subgrid lattice is exactly the
    adjoint of Eq. 1 over the mirrored visibility set (each row of w < 0
    replaced by V^H of baseline (q, p) at -uvw): every subgrid carries
    (w' - w0) and each layer transform multiplies by e^{2 pi i w0 n'}
    (Eq. 11).  Its Hermitian part equals that of the direct adjoint of the
    visibilities as given, which the mirror cannot change (the footnote's
    symmetry)."""
    obs, geom, pl, A, vis = _layered_problem(oracle_mod, seed=1)
    assert pl.conj.any() and not pl.conj.all()
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    img = oracle_mod.invert(*_wrapper_args(obs, geom, pl), vis, A)
    o2, v2 = _brute.mirrored_set(obs, vis)
    r = N // L
    worst = worst_h = 0.0
    for (i, j) in [(8, 8), (2, 13), (13, 3), (5, 6), (10, 12)]:
        p, q = N // 2 + r * (i - L // 2), N // 2 + r * (j - L // 2)
        l, m = (p - N // 2) * fov / N, (q - N // 2) * fov / N
        want = _brute.dft_image(o2, v2, A, l, m).reshape(4)
        worst = max(worst, np.abs(img[:, q, p] - want).max() / np.abs(want).max())
        direct = _brute.dft_image(obs, vis, A, l, m).reshape(4, 1)
        worst_h = max(worst_h, np.abs(_herm(img[:, q, p].reshape(4, 1)) - _herm(direct)).max() / np.abs(direct).max())
    assert worst < 1e-9
    assert worst_h < 1e-9


def test_w_stacked_predict_of_a_lattice_point_source(oracle_mod):
    """A point source of Hermitian brightness on the lattice predicts Eq. 1
    for every visibility, mirrored rows included: the degridder predicts the
    mirror and returns its conjugate transpose, which for Hermitian B is the
    visibility itself."""
    obs, geom, pl, A, _ = _layered_problem(oracle_mod, seed=3)
    assert pl.conj.any() and not pl.conj.all()
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    r = N // L
    B = np.array([[1.1, -0.2j], [0.2j, 0.8]])
    for (i, j) in [(8, 8), (3, 12), (12, 4)]:
        p, q = N // 2 + r * (i - L // 2), N // 2 + r * (j - L // 2)
        img = np.zeros((4, N, N), complex)
        img[:, q, p] = B.reshape(4)
        V = oracle_mod.predict(*_wrapper_args(obs, geom, pl), img, A)
        l, m = (p - N // 2) * fov / N, (q - N // 2) * fov / N
        assert _relerr(V, _brute.measurement_equation(obs, A, l, m, B)) < 1e-10


def test_w_stacked_predict_is_the_adjoint_of_invert(oracle_mod):
    """The mirror conjugates, so with w layers the pair is adjoint in the
    real inner product Re<x, y> (conjugation is real-linear)."""
    obs, geom, pl, A, vis = _layered_problem(oracle_mod, seed=4)
    assert pl.conj.any()
    N = obs.grid_size
    rng = np.random.default_rng(5)
    img = rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))
    lhs = np.vdot(oracle_mod.predict(*_wrapper_args(obs, geom, pl), img, A), vis).real
    rhs = np.vdot(img, oracle_mod.invert(*_wrapper_args(obs, geom, pl), vis, A)).real
    assert abs(lhs - rhs) / abs(rhs) < 1e-11


def test_w_layered_degrid_is_the_adjoint_of_grid(oracle_mod):
    """Gridding and degridding with mirrored subgrids on layered grids are
    adjoint in the real inner product."""
    obs, geom, pl, A, vis = _layered_problem(oracle_mod, seed=6)
    assert pl.conj.any()
    args = (geom, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)
    G = oracle_mod.grid(*args, vis, A)
    rng = np.random.default_rng(7)
    R = rng.standard_normal(G.shape) + 1j * rng.standard_normal(G.shape)
    lhs = np.vdot(oracle_mod.degrid(*args, R, A), vis).real
    rhs = np.vdot(R, G).real
    assert abs(lhs - rhs) / abs(rhs) < 1e-11


# ---------------------------------------------------------------- A-term power normalisation (Section 3.3)

def _segment_norms(obs, pl, A, l, m):
    """Per plan segment: (visibility count, f = ||A_p^H A_q||_F at (l, m)),
    with A interpolated by numpy (tests/_brute.bilinear_at)."""
    out = []
    for (s, a, tb, te) in pl.segments:
        b, _, _, c0, c1, _, _, dropped = [int(z) for z in pl.subgrids[s]]
        if dropped:
            continue
        p, q = obs.baselines[b]
        Ap = _brute.bilinear_at(A[a, p], obs.image_size, l, m)
        Aq = _brute.bilinear_at(A[a, q], obs.image_size, l, m)
        out.append(((te - tb) * (c1 - c0), np.linalg.norm(Ap.conj().T @ Aq)))
    return out


def test_normalised_weights_are_the_segment_frobenius_norms(oracle_mod):
    """The weight map is sum over segments of n_seg / ||A_p^H A_q||_F at every
    subgrid lattice point, and its last slot the number of visibilities."""
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=11)
    L, fov = obs.subgrid_size, obs.image_size
    _, W = _grid(oracle_mod, obs, geom, pl, vis, A, normalize=True)
    assert W[L * L] == obs.n_baselines * obs.n_timesteps * obs.n_channels
    worst = 0.0
    for (i, j) in [(0, 0), (8, 8), (3, 11), (15, 2), (9, 14)]:
        l, m = (i - L // 2) * fov / L, (j - L // 2) * fov / L
        want = sum(n / f for n, f in _segment_norms(obs, pl, A, l, m))
        worst = max(worst, abs(W[j * L + i] - want) / want)
    assert worst < 1e-12


def test_normalised_invert_on_the_lattice_is_the_weighted_direct_adjoint(oracle_mod):
    """On the subgrid lattice the normalised dirty image is
      [sum_seg adj_seg(l,m) / f_seg(l,m)] / [(sum_seg n_seg / f_seg(l,m)) / sum n_seg],
    adj_seg the adjoint of Eq. 1 over the segment's visibilities (a direct sum)."""
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=12)
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    img = oracle_mod.invert(*_wrapper_args(obs, geom, pl), vis, A, normalize=True)
    u, v, w = _brute.uvw_lambda(obs)
    n_tot = obs.n_baselines * obs.n_timesteps * obs.n_channels
    r = N // L
    worst = 0.0
    for (i, j) in [(8, 8), (3, 11), (12, 2), (5, 7)]:
        p, q = N // 2 + r * (i - L // 2), N // 2 + r * (j - L // 2)
        l, m = (p - N // 2) * fov / N, (q - N // 2) * fov / N
        n1 = np.sqrt(1.0 - l * l - m * m) - 1.0
        num = np.zeros((2, 2), np.complex128)
        den = 0.0
        for (s, a, tb, te) in pl.segments:
            b, _, _, c0, c1 = [int(z) for z in pl.subgrids[s][:5]]
            pa, qa = obs.baselines[b]
            Ap = _brute.bilinear_at(A[a, pa], fov, l, m)
            Aq = _brute.bilinear_at(A[a, qa], fov, l, m)
            f = np.linalg.norm(Ap.conj().T @ Aq)
            ph = np.exp(2j * np.pi * (u[b, tb:te, c0:c1] * l + v[b, tb:te, c0:c1] * m + w[b, tb:te, c0:c1] * n1))
            S = np.einsum("tc,tce->e", ph, vis[b, tb:te, c0:c1]).reshape(2, 2)
            num += Ap.conj().T @ S @ Aq / f
            den += (te - tb) * (c1 - c0) / f
        want = (num / (den / n_tot)).reshape(4)
        worst = max(worst, np.abs(img[:, q, p] - want).max() / np.abs(want).max())
    assert worst < 1e-9


def test_normalisation_is_a_no_op_for_identity_aterms(oracle_mod):
    """Identity A-terms: f = sqrt(2) everywhere, so the normalised image
    equals the plain one."""
    obs, geom, pl, _, vis = _problem(oracle_mod, seed=13)
    A = synth.aterms_identity(obs.n_intervals, obs.n_stations, obs.aterm_nodes).astype(np.complex128)
    plain = oracle_mod.invert(*_wrapper_args(obs, geom, pl), vis, A)
    norm = oracle_mod.invert(*_wrapper_args(obs, geom, pl), vis, A, normalize=True)
    assert _relerr(norm, plain) < 1e-12
    L = obs.subgrid_size
    _, W = _grid(oracle_mod, obs, geom, pl, vis, A, normalize=True)
    assert np.allclose(W[: L * L], W[L * L] / np.sqrt(2.0), rtol=1e-13, atol=0)


def test_lattice_to_image_reproduces_bilinear_fields(oracle_mod):
    """A map that is bilinear in (l, m) on the lattice is reproduced exactly at
    every image pixel inside the lattice, and extended flat beyond it."""
    N, L = 64, 16
    li = np.arange(L) - L // 2
    field = 2.0 + 0.3 * li[None, :] - 0.1 * li[:, None] + 0.01 * li[None, :] * li[:, None]   # [j][i]
    img = oracle_mod.lattice_to_image(field, N, L)
    x = (np.arange(N) - N // 2) * (L / N)        # lattice offset of pixel p
    inside = x <= L // 2 - 1
    want = 2.0 + 0.3 * x[None, :] - 0.1 * x[:, None] + 0.01 * x[None, :] * x[:, None]
    assert np.allclose(img[np.ix_(inside, inside)], want[np.ix_(inside, inside)], rtol=0, atol=1e-12)
    assert np.allclose(img[:, -1], img[:, np.flatnonzero(inside)[-1]])


# ---------------------------------------------------------------- Stokes I (one image plane)

def _stokes_geom(oracle_mod, obs, geom):
    return oracle_mod.Geometry(geom.grid_size, geom.subgrid_size, geom.kernel_padding, geom.image_size,
                               aterm_nodes=geom.aterm_nodes, flags=geom.flags | oracle_mod.FLAG_STOKES_I)


def test_stokes_i_invert_on_the_lattice_is_half_the_trace_of_the_direct_adjoint(oracle_mod):
    """With one Stokes-I plane the dirty image on the subgrid lattice is
    (XX + YY) / 2 of the adjoint of Eq. 1 with A-terms (a direct sum)."""
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=21)
    gi = _stokes_geom(oracle_mod, obs, geom)
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    img = oracle_mod.invert(gi, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl, vis, A)
    assert img.shape == (1, N, N)
    r = N // L
    worst = 0.0
    for (i, j) in [(8, 8), (3, 11), (12, 2), (5, 7)]:
        p, q = N // 2 + r * (i - L // 2), N // 2 + r * (j - L // 2)
        l, m = (p - N // 2) * fov / N, (q - N // 2) * fov / N
        adj = _brute.dft_image(obs, vis, A, l, m)
        want = 0.5 * (adj[0, 0] + adj[1, 1])
        worst = max(worst, abs(img[0, q, p] - want) / abs(want))
    assert worst < 1e-9


def test_stokes_i_predict_of_a_lattice_point_source_is_the_measurement_equation(oracle_mod):
    """An unpolarised point source S on one lattice pixel of the Stokes-I
    image predicts Eq. 1 with brightness S times the identity."""
    obs, geom, pl, A, _ = _problem(oracle_mod, seed=22)
    gi = _stokes_geom(oracle_mod, obs, geom)
    N, L, fov = obs.grid_size, obs.subgrid_size, obs.image_size
    r = N // L
    for (i, j, S) in [(8, 8, 1.3), (4, 10, 0.7)]:
        p, q = N // 2 + r * (i - L // 2), N // 2 + r * (j - L // 2)
        img = np.zeros((1, N, N), complex)
        img[0, q, p] = S
        V = oracle_mod.predict(gi, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl, img, A)
        l, m = (p - N // 2) * fov / N, (q - N // 2) * fov / N
        want = _brute.measurement_equation(obs, A, l, m, S * np.eye(2))
        assert _relerr(V, want) < 1e-10


def test_stokes_i_pair_is_adjoint_up_to_one_half(oracle_mod):
    """invert takes (XX + YY) / 2 while predict puts I on XX and YY, so
    <predict(img), v> = 2 <img, invert(v)>."""
    obs, geom, pl, A, vis = _problem(oracle_mod, seed=23)
    gi = _stokes_geom(oracle_mod, obs, geom)
    N = obs.grid_size
    rng = np.random.default_rng(5)
    img = rng.standard_normal((1, N, N)) + 1j * rng.standard_normal((1, N, N))
    args = (gi, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets, pl)
    lhs = np.vdot(oracle_mod.predict(*args, img, A), vis)
    rhs = np.vdot(img, oracle_mod.invert(*args, vis, A))
    assert abs(lhs - 2.0 * rhs) / abs(lhs) < 1e-11
