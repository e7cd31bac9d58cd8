"""CPU tests of libidg: the C ABI exports and the host planner (no device
work; plans are created with IDG_HOST_ONLY)."""
import os
import re

import numpy as np
import pytest

from paper_2502_17789_gb300 import synth
from tests import _brute

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "idg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(idg_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ["idg_plan_create", "idg_grid", "idg_degrid", "idg_plan_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(idg_mod):
    lib = idg_mod.load()
    names = _declared_functions()
    assert sorted(idg_mod.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n
    assert idg_mod.idg_abi_version() == 3


def _host_plan(idg_mod, obs, flags=0, L=None):
    g, keep = idg_mod.make_geometry(obs.grid_size, L or obs.subgrid_size, obs.kernel_padding, obs.image_size,
                                    aterm_nodes=obs.aterm_nodes, flags=flags | idg_mod.IDG_HOST_ONLY)
    h = idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets)
    try:
        return idg_mod.idg_plan_subgrids(h), idg_mod.idg_plan_segments(h), idg_mod.idg_plan_stats(h)
    finally:
        idg_mod.idg_plan_destroy(h)


def _oracle_plan(oracle_mod, obs, flags=0, L=None):
    geom = oracle_mod.Geometry(obs.grid_size, L or obs.subgrid_size, obs.kernel_padding, obs.image_size,
                               aterm_nodes=obs.aterm_nodes, flags=flags)
    return oracle_mod.plan(geom, obs.uvw, obs.freqs, obs.aterm_offsets)


CASES = [
    ("small", lambda: synth.config(1), None),
    ("small-L64", lambda: synth.config(1), 64),
    ("mwa-like-reduced", lambda: synth.config(2, n_stations=40, n_timesteps=20), None),
    ("mwa-like-reduced-L128", lambda: synth.config(2, n_stations=30, n_timesteps=16), 128),
    ("uneven-reduced", lambda: synth.config(4, n_stations=48, n_timesteps=40), 64),
]


@pytest.mark.parametrize("name,make,L", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("split", [False, True])
def test_planner_bit_exact_against_oracle(idg_mod, oracle_mod, name, make, L, split):
    obs = make()
    f_lib = idg_mod.IDG_SPLIT_AT_ATERM_INTERVALS if split else 0
    f_or = oracle_mod.FLAG_SPLIT_INTERVALS if split else 0
    sg, seg, st = _host_plan(idg_mod, obs, f_lib, L)
    ref = _oracle_plan(oracle_mod, obs, f_or, L)
    np.testing.assert_array_equal(sg, ref.subgrids)
    np.testing.assert_array_equal(seg, ref.segments)
    assert st.n_vis == obs.n_vis and st.n_subgrids == len(sg)
    assert sum(st.occupancy_hist) == len(sg)


def test_planner_drop_flag_bit_exact(idg_mod, oracle_mod):
    obs = _brute.tiny_observation(seed=4, n_st=8)
    u, v, _ = _brute.uvw_lambda(obs)
    reach = np.abs(np.stack([u, v])).max(axis=(0, 2, 3)) * obs.image_size
    obs.uvw = obs.uvw * (1.2 * (obs.grid_size / 2 - obs.subgrid_size / 2) / np.median(reach))
    obs.uvw[..., 2] = 0.0
    with pytest.raises(idg_mod.IdgError) as e:
        _host_plan(idg_mod, obs)
    assert e.value.status == 3
    sg, seg, st = _host_plan(idg_mod, obs, idg_mod.IDG_DROP_OUT_OF_GRID)
    ref = _oracle_plan(oracle_mod, obs, oracle_mod.FLAG_DROP)
    np.testing.assert_array_equal(sg, ref.subgrids)
    np.testing.assert_array_equal(seg, ref.segments)
    assert st.n_subgrids_dropped == int(ref.subgrids[:, 7].sum()) > 0


def test_planner_error_codes(idg_mod):
    obs = _brute.tiny_observation(seed=1)
    bad = obs.freqs[::-1].copy()
    g, _ = idg_mod.make_geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                                 flags=idg_mod.IDG_HOST_ONLY)
    with pytest.raises(idg_mod.IdgError) as e:
        idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, bad, obs.aterm_offsets)
    assert e.value.status == 2 and "ascending" in str(e.value)
    w = obs.uvw.copy()
    w[..., 2] = 500.0
    with pytest.raises(idg_mod.IdgError) as e:
        idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, w, obs.freqs, obs.aterm_offsets)
    assert e.value.status == 4
    with pytest.raises(idg_mod.IdgError) as e:
        idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, np.array([0, 1], np.int32))
    assert e.value.status == 1
    # device plans accept only the compiled subgrid sizes
    g2, _ = idg_mod.make_geometry(obs.grid_size, 16, obs.kernel_padding, obs.image_size)
    with pytest.raises(idg_mod.IdgError) as e:
        idg_mod.idg_plan_create(g2, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets)
    assert e.value.status == 8
    bl = obs.baselines.copy()
    bl[0, 1] = 99
    with pytest.raises(idg_mod.IdgError) as e:
        idg_mod.idg_plan_create(g, obs.n_stations, bl, obs.uvw, obs.freqs, obs.aterm_offsets)
    assert e.value.status == 1


def test_empty_observation_plans_to_nothing(idg_mod):
    obs = _brute.tiny_observation(seed=1, n_t=0)
    sg, seg, st = _host_plan(idg_mod, obs)
    assert len(sg) == 0 and len(seg) == 0 and st.n_vis == 0


def test_wait_selftest_rejects_host_plans(idg_mod):
    obs = _brute.tiny_observation(seed=1)
    g, _ = idg_mod.make_geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                                 flags=idg_mod.IDG_HOST_ONLY)
    plan = idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets)
    try:
        with pytest.raises(idg_mod.IdgError) as e:
            idg_mod.idg_wait_selftest(plan, 1000)
        assert e.value.status == 1
    finally:
        idg_mod.idg_plan_destroy(plan)


def test_aterm_nodes_bounds(idg_mod):
    obs = _brute.tiny_observation(seed=1)
    for nodes, ok in ((1, False), (2, True), (25, True), (26, False)):
        g, _ = idg_mod.make_geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                                     aterm_nodes=nodes, flags=idg_mod.IDG_HOST_ONLY)
        if ok:
            idg_mod.idg_plan_destroy(idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs,
                                                             obs.aterm_offsets))
        else:
            with pytest.raises(idg_mod.IdgError) as e:
                idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets)
            assert e.value.status == 1


def _non_coplanar(seed, n_st=16, height=300.0, **kw):
    """An array with station heights of a few hundred metres: |w| exceeds
    the single-layer limit, so planning needs w layers."""
    obs = synth.config(2, seed=seed, n_stations=n_st, n_timesteps=24, **kw)
    rng = np.random.default_rng(seed + 50)
    enu = obs.enu.copy()
    enu[:, 2] = rng.normal(0.0, height, enu.shape[0])
    return synth.make_observation(enu, obs.n_timesteps, 2.0, obs.freqs, 4, obs.grid_size, obs.subgrid_size,
                                  obs.kernel_padding, obs.image_size, name="non-coplanar")


@pytest.mark.parametrize("seed,L", [(0, 96), (1, 64), (2, 128)])
def test_planner_w_layers_bit_exact(idg_mod, oracle_mod, seed, L):
    obs = _non_coplanar(seed)
    with pytest.raises(idg_mod.IdgError) as e:
        _host_plan(idg_mod, obs, 0, L)
    assert e.value.status == 4
    ref = _oracle_plan(oracle_mod, obs, oracle_mod.FLAG_W_LAYERS, L)
    g, _ = idg_mod.make_geometry(obs.grid_size, L, obs.kernel_padding, obs.image_size, aterm_nodes=obs.aterm_nodes,
                                 flags=idg_mod.IDG_W_LAYERS | idg_mod.IDG_HOST_ONLY)
    h = idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets)
    try:
        np.testing.assert_array_equal(idg_mod.idg_plan_subgrids(h), ref.subgrids)
        np.testing.assert_array_equal(idg_mod.idg_plan_segments(h), ref.segments)
        np.testing.assert_array_equal(idg_mod.idg_plan_layers(h), np.stack([ref.layers, ref.conj], axis=1))
        assert ref.conj.any() and not ref.conj.all()
        st = idg_mod.idg_plan_stats(h)
        k_min, n_layers = ref.k_range
        assert (st.w_layer_min, st.n_w_layers) == (k_min, n_layers) and n_layers >= 2
        assert st.w_layer_step == ref.w_step
    finally:
        idg_mod.idg_plan_destroy(h)


def test_aterm_weights_need_a_device_plan_with_the_flag(idg_mod):
    """idg_aterm_weights reads the weights of IDG_NORMALIZE_ATERM device
    plans; a host-only plan (even with the flag) has none."""
    import ctypes
    import numpy as np
    obs = _brute.tiny_observation(seed=2)
    g, _ = idg_mod.make_geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                                 flags=idg_mod.IDG_HOST_ONLY | idg_mod.IDG_NORMALIZE_ATERM)
    plan = idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets)
    try:
        out = np.zeros(obs.subgrid_size ** 2 + 1)
        st = idg_mod.load().idg_aterm_weights(plan, out.ctypes.data_as(ctypes.c_void_p), 0)
        assert st == 1 and not out.any()
    finally:
        idg_mod.idg_plan_destroy(plan)


def test_planner_shrink_golden(idg_mod):
    """The library planner's final shrink on the hand-worked track of
    tests/golden/planner_handworked.json (Section 3.1: corners checked while
    growing, every member after): [0,3) and [3,6)."""
    import json
    gd = json.load(open(os.path.join(ROOT, "tests", "golden", "planner_handworked.json")))
    g, sc = gd["geometry"], gd["shrink_case"]
    xi = np.array(sc["xi"])
    uvw = np.zeros((1, xi.size, 3))
    uvw[0, :, 0] = (xi - g["N"] / 2) * synth.SPEED_OF_LIGHT / sc["f0"]
    geo, _ = idg_mod.make_geometry(g["N"], g["L"], g["P"], g["fov"], flags=idg_mod.IDG_HOST_ONLY)
    h = idg_mod.idg_plan_create(geo, 2, np.array([[0, 1]], np.int32), uvw, np.array([sc["f0"]]),
                                np.array([0, xi.size], np.int32))
    try:
        np.testing.assert_array_equal(idg_mod.idg_plan_subgrids(h), np.array(sc["expected"], np.int32))
    finally:
        idg_mod.idg_plan_destroy(h)


def test_tuning_choices_are_validated_and_reported(idg_mod):
    """grid_chunk (32, 48, 64; 0 = default 48) and degrid_channels (0, 1, 2, 4)
    are checked at plan creation and reported by idg_plan_stats; channel
    groups need uniformly spaced channels and fall back to 1."""
    obs = _brute.tiny_observation(seed=1)
    for chunk, ch, ok in ((0, 0, True), (32, 2, True), (64, 4, True), (8, 1, False), (65, 1, False), (48, 3, False)):
        g, _ = idg_mod.make_geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                                     flags=idg_mod.IDG_HOST_ONLY, grid_chunk=chunk, degrid_channels=ch)
        if ok:
            h = idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets)
            st = idg_mod.idg_plan_stats(h)
            assert st.grid_chunk == (chunk or 48) and st.degrid_channels == (ch or 1)
            idg_mod.idg_plan_destroy(h)
        else:
            with pytest.raises(idg_mod.IdgError) as e:
                idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, obs.freqs, obs.aterm_offsets)
            assert e.value.status == 1
    freqs = obs.freqs.copy()
    freqs[-1] += 0.3e6   # one uneven step
    g, _ = idg_mod.make_geometry(obs.grid_size, obs.subgrid_size, obs.kernel_padding, obs.image_size,
                                 flags=idg_mod.IDG_HOST_ONLY, degrid_channels=4)
    h = idg_mod.idg_plan_create(g, obs.n_stations, obs.baselines, obs.uvw, freqs, obs.aterm_offsets)
    assert idg_mod.idg_plan_stats(h).degrid_channels == 1
    idg_mod.idg_plan_destroy(h)
