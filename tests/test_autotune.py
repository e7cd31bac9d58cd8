"""Autotuner selection and cache logic (CPU, injected timings) and one GPU
run on a small observation."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import autotune, synth


def test_selects_fastest_and_caches(tmp_path):
    """Staged search: every (L, mode) with the defaults (tensor-core
    degridder), then the chunk, then the FP32 degridder with 1, 2 or 4
    channels per lane, then the gridder on the tensor cores too; the winner
    is cached per GPU and shape."""
    obs = synth.config(1, n_stations=6)
    calls = []
    T, F, TD = autotune.MAC_TENSOR, autotune.MAC_FP32, autotune.MAC_TENSOR_DEGRID

    def fake(o, L, mode, chunk, ch, mac):
        calls.append((L, mode, chunk, ch, mac))
        if L == 128:
            return None  # e.g. the plan could not be made
        unit = {TD: 0.0, T: -0.02, F: 0.1 + {1: 0.0, 2: -0.05, 4: 0.3}[ch]}[mac]
        return ({64: 5.0, 96: 3.0}[L] + (0.5 if mode == "persistent" else 0.0)
                + {32: 0.2, 48: 0.1, 64: 0.0}[chunk] + unit)

    path = str(tmp_path / "tune.json")
    c = autotune.autotune(obs, cache_path=path, device_name="fake", measure=fake)
    assert (c.subgrid_size, c.mode, c.grid_chunk, c.degrid_channels, c.mac_unit) == (96, "blocks", 64, 1, T)
    assert c.ms == pytest.approx(3.0 - 0.02)
    n = len(calls)
    # stage 1: 3 x 2; stage 2: the two other chunks; stage 3: three FP32 degridders; stage 4: both on tensor cores
    assert n == len(autotune.CANDIDATE_L) * len(autotune.MODES) + 2 + 3 + 1
    assert calls[6:] == [(96, "blocks", 32, 1, TD), (96, "blocks", 64, 1, TD), (96, "blocks", 64, 1, F),
                         (96, "blocks", 64, 2, F), (96, "blocks", 64, 4, F), (96, "blocks", 64, 1, T)]
    c2 = autotune.autotune(obs, cache_path=path, device_name="fake", measure=fake)
    assert len(calls) == n and (c2.grid_chunk, c2.degrid_channels, c2.mac_unit) == (64, 1, T)
    autotune.autotune(obs, cache_path=path, device_name="fake", measure=fake, refresh=True)
    assert len(calls) == 2 * n
    # a different GPU or shape is a different key
    autotune.autotune(obs, cache_path=path, device_name="other", measure=fake)
    assert len(calls) == 3 * n
    import types
    fake_idg = types.SimpleNamespace(IDG_PERSISTENT=8)
    assert c.plan_kwargs(fake_idg) == {"subgrid_size": 96, "flags": 0, "grid_chunk": 64, "degrid_channels": 1,
                                       "mac_unit": T}


def test_no_candidate_raises(tmp_path):
    obs = synth.config(1, n_stations=4)
    with pytest.raises(RuntimeError):
        autotune.autotune(obs, cache_path=None, device_name="fake", measure=lambda *a: None)


@pytest.mark.gpu
def test_gpu_autotune_small(tmp_path, idg_mod, cuda_device):
    obs = synth.config(2, n_stations=10, n_timesteps=8)
    c = autotune.autotune(obs, candidates=(64, 96), cache_path=str(tmp_path / "t.json"))
    assert c.subgrid_size in (64, 96) and c.mode in autotune.MODES and c.ms > 0
    assert c.grid_chunk in autotune.GRID_CHUNKS and c.degrid_channels in autotune.DEGRID_CHANNELS
    assert c.mac_unit in (autotune.MAC_FP32, autotune.MAC_TENSOR, autotune.MAC_TENSOR_DEGRID)
    assert len(c.timings) in (4 + 2 + 3, 4 + 2 + 3 + 1) and all(v is None or v > 0 for v in c.timings.values())
