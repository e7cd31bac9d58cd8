"""Autotuner selection and cache logic (CPU, injected timings) and one GPU
run on a small observation."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import autotune, synth


def test_selects_fastest_and_caches(tmp_path):
    obs = synth.config(1, n_stations=6)
    calls = []

    def fake(o, L, mode, budget):
        calls.append((L, mode, budget))
        if L == 128:
            return None  # e.g. the plan could not be made
        return {64: 5.0, 96: 3.0}[L] + (0.5 if mode == "persistent" else 0.0)

    path = str(tmp_path / "tune.json")
    c = autotune.autotune(obs, cache_path=path, device_name="fake", measure=fake)
    assert (c.subgrid_size, c.mode) == (96, "blocks") and c.ms == 3.0
    n = len(calls)
    assert n == len(autotune.CANDIDATE_L) * len(autotune.MODES) * len(autotune.BUDGETS)
    c2 = autotune.autotune(obs, cache_path=path, device_name="fake", measure=fake)
    assert len(calls) == n and (c2.subgrid_size, c2.mode) == (96, "blocks")
    autotune.autotune(obs, cache_path=path, device_name="fake", measure=fake, refresh=True)
    assert len(calls) == 2 * n
    # a different GPU or shape is a different key
    autotune.autotune(obs, cache_path=path, device_name="other", measure=fake)
    assert len(calls) == 3 * n


def test_no_candidate_raises(tmp_path):
    obs = synth.config(1, n_stations=4)
    with pytest.raises(RuntimeError):
        autotune.autotune(obs, cache_path=None, device_name="fake", measure=lambda *a: None)


@pytest.mark.gpu
def test_gpu_autotune_small(tmp_path, idg_mod, cuda_device):
    obs = synth.config(2, n_stations=10, n_timesteps=8)
    c = autotune.autotune(obs, candidates=(64, 96), cache_path=str(tmp_path / "t.json"))
    assert c.subgrid_size in (64, 96) and c.mode in autotune.MODES and c.ms > 0
    assert all(v is None or v > 0 for v in c.timings.values())
