"""Serving loop: admission, failure handling (host side) and, on the GPU,
that each request's result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_2502_17789_gb300 import serve, synth


def _req(rid, kind="grid", n_st=8, arrival=0.0, seed=None, idx=1, **kw):
    obs = synth.config(idx, seed=rid, n_stations=n_st, **kw)
    A = synth.aterms_identity(obs.n_intervals, obs.n_stations)
    return serve.Request(rid, kind, obs, arrival, A, seed=rid if seed is None else seed)


def test_footprint_grows_with_request():
    small, big = _req(0, n_st=8), _req(1, n_st=32)
    assert serve.footprint_bytes(big) > serve.footprint_bytes(small) > 0


def test_stream_is_poisson_and_seeded():
    a = serve.make_stream(20, seed=3, rate_hz=5.0, stations=(8, 16), channels=(4, 8), timesteps=(4, 8))
    b = serve.make_stream(20, seed=3, rate_hz=5.0, stations=(8, 16), channels=(4, 8), timesteps=(4, 8))
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(x.arrival < y.arrival for x, y in zip(a, a[1:]))
    assert {r.kind for r in a} <= {"grid", "degrid"}


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["batched", "streams"])
def test_same_result_alone_and_in_the_mix(idg_mod, cuda_device, mode):
    """Each result of a mixed stream (grid and degrid, both geometries,
    requests overlapping on the GPU) equals the same request served alone,
    in the wave mode (shared launches) and the stream-per-request mode."""
    reqs = [_req(i, kind=("grid" if i % 2 == 0 else "degrid"), n_st=8 + 2 * i, arrival=0.01 * i,
                 idx=1 if i % 3 else 2, n_timesteps=6) for i in range(8)]
    mixed = serve.Server(hbm_budget_bytes=48 << 30, max_slots=6, mode=mode).run(reqs)
    assert all(r.status == "ok" for r in mixed)
    for r in reqs:
        r.arrival = 0.0
    for r, m in zip(reqs, mixed):
        alone = serve.Server(hbm_budget_bytes=48 << 30, mode="plain").run([r])[0]
        a, b = alone.output, m.output
        if r.kind == "grid":
            assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-5
        else:
            assert np.sqrt(np.mean(np.abs(a - b) ** 2)) / np.abs(a).max() < 1e-5
    s = serve.summarize(mixed)
    assert s["ok"] == 8 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["batched", "streams"])
def test_rejection_cancellation_and_failed_plans(idg_mod, cuda_device, mode):
    ok = _req(0, n_st=6)
    too_big = _req(1, n_st=6)
    cancelled = _req(2, n_st=6)
    cancelled.cancelled = True
    bad = _req(3, n_st=6)
    bad.obs.uvw = bad.obs.uvw.copy()
    bad.obs.uvw[..., 2] = 5000.0  # w fringe too wide: the plan fails
    budget = serve.footprint_bytes(ok) + 1
    srv = serve.Server(hbm_budget_bytes=budget, max_slots=2, mode=mode)
    too_big.obs = synth.config(2, seed=1, n_stations=6)  # 4096^2 grid: needs more than the budget
    res = srv.run([ok, too_big, cancelled, bad])
    assert res[0].status == "ok"
    assert res[1].status.startswith("rejected")
    assert res[2].status == "cancelled"
    assert res[3].status.startswith("failed") and "W_TOO_LARGE" in res[3].status
