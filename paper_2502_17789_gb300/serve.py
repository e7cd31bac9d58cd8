"""Serving loop: continuous batching of imaging requests on one GPU.

A request grids the visibilities of one snapshot observation (or degrids a
model grid into them).  Requests arrive as a Poisson stream.  The server
admits a request when its device footprint fits the HBM budget and a slot is
free; its plan, visibilities and grid stay resident on the device until its
result has been copied back, then the memory and the slot are released and
the next waiting request is admitted.  Plan creation (host partitioning)
runs on a thread pool so it overlaps GPU work.

Modes:
  "batched"  continuous batching through the library's shared work queue:
             the admitted requests whose plans are ready go to the GPU
             together as a wave -- per kind of work one idg_grid_many or
             idg_degrid_many call, whose launches hold the work items of all
             the wave's requests, longest first -- while the next wave
             collects the requests that arrive meanwhile; two waves are in
             flight at a time, on two streams.
  "streams"  every admitted request runs its own idg_grid / idg_degrid on
             its own stream (requests overlap at the granularity of the
             kernels).
  "plain"    one request at a time on one stream: the per-request baseline.

Results come back through a pool of page-locked host buffers that the
process keeps and reuses (page-locking a buffer of a GiB or more is a slow
host operation, so a server reserves its staging memory once, as it does
its device memory).

Failures stay on the host: a request whose footprint can never fit is
rejected, a cancelled request is skipped, and a plan that cannot be made
(for example IDG_ERR_W_TOO_LARGE) fails that request only.

Every result carries its host planning time, its device time (CUDA events
on its stream) and its pinned-buffer wait, so a run shows where a request's
latency goes.
"""
from __future__ import annotations

import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import idg, synth

GRID_BYTES_PER_CELL = 4 * 16  # complex128, 4 correlations


@dataclass
class Request:
    """One snapshot request.  Its input (visibilities of a grid request, the
    model grid of a degrid request) is synthesised on the device when the
    request is admitted, from `seed` -- a stand-in for data arriving from the
    correlator or left on the GPU by the previous imaging cycle."""
    rid: int
    kind: str                       # "grid" or "degrid"
    obs: synth.Observation
    arrival: float                  # seconds after the start of the stream
    aterms: np.ndarray              # complex64 [n_int][n_st][nodes][nodes][4]
    seed: int = 0
    cancelled: bool = False


@dataclass
class Result:
    rid: int
    kind: str
    status: str                     # "ok", "rejected", "cancelled", "failed: ..."
    n_vis: int = 0
    arrival: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0
    output: np.ndarray | None = None
    plan_s: float = 0.0             # host planning (idg_plan_create, on the planning pool)
    gpu_s: float = 0.0              # device time of the request's work on its stream
    pinned_s: float = 0.0           # time spent obtaining the page-locked result buffer

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def footprint_bytes(req: Request) -> int:
    """Device memory a request holds while resident: its input and output
    arrays, the plan's subgrid scratch (bounded by the 1 GiB batch budget),
    staged records and tables."""
    o = req.obs
    vis = o.n_vis * 32
    grid = o.grid_size * o.grid_size * GRID_BYTES_PER_CELL
    per_sg = 4 * o.subgrid_size ** 2 * 8
    # subgrids <= visibilities; the plan's scratch holds at most 1 GiB of images
    scratch = min(1 << 30, max(1, o.n_vis) * per_sg)
    records = o.n_vis * 128
    tables = o.uvw.nbytes + (64 << 20)
    return int(vis + grid + scratch + records + tables + req.aterms.nbytes)


def request_shape(n_st, n_ch, n_t):
    return n_st * (n_st - 1) // 2 * n_ch * n_t


class PinnedPool:
    """Page-locked host buffers kept for the life of the process and handed
    out again to any request whose result fits (smallest free buffer that is
    large enough; a new one, rounded up to a power of two, only when none
    is)."""

    def __init__(self):
        self._free: list = []
        self._lock = threading.Lock()
        self.allocated_bytes = 0

    def take(self, nbytes: int):
        import torch
        with self._lock:
            fits = [i for i, b in enumerate(self._free) if b.numel() >= nbytes]
            if fits:
                i = min(fits, key=lambda k: self._free[k].numel())
                return self._free.pop(i)
        size = 1 << max(20, int(nbytes - 1).bit_length())
        buf = torch.empty(size, dtype=torch.uint8, pin_memory=True)
        with self._lock:
            self.allocated_bytes += size
        return buf

    def give(self, buf):
        with self._lock:
            self._free.append(buf)


PINNED = PinnedPool()


def _pinned_view(buf, shape, dtype):
    import torch
    n = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
    return buf[:n].view(dtype).view(shape)


@dataclass(eq=False)   # slots compare by identity
class _Slot:
    req: Request
    admitted: float
    future: cf.Future | None = None
    plan: idg.Plan | None = None
    stream: object = None
    event: object = None
    start: object = None
    bufs: dict = field(default_factory=dict)
    host_out: object = None
    host_buf: object = None
    plan_s: float = 0.0
    pinned_s: float = 0.0


class Server:
    def __init__(self, hbm_budget_bytes: int = 64 << 30, max_slots: int = 8, mode: str = "batched",
                 device: int = 0, keep_outputs: bool = True, plan_workers: int = 4):
        import torch

        if mode not in ("batched", "streams", "plain"):
            raise ValueError("mode must be 'batched', 'streams' or 'plain'")
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.max_slots = 1 if mode == "plain" else int(max_slots)
        self.mode = mode
        self.device = torch.device("cuda", device)
        self.keep_outputs = keep_outputs
        self.plan_workers = plan_workers
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.max_slots)]

    # ---------------------------------------------------------------- request lifecycle

    def _make_plan(self, req: Request, stream_handle: int):
        t = time.perf_counter()
        plan = idg.Plan(req.obs, stream=stream_handle)
        return plan, time.perf_counter() - t

    def _launch(self, slot: _Slot):
        torch = self.torch
        with torch.cuda.stream(slot.stream):
            slot.start = torch.cuda.Event(enable_timing=True)
            slot.start.record(slot.stream)
            self._synthesize(slot)
            if slot.req.kind == "grid":
                slot.plan.grid(slot.bufs["vis"], slot.bufs["A"], slot.bufs["G"])
                res = slot.bufs["G"]
            else:
                slot.plan.degrid(slot.bufs["G"], slot.bufs["A"], slot.bufs["vis"])
                res = slot.bufs["vis"]
            out = self._host_buffer(slot, res.shape, res.dtype)
            out.copy_(res, non_blocking=True)
            slot.host_out = out
            slot.event = torch.cuda.Event(enable_timing=True)
            slot.event.record(slot.stream)

    def _host_buffer(self, slot: _Slot, shape, dtype):
        t = time.perf_counter()
        n = int(np.prod(shape)) * self.torch.empty((), dtype=dtype).element_size()
        slot.host_buf = PINNED.take(n)
        slot.pinned_s = time.perf_counter() - t
        return _pinned_view(slot.host_buf, shape, dtype)

    def _synthesize(self, slot: _Slot):
        """Inputs of a request on the current stream: its A-terms, and its
        visibilities (grid) or model grid (degrid), from its seed."""
        torch = self.torch
        req = slot.req
        o = req.obs
        A = torch.as_tensor(req.aterms).to(self.device, non_blocking=True)
        N = o.grid_size
        gen = torch.Generator(device=self.device)
        gen.manual_seed(req.seed)
        if req.kind == "grid":
            vis = torch.randn((o.n_baselines, o.n_timesteps, o.n_channels, 4), dtype=torch.complex64,
                              device=self.device, generator=gen)
            G = torch.zeros((4, N, N), dtype=torch.complex128, device=self.device)
        else:
            u = (torch.arange(N, device=self.device, dtype=torch.float64) - N // 2) / o.image_size
            lm = (torch.rand((4, 2), device=self.device, dtype=torch.float64, generator=gen) - 0.5) \
                * (o.image_size / 1.5)
            amp = torch.randn((4,), dtype=torch.complex128, device=self.device, generator=gen)
            ex = torch.polar(torch.ones_like(u)[None, :].expand(4, N), -2 * np.pi * lm[:, :1] * u[None, :])
            ey = torch.polar(torch.ones_like(u)[None, :].expand(4, N), -2 * np.pi * lm[:, 1:] * u[None, :])
            G = torch.zeros((4, N, N), dtype=torch.complex128, device=self.device)
            G[0] = torch.einsum("s,sy,sx->yx", amp, ey, ex)
            G[3] = G[0]
            vis = torch.empty((o.n_baselines, o.n_timesteps, o.n_channels, 4), dtype=torch.complex64,
                              device=self.device)
        slot.bufs = {"A": A, "vis": vis, "G": G}

    def _launch_wave(self, slots: list[_Slot], stream):
        """One wave.  Each request makes its inputs on its own stream; the
        wave's stream waits for all of them and runs, per kind of work, one
        call whose launches share the work items of the wave's requests;
        each request's stream then copies its result back and records its
        completion event.  Inputs and copies of one wave thus overlap the
        shared launches of others."""
        torch = self.torch
        inputs_ready = []
        for slot in slots:
            with torch.cuda.stream(slot.stream):
                slot.start = torch.cuda.Event(enable_timing=True)
                slot.start.record(slot.stream)
                self._synthesize(slot)
                ev = torch.cuda.Event()
                ev.record(slot.stream)
                inputs_ready.append(ev)
        with torch.cuda.stream(stream):
            for ev in inputs_ready:
                stream.wait_event(ev)
            groups: dict = {}
            for slot in slots:
                st = slot.plan.stats()
                key = (slot.req.kind, int(st.subgrid_size), int(st.degrid_channels), int(st.mac_unit))
                groups.setdefault(key, []).append(slot)
            for (kind, _, _, _), grp in groups.items():
                plans = [sl.plan for sl in grp]
                A = [sl.bufs["A"] for sl in grp]
                if kind == "grid":
                    idg.grid_many(plans, [sl.bufs["vis"] for sl in grp], A, [sl.bufs["G"] for sl in grp],
                                  stream=stream.cuda_stream)
                else:
                    idg.degrid_many(plans, [sl.bufs["G"] for sl in grp], A, [sl.bufs["vis"] for sl in grp],
                                    stream=stream.cuda_stream)
            done = torch.cuda.Event()
            done.record(stream)
        for slot in slots:
            with torch.cuda.stream(slot.stream):
                slot.stream.wait_event(done)
                res = slot.bufs["G"] if slot.req.kind == "grid" else slot.bufs["vis"]
                out = self._host_buffer(slot, res.shape, res.dtype)
                out.copy_(res, non_blocking=True)
                slot.host_out = out
                slot.event = torch.cuda.Event(enable_timing=True)
                slot.event.record(slot.stream)
        return done

    def run(self, requests: list[Request]) -> list[Result]:
        """Serve `requests` (arrival times relative to now); returns one
        Result per request in request order."""
        if self.mode == "batched":
            return self._run_waves(requests)
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: list[Request] = []
        running: list[_Slot] = []
        free_streams = list(self.streams)
        used = 0
        results: dict[int, Result] = {}
        pool = cf.ThreadPoolExecutor(max_workers=self.plan_workers)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        try:
            while pending or queue or running:
                t = now()
                while pending and pending[0].arrival <= t:
                    queue.append(pending.pop(0))
                # admission, first come first served
                while queue and free_streams:
                    req = queue[0]
                    if req.cancelled:
                        queue.pop(0)
                        results[req.rid] = Result(req.rid, req.kind, "cancelled", req.obs.n_vis, req.arrival)
                        continue
                    need = footprint_bytes(req)
                    if need > self.budget:
                        queue.pop(0)
                        results[req.rid] = Result(req.rid, req.kind, "rejected: footprint exceeds the HBM budget",
                                                  req.obs.n_vis, req.arrival)
                        continue
                    if used + need > self.budget:
                        break
                    queue.pop(0)
                    stream = free_streams.pop()
                    slot = _Slot(req, now(), stream=stream)
                    slot.future = pool.submit(self._make_plan, req, stream.cuda_stream)
                    running.append(slot)
                    used += need
                progressed = False
                for slot in list(running):
                    if slot.plan is None and slot.future is not None and slot.future.done():
                        try:
                            slot.plan, slot.plan_s = slot.future.result()
                        except idg.IdgError as e:
                            running.remove(slot)
                            used -= footprint_bytes(slot.req)
                            free_streams.append(slot.stream)
                            results[slot.req.rid] = Result(slot.req.rid, slot.req.kind, f"failed: {e}",
                                                           slot.req.obs.n_vis, slot.req.arrival, slot.admitted,
                                                           now())
                            progressed = True
                            continue
                        self._launch(slot)
                        progressed = True
                    elif slot.event is not None and slot.event.query():
                        slot.plan.synchronize()
                        r = Result(slot.req.rid, slot.req.kind, "ok", slot.req.obs.n_vis, slot.req.arrival,
                                   slot.admitted, now(), slot.host_out.numpy().copy() if self.keep_outputs else None,
                                   plan_s=slot.plan_s, gpu_s=1e-3 * slot.start.elapsed_time(slot.event),
                                   pinned_s=slot.pinned_s)
                        results[r.rid] = r
                        PINNED.give(slot.host_buf)
                        slot.plan.close()
                        slot.bufs.clear()
                        running.remove(slot)
                        used -= footprint_bytes(slot.req)
                        free_streams.append(slot.stream)
                        progressed = True
                if not progressed:
                    time.sleep(0.0002)
        finally:
            pool.shutdown(wait=True)
            torch.cuda.synchronize(self.device)
        return [results[r.rid] for r in requests]


class _Wave:
    """A wave in flight: its stream (free again once `done`, the event after
    its shared launches, has passed) and its requests not yet finished."""

    def __init__(self, stream, done, slots):
        self.stream, self.done, self.slots = stream, done, slots


def _finish(server, slot, now):
    r = Result(slot.req.rid, slot.req.kind, "ok", slot.req.obs.n_vis, slot.req.arrival, slot.admitted, now,
               slot.host_out.numpy().copy() if server.keep_outputs else None, plan_s=slot.plan_s,
               gpu_s=1e-3 * slot.start.elapsed_time(slot.event), pinned_s=slot.pinned_s)
    PINNED.give(slot.host_buf)
    slot.plan.close()
    slot.bufs.clear()
    return r


def _run_waves(self, requests):
    """The batched mode: see the module docstring."""
    torch = self.torch
    pending = sorted(requests, key=lambda r: r.arrival)
    queue: list[Request] = []
    planning: list[_Slot] = []
    ready: list[_Slot] = []
    waves: list[_Wave] = []                  # in flight
    free_streams = [torch.cuda.Stream(self.device) for _ in range(4)]
    request_streams = list(self.streams)     # one per admitted request
    admitted = 0
    used = 0
    results: dict[int, Result] = {}
    pool = cf.ThreadPoolExecutor(max_workers=self.plan_workers)
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    plan_stream = torch.cuda.Stream(self.device)   # plan uploads; every plan synchronises it when made
    try:
        while pending or queue or planning or ready or waves:
            t = now()
            while pending and pending[0].arrival <= t:
                queue.append(pending.pop(0))
            while queue and admitted < self.max_slots:
                req = queue[0]
                if req.cancelled:
                    queue.pop(0)
                    results[req.rid] = Result(req.rid, req.kind, "cancelled", req.obs.n_vis, req.arrival)
                    continue
                need = footprint_bytes(req)
                if need > self.budget:
                    queue.pop(0)
                    results[req.rid] = Result(req.rid, req.kind, "rejected: footprint exceeds the HBM budget",
                                              req.obs.n_vis, req.arrival)
                    continue
                if used + need > self.budget:
                    break
                queue.pop(0)
                slot = _Slot(req, now(), stream=request_streams.pop())
                slot.future = pool.submit(self._make_plan, req, plan_stream.cuda_stream)
                planning.append(slot)
                admitted += 1
                used += need
            progressed = False
            for slot in list(planning):
                if slot.future.done():
                    planning.remove(slot)
                    progressed = True
                    try:
                        slot.plan, slot.plan_s = slot.future.result()
                        ready.append(slot)
                    except idg.IdgError as e:
                        admitted -= 1
                        used -= footprint_bytes(slot.req)
                        request_streams.append(slot.stream)
                        results[slot.req.rid] = Result(slot.req.rid, slot.req.kind, f"failed: {e}",
                                                       slot.req.obs.n_vis, slot.req.arrival, slot.admitted, now())
            for w in list(waves):
                if w.done is not None and w.done.query():   # the shared launches are done: the stream is free
                    free_streams.append(w.stream)
                    w.done = None
                for sl in list(w.slots):
                    if sl.event.query():
                        sl.plan.synchronize()
                        results[sl.req.rid] = _finish(self, sl, now())
                        w.slots = [x for x in w.slots if x is not sl]
                        request_streams.append(sl.stream)
                        admitted -= 1
                        used -= footprint_bytes(sl.req)
                        progressed = True
                if not w.slots and w.done is None:
                    waves = [x for x in waves if x is not w]
            if ready and free_streams:
                stream = free_streams.pop()
                done = self._launch_wave(ready, stream)
                waves.append(_Wave(stream, done, list(ready)))
                ready = []
                progressed = True
            if not progressed:
                time.sleep(0.0002)
    finally:
        pool.shutdown(wait=True)
        torch.cuda.synchronize(self.device)
    return [results[r.rid] for r in requests]


Server._run_waves = _run_waves


# -------------------------------------------------------------------- workload

def make_stream(n_requests: int = 200, seed: int = 0, rate_hz: float = 2.0, stations=(64, 256),
                channels=(8, 48), timesteps=(8, 120), kinds=("grid", "degrid")) -> list[Request]:
    """Poisson stream of snapshot requests mixing the small (512^2, L=32) and
    MWA-like (4096^2, L=96) geometries, half grid half degrid."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        n_st = int(rng.integers(stations[0], stations[1] + 1))
        n_ch = int(rng.integers(channels[0], channels[1] + 1))
        n_t = int(rng.integers(timesteps[0], timesteps[1] + 1))
        kind = kinds[int(rng.integers(0, len(kinds)))]
        geo = int(rng.integers(0, 3))  # 0: small geometry, 1 and 2: MWA-like
        sub = int(rng.integers(0, 1 << 30))
        if geo == 0:
            obs = synth.config(1, seed=sub, n_stations=n_st, n_timesteps=n_t, n_channels=n_ch)
        else:
            obs = synth.config(2, seed=sub, n_stations=n_st, n_timesteps=n_t, n_channels=n_ch)
        r2 = np.random.default_rng(sub)
        A = synth.aterms_random(r2, obs.n_intervals, obs.n_stations, obs.aterm_nodes, leakage=0.05)
        reqs.append(Request(rid, kind, obs, t, A, seed=sub))
    return reqs


def summarize(results: list[Result], t_wall: float | None = None) -> dict:
    ok = [r for r in results if r.status == "ok"]
    lat = np.array([r.latency for r in ok]) if ok else np.array([np.nan])
    span = (max(r.finished for r in ok) - min(r.arrival for r in ok)) if ok else float("nan")
    return {"requests": len(results), "ok": len(ok),
            "rejected": sum(r.status.startswith("rejected") for r in results),
            "failed": sum(r.status.startswith("failed") for r in results),
            "cancelled": sum(r.status == "cancelled" for r in results),
            "vis": int(sum(r.n_vis for r in ok)), "makespan_s": span,
            "throughput_vis_per_s": (sum(r.n_vis for r in ok) / span) if ok else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            # where the time goes, summed over the served requests
            "host_plan_s": float(sum(r.plan_s for r in ok)), "gpu_s": float(sum(r.gpu_s for r in ok)),
            "pinned_wait_s": float(sum(r.pinned_s for r in ok)),
            "per_request": [[r.kind, r.n_vis, round(1e3 * r.plan_s, 1), round(1e3 * r.gpu_s, 1),
                             round(1e3 * (r.admitted - r.arrival), 1), round(1e3 * r.latency, 1)] for r in ok]}


def compare(n_requests: int = 40, seed: int = 0, loads=(0.7, 2.0), budget_gb: float = 64.0, slots: int = 8,
            stations=(64, 256), channels=(8, 48), timesteps=(8, 120), modes=("plain", "batched")) -> dict:
    """Modes side by side on the same Poisson streams.  A calibration pass
    measures the plain capacity on the stream's own mix of requests (its
    first 8, arriving at once); each load is an arrival rate in units of that
    capacity, and load "burst" puts every request at t = 0 (service capacity
    under saturation)."""
    import torch

    torch.cuda.init()
    shape = dict(stations=tuple(stations), channels=tuple(channels), timesteps=tuple(timesteps))
    calib = make_stream(min(8, n_requests), seed=seed, rate_hz=1e9, **shape)
    Server(int(budget_gb * 2**30), mode="plain", keep_outputs=False).run(calib[:1])  # warm-up
    t = time.perf_counter()
    Server(int(budget_gb * 2**30), mode="plain", keep_outputs=False).run(calib)
    cap = len(calib) / (time.perf_counter() - t)
    out = {"calibration_plain_requests_per_s": cap, "shape": shape, "budget_gb": budget_gb, "slots": slots}
    for load in loads:
        burst = load == "burst"
        key = "burst" if burst else f"load_{load:g}"
        rate = 1e9 if burst else load * cap
        out[key] = {"arrival_rate_hz": None if burst else rate}
        for mode in modes:
            stream = make_stream(n_requests, seed=seed, rate_hz=rate, **shape)
            srv = Server(int(budget_gb * 2**30), max_slots=slots, mode=mode, keep_outputs=False)
            out[key][mode] = summarize(srv.run(stream))
            del stream
    return out


def main(argv=None):
    import argparse
    import json

    from . import build

    ap = argparse.ArgumentParser(description="IDG serving benchmark: shared-queue, per-stream and plain forms "
                                             "on one GPU")
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--load", type=float, default=0.7, help="arrival rate as a fraction of plain capacity")
    ap.add_argument("--saturated-load", type=float, default=2.0, help="second, saturating arrival rate")
    ap.add_argument("--modes", nargs="+", default=["plain", "streams", "batched"])
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--stations", type=int, nargs=2, default=(64, 256))
    ap.add_argument("--channels", type=int, nargs=2, default=(8, 48))
    ap.add_argument("--timesteps", type=int, nargs=2, default=(8, 120))
    args = ap.parse_args(argv)
    build.build()
    out = compare(args.requests, args.seed, (args.load, args.saturated_load, "burst"), args.budget_gb, args.slots,
                  args.stations, args.channels, args.timesteps, modes=tuple(args.modes))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
