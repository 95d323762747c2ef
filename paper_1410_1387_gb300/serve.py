"""Continuous-batching shot server over the batch C ABI (fd_batch_*).

Requests arrive over time.  The server admits them in arrival order while
their device memory (the grid arena of fd_required_bytes plus the receiver
traces) fits in an HBM budget, keeps admitted wavefields resident, and each
iteration advances every resident shot by ``steps_per_iter`` steps, one batch
launch per step covering all of them (radius-4 and radius-8 shots each get
their own kernel in the same step).  A shot that has run its steps returns
its traces and frees its memory, and requests that arrived meanwhile are
admitted before the next iteration: work from different requests overlaps on
the GPU instead of queueing behind one another.

``fifo_loop`` is the baseline: one request at a time, in arrival order, each
run to its end with fd_run.  Both produce bit-identical traces per request
(the batch kernel and the single-shot kernel share the per-point arithmetic).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass

import numpy as np

from . import fd, synth
from .batch import Batch


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    points: int
    traces: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def shot_bytes(shot) -> int:
    desc, _ = fd.GridSpec.from_shot(shot).desc()
    return fd.fd_required_bytes(desc) + 256 + 4 * len(shot.receivers) * shot.nsteps


def _open_request(req, device, stream=None):
    """Grid of a request with its model drawn on the GPU, source and receivers,
    all set up on `stream` (None: the current stream)."""
    import torch
    shot = synth.request_shot(req)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    st = torch.cuda.current_stream(dev) if stream is None else stream
    with torch.cuda.device(dev), torch.cuda.stream(st):
        g = fd.Grid(fd.GridSpec.from_shot(shot), device=dev, stream=st)
        v = synth.layered_model_device(req.n, req.seed, dev)
        g.set_model(v)
        del v
        g.add_source(*shot.src, freq_hz=shot.src_f, t0=shot.src_t0, amp=shot.src_amp)
        g.set_receivers(shot.receivers, shot.nsteps)
    return shot, g


def _wait_until(t0, when):
    while True:
        left = when - (time.perf_counter() - t0)
        if left <= 0:
            return
        time.sleep(min(left, 0.002))


class ShotServer:
    """Continuous batching with two admission limits: the HBM budget (bytes of
    every resident shot) and the resident work (grid points of every resident
    shot, `max_points`).  The second keeps just enough shots resident to fill
    the GPU: beyond that, sharing the GPU among more shots only slows each of
    them down (every resident shot advances one step per launch), which raises
    latency without raising throughput.  One shot is always admitted when none
    is resident."""

    def __init__(self, budget_bytes: int, steps_per_iter: int = 25, device=None, launch=None,
                 graph_steps: int = 0, keep_traces: bool = False, max_points: int = 160_000_000):
        self.budget = int(budget_bytes)
        self.max_points = int(max_points)
        self.k = int(steps_per_iter)
        self.device = device
        self.launch = launch or {}
        self.graph_steps = graph_steps
        self.keep = keep_traces
        self.max_resident = 0

    def serve(self, requests, realtime: bool = True):
        """Serve the requests; returns one Result per request (sorted by id).

        The GPU is kept fed: each iteration's batch launches are enqueued
        before the host waits for the previous iteration, new requests are set
        up and finished traces read back on a side stream while the batch
        stream computes.  A shot that ran its last step in iteration i leaves
        the batch before iteration i+1 is enqueued, and its grid is released
        only after iteration i's event."""
        import torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        b = Batch(device=self.device)
        side = torch.cuda.Stream(b.device)
        for r, cfg in self.launch.items():
            b.set_launch(r, *cfg)
        if self.graph_steps:
            b.set_graph(self.graph_steps)
        active = {}                     # grid handle -> (request, grid, shot, bytes, admitted)
        inflight = deque()              # (event after iteration, [finished entries])
        used = 0
        resident_pts = 0
        results = []

        def retire(ev, done):
            nonlocal used, resident_pts
            side.wait_event(ev)
            for req, g, shot, need, adm in done:
                tr = g.traces()                       # on the side stream, after `ev`
                fin = time.perf_counter() - t0
                g.close()
                used -= need
                resident_pts -= shot.points
                results.append(Result(req.rid, req.arrival, adm, fin, shot.points * shot.nsteps,
                                      tr if self.keep else None))

        t0 = time.perf_counter()
        while pending or active or inflight:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                req = pending[0]
                need = shot_bytes(synth.request_shot(req))
                if need > self.budget:
                    raise ValueError(f"request {req.rid} needs {need} bytes, above the whole budget")
                if used + need > self.budget:
                    break
                if (active or inflight) and resident_pts + req.n ** 3 > self.max_points:
                    break
                pending.popleft()
                shot, g = _open_request(req, b.device, side)
                g.arena.record_stream(b.stream)
                g.trace.record_stream(b.stream)
                b.add(g, shot.nsteps)
                active[g.h] = (req, g, shot, need, time.perf_counter() - t0)
                used += need
                resident_pts += shot.points
                now = time.perf_counter() - t0
            self.max_resident = max(self.max_resident, len(active))
            if active:
                b.run(self.k)
                ev = torch.cuda.Event()
                ev.record(b.stream)
                done = []
                for h in list(active):
                    if b.steps_left(active[h][1]) == 0:
                        done.append(active.pop(h))
                        b.remove(done[-1][1])
                inflight.append((ev, done))
            # keep one iteration queued on the GPU while the host waits for the older one
            while inflight and (len(inflight) > 1 or not active):
                ev, done = inflight.popleft()
                ev.synchronize()
                retire(ev, done)
            if not active and not inflight and pending and realtime:
                _wait_until(t0, pending[0].arrival)
        b.close()
        return sorted(results, key=lambda r: r.rid)


def fifo_loop(requests, device=None, realtime: bool = True, keep_traces: bool = False):
    """Baseline: one request at a time in arrival order, each run to its end."""
    import torch
    results = []
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        if realtime:
            _wait_until(t0, req.arrival)
        adm = time.perf_counter() - t0
        shot, g = _open_request(req, device)
        g.run(shot.nsteps)
        tr = g.traces()
        fin = time.perf_counter() - t0
        g.close()
        torch.cuda.synchronize()
        results.append(Result(req.rid, req.arrival, adm, fin, shot.points * shot.nsteps,
                              tr if keep_traces else None))
    return results


def summary(results, wall: float | None = None) -> dict:
    lat = np.array([r.latency for r in results])
    end = max(r.finished for r in results)
    start = min(r.arrival for r in results)
    span = wall if wall is not None else end - start
    pts = sum(r.points for r in results)
    return {"shots": len(results), "shots_per_s": len(results) / span, "points_per_s": pts / span,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "makespan_s": span}
