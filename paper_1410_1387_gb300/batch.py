"""Batched shots and the launch-shape autotuner, over the C ABI (fd_batch_*).

``Batch`` wraps one fd_batch: member grids advance together, one launch per
time step covering every member's tiles.  ``run_batched`` and
``run_per_shot`` run the same list of shots the two ways (the per-shot loop is
the baseline the batch is measured against; both produce bit-identical
traces).  ``Autotuner`` times candidate tile / z-chunk / lookahead choices on
the GPU and caches the winner per (GPU, radius, grid size) in a JSON file.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import fd


class Batch:
    def __init__(self, stream=None, device=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        with torch.cuda.device(self.device):
            self.h = fd.fd_batch_create(self.stream.cuda_stream)
        self.members = {}

    def set_launch(self, radius, tx, ty, zchunk, lookahead):
        fd.fd_batch_set_launch(self.h, radius, tx, ty, zchunk, lookahead)

    def set_graph(self, steps):
        fd.fd_batch_set_graph(self.h, steps)

    def add(self, grid: fd.Grid, nsteps: int):
        fd.fd_batch_add(self.h, grid.h, nsteps)
        self.members[grid.h] = grid

    def remove(self, grid: fd.Grid):
        fd.fd_batch_remove(self.h, grid.h)
        self.members.pop(grid.h, None)

    def steps_left(self, grid: fd.Grid) -> int:
        return fd.fd_batch_steps_left(self.h, grid.h)

    def run(self, max_steps: int) -> int:
        with self.torch.cuda.device(self.device):
            return fd.fd_batch_run(self.h, max_steps)

    def close(self):
        if getattr(self, "h", None):
            with self.torch.cuda.device(self.device):
                fd.fd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_batched(shots, device=None, graph_steps=0, launch=None, keep_grids=False):
    """All shots as one batch until each has run its own step count.  The
    batch runs until a member finishes (64 steps at least), and finished members
    leave before the next run (their work items would otherwise still be
    launched, only to find their shot done).

    Returns (traces per shot, seconds from the first launch to the last trace
    read, grids if keep_grids)."""
    import torch
    grids = [fd.grid_from_shot(s, device=device) for s in shots]
    b = Batch(device=device)
    if launch:
        for radius, cfg in launch.items():
            b.set_launch(radius, *cfg)
    if graph_steps:
        b.set_graph(graph_steps)
    for g, s in zip(grids, shots):
        b.add(g, s.nsteps)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record(b.stream)
    live = list(grids)
    while live:
        # at least 64 steps per run: each change of membership rebuilds the work
        # list and re-captures the graph, so members that finish a little
        # earlier idle until the run ends
        b.run(max(64, min(b.steps_left(g) for g in live)))
        for g in [g for g in live if b.steps_left(g) == 0]:
            b.remove(g)
            live.remove(g)
    ev1.record(b.stream)
    traces = [g.traces() if g.nrec else None for g in grids]
    el = time.perf_counter() - t0
    gpu_s = ev0.elapsed_time(ev1) * 1e-3
    b.close()
    if not keep_grids:
        for g in grids:
            g.close()
        grids = None
    return traces, el, grids, gpu_s


def run_per_shot(shots, device=None, keep_grids=False):
    """The plain loop: one grid after the other, each run to its end.
    Returns (traces, seconds including the trace read-back, grids, GPU seconds
    of the steps alone)."""
    import torch
    grids = [fd.grid_from_shot(s, device=device) for s in shots]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record(grids[0].stream)
    for g, s in zip(grids, shots):
        g.run(s.nsteps)
    ev1.record(grids[0].stream)
    traces = [g.traces() if g.nrec else None for g in grids]
    el = time.perf_counter() - t0
    gpu_s = ev0.elapsed_time(ev1) * 1e-3
    if not keep_grids:
        for g in grids:
            g.close()
        grids = None
    return traces, el, grids, gpu_s


# --------------------------------------------------------------------------
# autotuner
# --------------------------------------------------------------------------

# candidate (tx, ty, lookahead) per radius; every one is built into libfd.so
TILES = {4: [(64, 16, 3), (64, 16, 2), (64, 16, 4), (128, 8, 3), (64, 8, 3), (32, 16, 3), (32, 32, 3), (32, 32, 2)],
         8: [(32, 32, 2), (64, 8, 2), (64, 8, 3), (32, 16, 2)]}
ZCHUNKS = [16, 32, 64, 96, 128]


def _cache_path():
    return os.environ.get("FD_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fdwave", "tune.json"))


class Autotuner:
    """Times launch shapes on the GPU and caches the best per key in JSON."""

    def __init__(self, path=None):
        self.path = path or _cache_path()
        try:
            self.cache = json.load(open(self.path))
        except (OSError, ValueError):
            self.cache = {}

    def _save(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        json.dump(self.cache, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    @staticmethod
    def _gpu():
        import torch
        return torch.cuda.get_device_name().replace(" ", "_")

    def single(self, shot, steps=20, candidates=None):
        """Best (tx, ty, zchunk, lookahead) for fd_run on this shot's grid size."""
        import torch
        key = f"{self._gpu()}|single|R{shot.r_xy}|{shot.nx}x{shot.ny}x{shot.nz}"
        if key in self.cache:
            return tuple(self.cache[key]["launch"])
        g = fd.grid_from_shot(shot, receivers=False)
        best = None
        cands = candidates or [(tx, ty, zc, la) for (tx, ty, la) in TILES[shot.r_xy] for zc in ZCHUNKS
                               if zc <= shot.nz]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for c in cands:
            try:
                g.set_launch(*c)
            except fd.FdError:
                continue
            g.run(2)
            ev0.record(g.stream)
            g.run(steps)
            ev1.record(g.stream)
            torch.cuda.synchronize()
            t = ev0.elapsed_time(ev1) / steps
            if best is None or t < best[0]:
                best = (t, c)
        g.close()
        self.cache[key] = {"launch": list(best[1]), "ms_per_step": best[0]}
        self._save()
        return best[1]

    def batch(self, shots, steps=6, zchunks=(32, 64, 128)):
        """Best {radius: (tx, ty, zchunk, lookahead)} for a batch of these shots."""
        import torch
        radii = sorted({s.r_xy for s in shots})
        sizes = sorted(s.nx * s.ny * s.nz for s in shots)
        key = f"{self._gpu()}|batch|R{radii}|n{len(shots)}|p{sizes[len(sizes) // 2]}"
        if key in self.cache:
            cached = {int(r): tuple(v) for r, v in self.cache[key]["launch"].items()}
            if all((v[0], v[1], v[3]) in TILES.get(r, []) for r, v in cached.items()):
                return cached
        grids = [fd.grid_from_shot(s, receivers=False) for s in shots]
        choice = {}
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for r in radii:
            best = None
            for (tx, ty, la) in TILES[r]:
                for zc in zchunks:
                    b = Batch()
                    b.set_launch(r, tx, ty, zc, la)
                    for g, s in zip(grids, shots):
                        if s.r_xy == r:
                            b.add(g, 2 + steps)
                    b.run(2)
                    ev0.record(b.stream)
                    b.run(steps)
                    ev1.record(b.stream)
                    torch.cuda.synchronize()
                    t = ev0.elapsed_time(ev1) / steps
                    b.close()
                    if best is None or t < best[0]:
                        best = (t, (tx, ty, zc, la))
            choice[r] = best[1]
        for g in grids:
            g.close()
        self.cache[key] = {"launch": {str(r): list(v) for r, v in choice.items()}}
        self._save()
        return choice


def traces_equal(a, b) -> bool:
    return all((x is None and y is None) or np.array_equal(x, y) for x, y in zip(a, b))
