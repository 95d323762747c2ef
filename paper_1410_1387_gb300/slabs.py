"""One shot cut along z into slabs that exchange ghost planes after every step.

A step (Eq. 3 with the stencils of Eqs. 4-5) updates a point from points at
most R planes away in z, so a slab that stores P >= R ghost planes beyond each
cut, refreshed from its neighbours after every step, computes its own planes
exactly as the whole grid would (bit for bit: the per-point arithmetic does
not depend on the grid it sits in).  The damping layer follows the whole
column (``fd_set_z_window``); the source and the receivers belong to the slab
that owns their plane.

Each step updates only the planes a slab owns (``fd_step_planes``): its ghost
planes would be overwritten by the exchange anyway.  ``SlabShot`` runs all
slabs of one shot on one GPU, the exchange done by the library
(``fd_halo_exchange``: device-to-device copies on the slabs' stream).
``RankSlab`` is one slab per process (one per GPU): it updates the owned
planes next to each cut first, posts their point-to-point exchange with the
neighbouring ranks (``dist.halo_exchange_start``), updates its interior while
the planes are in flight, then waits for the exchange.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from . import dist as fdist
from . import fd


@dataclass(frozen=True)
class Slab:
    a: int      # first plane owned (global index)
    b: int      # one past the last plane owned
    lo: int     # first plane stored (a - P, or 0 for the first slab)
    hi: int     # one past the last plane stored (b + P, or nz for the last slab)

    @property
    def nz(self) -> int:
        return self.hi - self.lo


def slab_bounds(nz: int, nslabs: int, halo: int) -> list[Slab]:
    """Split planes [0, nz) into nslabs contiguous slabs of nearly equal size,
    each stored with `halo` ghost planes on every side that has a neighbour."""
    if nslabs < 1 or halo < 1:
        raise ValueError("need at least one slab and one ghost plane")
    base, extra = divmod(nz, nslabs)
    if base < halo:
        raise ValueError(f"{nz} planes in {nslabs} slabs leave fewer than {halo} planes per slab")
    out, a = [], 0
    for s in range(nslabs):
        b = a + base + (1 if s < extra else 0)
        out.append(Slab(a, b, a - halo if s > 0 else 0, b + halo if s < nslabs - 1 else nz))
        a = b
    return out


def step_parts(sl: Slab, halo: int, lower: bool, upper: bool):
    """The owned planes of slab `sl` (local indices) as (boundary parts, interior
    part): the planes next to a cut that has a neighbour, which the neighbour
    needs as ghost planes, and the rest.  Boundary parts that would overlap
    merge; the interior may be empty (None)."""
    a, b = sl.a - sl.lo, sl.b - sl.lo
    bnd = []
    if lower:
        bnd.append([a, a + halo])
    if upper:
        if bnd and bnd[-1][1] >= b - halo:
            bnd[-1][1] = b
        else:
            bnd.append([b - halo, b])
    lo_i = a + (halo if lower else 0)
    hi_i = b - (halo if upper else 0)
    interior = (lo_i, hi_i) if hi_i > lo_i else None
    return [tuple(x) for x in bnd], interior


def z_halo(shot) -> int:
    """Ghost planes a slab of this shot needs: the z radius."""
    return shot.r_z if shot.mode == "vti" else shot.r_xy


def slab_shot(shot, sl: Slab):
    """The part of a synth.Shot that slab `sl` stores, in local indices: model
    planes [lo, hi); the source and receivers only where the slab owns them."""
    if shot.dzk is not None:
        raise ValueError("slabs need a uniform dz")
    cut = (lambda x: None if x is None else np.ascontiguousarray(x[sl.lo:sl.hi]))
    src = None
    if shot.src is not None and sl.a <= shot.src[2] < sl.b:
        src = (shot.src[0], shot.src[1], shot.src[2] - sl.lo)
    rec, keep = None, np.zeros(0, dtype=np.int64)
    if shot.receivers is not None and len(shot.receivers):
        r = np.asarray(shot.receivers)
        keep = np.nonzero((r[:, 2] >= sl.a) & (r[:, 2] < sl.b))[0]
        rec = r[keep].copy()
        rec[:, 2] -= sl.lo
    part = replace(shot, nz=sl.nz, v=cut(shot.v), eps=cut(shot.eps), delta=cut(shot.delta), src=src,
                   receivers=rec if rec is not None and len(rec) else None)
    return part, keep


class SlabShot:
    """A shot advanced as `nslabs` z slabs on one GPU (one stream), with the
    ghost planes exchanged by the library after every step."""

    def __init__(self, shot, nslabs: int, device=None, nt_cap=None):
        self.shot = shot
        self.halo = z_halo(shot)
        self.bounds = slab_bounds(shot.nz, nslabs, self.halo)
        self.grids, self.rec_keep = [], []
        cap = shot.nsteps if nt_cap is None else nt_cap
        for sl in self.bounds:
            part, keep = slab_shot(shot, sl)
            g = fd.Grid(fd.GridSpec.from_shot(part), device=device)
            fd.fd_set_z_window(g.h, sl.lo, shot.nz)
            if part.mode == "vti":
                g.set_model(part.v, part.eps, part.delta)
            else:
                g.set_model(part.v)
            if part.src is not None:
                g.add_source(*part.src, freq_hz=part.src_f, t0=part.src_t0, amp=part.src_amp,
                             inject_q=part.src_into_q)
            if part.receivers is not None:
                g.set_receivers(part.receivers, cap)
            self.grids.append(g)
            self.rec_keep.append(keep)

    def run(self, nsteps: int) -> None:
        """nsteps steps: every slab updates its own planes, then each cut
        exchanges its ghost planes."""
        for _ in range(nsteps):
            for g, sl in zip(self.grids, self.bounds):
                g.step_planes(sl.a - sl.lo, sl.b - sl.lo, True)
            for s in range(len(self.grids) - 1):
                fd.fd_halo_exchange(self.grids[s].h, self.grids[s + 1].h, self.halo)

    def state(self):
        """The whole grid's stored levels, assembled from the slabs' own planes."""
        parts = [g.state() for g in self.grids]
        out = []
        for f in range(len(parts[0])):
            out.append(np.concatenate([p[f][sl.a - sl.lo:sl.b - sl.lo]
                                       for p, sl in zip(parts, self.bounds)], axis=0))
        return tuple(out)

    def traces(self) -> np.ndarray:
        """Receiver traces in the shot's receiver order."""
        nrec = 0 if self.shot.receivers is None else len(self.shot.receivers)
        nt = self.grids[0].time_index
        out = np.zeros((nt, nrec), dtype=np.float32)
        for g, keep in zip(self.grids, self.rec_keep):
            if len(keep):
                out[:, keep] = g.traces()
        return out

    def sync(self):
        for g in self.grids:
            g.sync()

    def close(self):
        for g in self.grids:
            g.close()


class RankSlab:
    """Slab `rank` of a shot split over the ranks of the default process group
    (one GPU each): each step runs locally, then the ghost planes of the new
    level travel point to point to and from the neighbouring ranks."""

    def __init__(self, shot, rank: int, world: int, device=None, nt_cap=None):
        self.shot = shot
        self.halo = z_halo(shot)
        self.bounds = slab_bounds(shot.nz, world, self.halo)
        self.rank, self.world = rank, world
        self.sl = self.bounds[rank]
        part, self.rec_keep = slab_shot(shot, self.sl)
        self.grid = g = fd.Grid(fd.GridSpec.from_shot(part), device=device)
        fd.fd_set_z_window(g.h, self.sl.lo, shot.nz)
        g.set_model(part.v, part.eps, part.delta) if part.mode == "vti" else g.set_model(part.v)
        if part.src is not None:
            g.add_source(*part.src, freq_hz=part.src_f, t0=part.src_t0, amp=part.src_amp,
                         inject_q=part.src_into_q)
        if part.receivers is not None:
            g.set_receivers(part.receivers, shot.nsteps if nt_cap is None else nt_cap)

    def run(self, nsteps: int) -> None:
        """nsteps steps, each: the owned planes next to the cuts, then their
        exchange posted, then the interior while the planes are in flight."""
        lower = self.rank - 1 if self.rank > 0 else None
        upper = self.rank + 1 if self.rank < self.world - 1 else None
        bnd, interior = step_parts(self.sl, self.halo, lower is not None, upper is not None)
        parts = bnd + ([interior] if interior else [])
        # the buffers the step writes: the stored older levels (ISO: u; VTI: p, q)
        fields = (1, 3) if self.shot.mode == "vti" else (1,)
        for _ in range(nsteps):
            new = [self.grid.field_view(f) for f in fields]
            for i, (k0, k1) in enumerate(bnd):
                self.grid.step_planes(k0, k1, i == len(parts) - 1)
            posted = [fdist.halo_exchange_start(v, self.halo, lower, upper) for v in new]
            if interior:
                self.grid.step_planes(interior[0], interior[1], True)
            for p in posted:
                p.wait()
