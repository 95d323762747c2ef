"""z slabs of one shot on CPU: the slab bookkeeping, and the rank-to-rank
ghost-plane exchange of ``dist.halo_exchange`` driving the FP64 oracle on two
and three gloo ranks, whose owned planes must equal the unsplit oracle run bit
for bit (a step reads nothing beyond R planes, and the oracle's per-point
arithmetic does not depend on the grid it runs on)."""
import os
import socket

import numpy as np
import pytest

from paper_1410_1387_gb300 import slabs, synth
from tests.helpers import iso_shot, oracle_problem


def test_slab_bounds_cover_the_column_with_ghosts():
    for nz, S, P in [(24, 2, 4), (80, 3, 4), (81, 3, 8), (512, 8, 4), (9, 1, 4), (16, 4, 4)]:
        bs = slabs.slab_bounds(nz, S, P)
        assert len(bs) == S and bs[0].a == 0 and bs[-1].b == nz
        for s, sl in enumerate(bs):
            assert sl.b - sl.a >= P
            assert sl.lo == (sl.a - P if s > 0 else 0) and sl.hi == (sl.b + P if s < S - 1 else nz)
            if s:
                assert sl.a == bs[s - 1].b
                # the windows overlap by 2P planes, as fd_halo_exchange requires
                assert sl.lo == bs[s - 1].hi - 2 * P
        sizes = [sl.b - sl.a for sl in bs]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slabs.slab_bounds(15, 4, 4)
    with pytest.raises(ValueError):
        slabs.slab_bounds(16, 0, 4)


def test_slab_shot_assigns_source_and_receivers_to_the_owner():
    rec = np.array([[1, 2, 3], [4, 5, 20], [6, 7, 12], [8, 9, 11]], dtype=np.int32)
    s = iso_shot(20, 18, 24, 4, 5, seed=3, src=(10, 9, 13), receivers=rec)
    bs = slabs.slab_bounds(24, 2, 4)          # owned [0, 12) and [12, 24)
    p0, k0 = slabs.slab_shot(s, bs[0])
    p1, k1 = slabs.slab_shot(s, bs[1])
    assert p0.src is None and p1.src == (10, 9, 13 - bs[1].lo)
    assert list(k0) == [0, 3] and list(k1) == [1, 2]
    assert p1.receivers[:, 2].tolist() == [20 - bs[1].lo, 12 - bs[1].lo]
    assert p0.nz == bs[0].nz and p1.nz == bs[1].nz
    np.testing.assert_array_equal(p1.v, s.v[bs[1].lo:bs[1].hi])
    with pytest.raises(ValueError):
        vs = synth.vti_shot(n=32, nsteps=2, seed=1)
        slabs.slab_shot(vs, slabs.slab_bounds(32, 2, vs.r_z)[0])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _shot(R):
    rec = synth.receiver_plane(20, 18, 7, stride=3)
    return iso_shot(20, 18, 30 if R == 4 else 36, R, 14, seed=11, src=(9, 8, 16), receivers=rec)


def _oracle_slab_worker(rank, world, port, R, q):
    import torch
    import torch.distributed as dist
    import oracle.oracle as O
    from paper_1410_1387_gb300 import dist as fdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shot = _shot(R)
        P = slabs.z_halo(shot)
        sl = slabs.slab_bounds(shot.nz, world, P)[rank]
        part, keep = slabs.slab_shot(shot, sl)
        prob = oracle_problem(O, part)
        u = np.zeros((part.nz, part.ny, part.nx))
        up = np.zeros_like(u)
        tr = np.zeros((shot.nsteps, len(keep)))
        lower = rank - 1 if rank > 0 else None
        upper = rank + 1 if rank < world - 1 else None
        for n in range(shot.nsteps):
            u, up, t = prob.iso_run(part.v, 1, u, up, n0=n)
            if len(keep):
                tr[n] = t[0]
            fdist.halo_exchange(torch.from_numpy(u), P, lower, upper)
        q.put((rank, sl, u[sl.a - sl.lo:sl.b - sl.lo], up[sl.a - sl.lo:sl.b - sl.lo], keep, tr))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _vti_shot():
    s = synth.vti_shot(24, nsteps=12, seed=5, with_model=False)
    s.nz = 40
    s.dzk, s.dz, s.nb = None, s.h, 0
    s.src = (12, 11, 21)
    s.receivers = synth.receiver_plane(24, 24, 9, stride=3)
    s.v = synth.layered_model(24, 24, 40, 5)
    s.eps, s.delta = synth.layered_anisotropy(40, 24, 24, 5)
    return s


def _oracle_vti_slab_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle.oracle as O
    from paper_1410_1387_gb300 import dist as fdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shot = _vti_shot()
        P = slabs.z_halo(shot)
        sl = slabs.slab_bounds(shot.nz, world, P)[rank]
        part, keep = slabs.slab_shot(shot, sl)
        prob = oracle_problem(O, part)
        z = np.zeros((part.nz, part.ny, part.nx))
        p, pp, qq, qp = z.copy(), z.copy(), z.copy(), z.copy()
        tr = np.zeros((shot.nsteps, len(keep)))
        lower = rank - 1 if rank > 0 else None
        upper = rank + 1 if rank < world - 1 else None
        for n in range(shot.nsteps):
            p, pp, qq, qp, t = prob.vti_run(part.v, part.eps, part.delta, 1, p, pp, qq, qp, n0=n)
            if len(keep):
                tr[n] = t[0]
            fdist.halo_exchange(torch.from_numpy(p), P, lower, upper)
            fdist.halo_exchange(torch.from_numpy(qq), P, lower, upper)
        own = slice(sl.a - sl.lo, sl.b - sl.lo)
        q.put((rank, p[own], qq[own], keep, tr))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_oracle_vti_slabs_over_gloo_match_the_unsplit_run(O):
    """The paper's operator (R_xy = 12, R_z = 8, uniform dz) in two z slabs:
    p and q exchanged, owned planes and traces equal to the unsplit run."""
    import torch.multiprocessing as mp
    shot = _vti_shot()
    pr, _, qr, _, trr = oracle_problem(O, shot).vti_run(shot.v, shot.eps, shot.delta, shot.nsteps)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_vti_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr_ in procs:
        pr_.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for pr_ in procs:
        pr_.join(timeout=60)
        assert pr_.exitcode == 0
    assert np.array_equal(np.concatenate([o[1] for o in out]), pr)
    assert np.array_equal(np.concatenate([o[2] for o in out]), qr)
    tr = np.zeros_like(trr)
    for o in out:
        if len(o[3]):
            tr[:, o[3]] = o[4]
    assert np.array_equal(tr, trr) and np.abs(trr).max() > 0


@pytest.mark.parametrize("R,world", [(4, 2), (4, 3), (8, 2)])
def test_oracle_slabs_over_gloo_match_the_unsplit_run(O, R, world):
    import torch.multiprocessing as mp
    shot = _shot(R)
    u_ref, up_ref, tr_ref = oracle_problem(O, shot).iso_run(shot.v, shot.nsteps)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_slab_worker, args=(r, world, port, R, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u = np.concatenate([o[2] for o in out], axis=0)
    up = np.concatenate([o[3] for o in out], axis=0)
    assert np.array_equal(u, u_ref) and np.array_equal(up, up_ref)
    tr = np.zeros_like(tr_ref)
    for o in out:
        if len(o[4]):
            tr[:, o[4]] = o[5]
    assert np.array_equal(tr, tr_ref)
    assert np.abs(u_ref).max() > 0


def test_step_parts_cover_the_owned_planes():
    """The parts of a slab's step: boundary parts next to each cut that has a
    neighbour (what the neighbour needs as ghosts), the interior, disjoint and
    together exactly the owned planes; no part for the ghost planes."""
    for nz, S, P in [(80, 3, 4), (24, 3, 4), (16, 2, 8), (9, 1, 4), (512, 8, 4), (25, 3, 4)]:
        for s, sl in enumerate(slabs.slab_bounds(nz, S, P)):
            lower, upper = s > 0, s < S - 1
            bnd, interior = slabs.step_parts(sl, P, lower, upper)
            parts = bnd + ([interior] if interior else [])
            planes = sorted(k for k0, k1 in parts for k in range(k0, k1))
            assert planes == list(range(sl.a - sl.lo, sl.b - sl.lo))        # each owned plane once
            need = set()
            if lower:
                need |= set(range(sl.a - sl.lo, sl.a - sl.lo + P))
            if upper:
                need |= set(range(sl.b - sl.lo - P, sl.b - sl.lo))
            assert {k for k0, k1 in bnd for k in range(k0, k1)} == need        # boundary parts: exactly those
            assert all(k1 > k0 for k0, k1 in parts)
