"""One shot cut into z slabs on one GPU, ghost planes exchanged by the library
after every step: every level and every trace equals the unsplit grid's bit
for bit (isotropic R = 4 and 8 with the damping layer across the cuts, VTI with
uniform dz), and the exchange rejects slabs that do not fit together."""
import numpy as np
import pytest

from paper_1410_1387_gb300 import slabs, synth
from tests.helpers import iso_shot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_1387_gb300 import fd as fdmod
    return fdmod


def _compare(fd, shot, nslabs):
    ref = fd.grid_from_shot(shot, device="cuda:0")
    ref.run(shot.nsteps)
    st_ref, tr_ref = ref.state(), ref.traces()
    ss = slabs.SlabShot(shot, nslabs, device="cuda:0")
    ss.run(shot.nsteps)
    ss.sync()
    st, tr = ss.state(), ss.traces()
    for a, b in zip(st, st_ref):
        assert np.array_equal(a, b)
    assert np.array_equal(tr, tr_ref)
    assert np.abs(st_ref[0]).max() > 0 and np.abs(tr_ref).max() > 0
    ss.close()
    ref.close()


@pytest.mark.parametrize("R,nslabs", [(4, 3), (4, 2), (8, 2)])
def test_iso_slabs_bitwise(fd, R, nslabs):
    nz = 80 if R == 4 else 72
    rec = synth.receiver_plane(64, 48, 30, stride=2)
    shot = iso_shot(64, 48, nz, R, 60, seed=21, nb=10, src=(32, 24, nz // 2 - 1), receivers=rec)
    _compare(fd, shot, nslabs)


def test_vti_slabs_bitwise(fd):
    s = synth.vti_shot(48, nsteps=40, seed=4, with_model=False)
    s.dzk, s.dz, s.nb = None, s.h, 6
    s.src = (24, 20, 23)
    s.receivers = synth.receiver_plane(48, 48, 10, stride=3)
    s.v = synth.layered_model(48, 48, 48, 4)
    s.eps, s.delta = synth.layered_anisotropy(48, 48, 48, 4)
    _compare(fd, s, 2)


def test_exchange_rejects_mismatched_slabs(fd):
    shot = iso_shot(32, 32, 40, 4, 4, seed=2, nb=4)
    ss = slabs.SlabShot(shot, 2, device="cuda:0")
    lo, up = ss.grids
    with pytest.raises(fd.FdError) as e:
        fd.fd_halo_exchange(lo.h, up.h, 3)            # fewer planes than the radius
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FdError) as e:
        fd.fd_halo_exchange(up.h, lo.h, 4)            # wrong order: windows do not overlap
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FdError) as e:
        fd.fd_halo_exchange(lo.h, lo.h, 4)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    lo.run(1)
    with pytest.raises(fd.FdError) as e:
        fd.fd_halo_exchange(lo.h, up.h, 4)            # different time indices
    assert e.value.code == fd.FD_ERR_BAD_STATE
    with pytest.raises(fd.FdError) as e:
        fd.fd_set_z_window(lo.h, 30, 40)              # 24 planes from 30 overrun 40
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    ss.close()
    vs = synth.vti_shot(32, nsteps=2, seed=1)
    g = fd.grid_from_shot(vs, device="cuda:0")
    with pytest.raises(fd.FdError) as e:
        fd.fd_set_z_window(g.h, 0, 64)                # stretched dz
    assert e.value.code == fd.FD_ERR_UNSUPPORTED
    g.close()


@pytest.mark.parametrize("mode", ["iso4", "iso8", "vti"])
def test_step_in_parts_equals_the_whole_step(fd, mode):
    """A step enqueued as parts (fd_step_planes) in any order equals fd_step bit
    for bit: the levels, the lattice receivers, gathered receivers and the
    source (which sits in one part); a part alone leaves the other planes."""
    if mode == "vti":
        shot = synth.vti_shot(40, nsteps=12, seed=6, with_model=False)
        shot.dzk, shot.dz, shot.nb = None, shot.h, 5
        shot.src = (20, 19, 17)
        shot.v = synth.layered_model(40, 40, 40, 6)
        shot.eps, shot.delta = synth.layered_anisotropy(40, 40, 40, 6)
        shot.receivers = synth.receiver_plane(40, 40, 9, stride=3)
    else:
        R = 4 if mode == "iso4" else 8
        rec = np.array([[3, 4, 30], [20, 21, 5], [33, 2, 17], [7, 40, 44]], np.int32)   # gathered (not a lattice)
        shot = iso_shot(41, 44, 52, R, 12, seed=9, nb=5, src=(20, 21, 25), receivers=rec)
    whole = fd.grid_from_shot(shot, device="cuda:0", nt_cap=shot.nsteps + 1)    # one more step below
    parts = fd.grid_from_shot(shot, device="cuda:0", nt_cap=shot.nsteps + 1)
    nz = shot.nz
    cuts = [(17, 31), (0, 17), (31, nz)]            # out of order; the source plane inside one part
    for n in range(shot.nsteps):
        whole.step()
        order = cuts if n % 2 else cuts[::-1]
        for i, (k0, k1) in enumerate(order):
            parts.step_planes(k0, k1, i == len(order) - 1)
    for a, b in zip(whole.state(), parts.state()):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(whole.traces(), parts.traces())
    assert whole.time_index == parts.time_index == shot.nsteps
    assert np.abs(whole.traces()).max() > 0
    # one part alone: its planes step, the others keep their stored older values
    before = parts.state()
    parts.step_planes(5, 9, True)
    after = parts.state()
    whole.step()
    ref = whole.state()
    np.testing.assert_array_equal(after[0][5:9], ref[0][5:9])
    np.testing.assert_array_equal(after[0][:5], before[1][:5])
    np.testing.assert_array_equal(after[0][9:], before[1][9:])
    for bad in ((3, 3), (-1, 4), (0, nz + 1), (7, 2)):
        with pytest.raises(fd.FdError) as e:
            parts.step_planes(*bad, True)
        assert e.value.code == fd.FD_ERR_INVALID_ARG
    whole.close()
    parts.close()


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_shot(mode):
    if mode == "vti":
        s = synth.vti_shot(40, nsteps=30, seed=8, with_model=False)
        s.dzk, s.dz, s.nb = None, s.h, 5
        s.nz = 56
        s.src = (20, 19, 25)
        s.v = synth.layered_model(40, 40, 56, 8)
        s.eps, s.delta = synth.layered_anisotropy(56, 40, 40, 8)
        s.receivers = synth.receiver_plane(40, 40, 8, stride=2)
        return s
    R = 4 if mode == "iso4" else 8
    rec = synth.receiver_plane(48, 40, 12, stride=2)
    return iso_shot(48, 40, 70 if R == 4 else 80, R, 40, seed=13, nb=6, src=(24, 20, 33), receivers=rec)


def _rank_slab_worker(rank, world, port, mode, q):
    import os
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        shot = _rank_shot(mode)
        rs = slabs.RankSlab(shot, rank, world, device="cuda:0")
        rs.run(shot.nsteps)
        rs.grid.sync()
        sl = rs.sl
        st = rs.grid.state()
        own = slice(sl.a - sl.lo, sl.b - sl.lo)
        tr = rs.grid.traces() if len(rs.rec_keep) else None
        q.put((rank, [x[own] for x in st], rs.rec_keep, tr, rs.grid.time_index))
        rs.grid.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode,world", [("iso4", 2), ("iso4", 3), ("iso8", 2), ("vti", 2)])
def test_rank_slabs_on_gloo_ranks_match_the_unsplit_grid(fd, mode, world):
    """RankSlab, the slab-per-process route, driven through libfd.so by gloo
    ranks that share this GPU (each its own process and context; the ghost
    planes travel through pinned host memory while each slab updates its
    interior): every owned plane of both stored levels, every trace and the
    time index equal the unsplit grid's, bit for bit."""
    import torch.multiprocessing as mp
    shot = _rank_shot(mode)
    ref = fd.grid_from_shot(shot, device="cuda:0")
    ref.run(shot.nsteps)
    st_ref, tr_ref = ref.state(), ref.traces()
    ref.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_slab_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for f in range(len(st_ref)):
        np.testing.assert_array_equal(np.concatenate([o[1][f] for o in out], axis=0), st_ref[f])
    tr = np.zeros_like(tr_ref)
    for o in out:
        if len(o[2]):
            tr[:, o[2]] = o[3]
        assert o[4] == shot.nsteps
    np.testing.assert_array_equal(tr, tr_ref)
    assert np.abs(tr_ref).max() > 0


def test_step_parts_between_graph_runs(fd):
    """Parts of a step interleave with graph-replayed runs of the same grid
    (the graphs are kept per level parity): graph runs, a step in two parts,
    graph runs again, an odd number of plain steps, equal fd_step throughout."""
    rec = synth.receiver_plane(40, 36, 10, stride=3)
    shot = iso_shot(40, 36, 44, 4, 30, seed=4, nb=5, src=(20, 18, 22), receivers=rec)
    ref = fd.grid_from_shot(shot, device="cuda:0")
    ref.run(shot.nsteps)
    g = fd.grid_from_shot(shot, device="cuda:0")
    g.set_graph(4)
    g.run(8)
    g.step_planes(0, 20, False)
    g.step_planes(20, 44, True)
    g.run(9)
    g.step_planes(30, 44, False)
    g.step_planes(0, 30, True)
    g.run(11)
    assert g.time_index == ref.time_index == shot.nsteps
    for a, b in zip(g.state(), ref.state()):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(g.traces(), ref.traces())
    g.close()
    ref.close()
