"""Isotropic sweep on the GPU against the FP64 oracle, through the C ABI.

Tolerance (FP32 arithmetic with FP32 accumulation against FP64): one step
rounds each point to ~1e-7 of the field's scale (the kappa-weighted stencil sum
is small next to 2u - u_prev), and the error grows at most linearly with the
step count, so after 200 steps the field error stays within ~2.4e-5 of the
field maximum.  The tests use max |gpu - oracle| <= 1e-4 * max |oracle| per
element and relative L2 <= 1e-4 (the target on the 64^3 case); one step from
identical FP32 state is held to 2e-6 of the field maximum.
"""
import numpy as np
import pytest

from paper_1410_1387_gb300 import synth
from tests.helpers import iso_shot, max_rel, oracle_problem, rel_l2

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


def _run_gpu(fd, shot, nsteps, **kw):
    g = fd.grid_from_shot(shot, device="cuda:0", nt_cap=nsteps)
    for k, v in kw.items():
        getattr(g, k)(*v)
    g.run(nsteps)
    st = g.state()
    tr = g.traces() if g.nrec else None
    g.close()
    return st, tr


def test_parity_64_radius4_200_steps(fd, O):
    shot = synth.parity_shot_64()
    (u, up), tr = _run_gpu(fd, shot, 200)
    P = oracle_problem(O, shot)
    ur, upr, trr = P.iso_run(shot.v, 200)
    assert rel_l2(u, ur) <= 1e-4
    assert max_rel(u, ur) <= 1e-4
    assert rel_l2(tr, trr) <= 1e-4
    assert np.abs(ur).max() > 0 and np.isfinite(u).all()


@pytest.mark.parametrize("R,shape,nb,steps", [
    (4, (70, 45, 37), 6, 60),        # ragged x (not a multiple of 4), several tiles, sponge
    (4, (131, 17, 90), 9, 40),       # more z chunks than one, ragged tile in y
    (8, (66, 50, 41), 7, 60),
    (8, (29, 33, 19), 0, 30),
])
def test_parity_ragged(fd, O, R, shape, nb, steps):
    nx, ny, nz = shape
    rec = synth.receiver_plane(nx, ny, nz // 3, stride=2, x0=1, y0=2)
    shot = iso_shot(nx, ny, nz, R, steps, seed=7 + R, nb=nb, src=(nx // 3, ny // 2, nz // 2),
                    receivers=rec)
    (u, up), tr = _run_gpu(fd, shot, steps)
    P = oracle_problem(O, shot)
    ur, upr, trr = P.iso_run(shot.v, steps)
    assert max_rel(u, ur) <= 1e-4
    assert rel_l2(u, ur) <= 1e-4
    # stored older level: the oracle keeps G * (what the sweep stores)
    assert max_rel(P.sponge_field() * up, upr) <= 1e-4
    assert max_rel(tr, trr) <= 1e-4


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 1), (5, 7, 3), (4, 4, 9), (9, 1, 12)])
@pytest.mark.parametrize("R", [4, 8])
def test_parity_degenerate_grids(fd, O, R, shape):
    nx, ny, nz = shape
    shot = iso_shot(nx, ny, nz, R, 12, seed=3, nb=0, src=(nx // 2, ny // 2, nz // 2),
                    receivers=np.array([[nx - 1, ny - 1, nz - 1], [0, 0, 0]], np.int32),
                    layered=False)
    (u, up), tr = _run_gpu(fd, shot, 12)
    P = oracle_problem(O, shot)
    ur, upr, trr = P.iso_run(shot.v, 12)
    assert max_rel(u, ur) <= 1e-4
    assert max_rel(tr, trr) <= 1e-4


@pytest.mark.parametrize("shape", [(200003, 2, 3), (3, 70001, 2), (2, 3, 300001)])
def test_extreme_aspect_ratios(fd, O, shape):
    """Long thin grids: hundreds of thousands of points along one axis (tens of
    thousands of tiles in x or y, z chunks capped at their maximum in z)."""
    nx, ny, nz = shape
    src = (nx // 2, ny // 2, nz // 2)
    rec = np.array([[nx // 2 + 3 if nx > 10 else 0, ny // 2 + 3 if ny > 10 else 0,
                     nz // 2 + 3 if nz > 10 else 0]], np.int32)
    shot = iso_shot(nx, ny, nz, 4, 8, seed=2, src=src, receivers=rec, layered=False)
    (u, _), tr = _run_gpu(fd, shot, 8)
    ur, _, trr = oracle_problem(O, shot).iso_run(shot.v, 8)
    assert max_rel(u, ur) <= 1e-4 and max_rel(tr, trr) <= 1e-4 and np.abs(ur).max() > 0


def test_grid_beyond_2_to_the_31_points(fd):
    """1024 x 1024 x 2100 points (2.2e9 > 2^31, 26 GiB of arena): after 20 steps
    the values around the source equal, bit for bit, those of a 200^3 grid with
    the same source (the wave has not reached any boundary of either), so every
    offset of the big grid is formed in 64 bits."""
    import torch
    R, steps, c = 4, 20, 40
    h, v, dt = 10.0, 2000.0, 0.5 * synth.COURANT_LIMIT[4] * 10.0 / 2000.0

    def run(nx, ny, nz, src):
        spec = fd.GridSpec(fd.FD_MODE_ISO, nx, ny, nz, R, R, h, h, dt)
        g = fd.Grid(spec, device="cuda:0")
        g.set_model(torch.full((nz, ny, nx), v, dtype=torch.float32, device="cuda:0"))
        g.add_source(*src)
        g.run(steps)
        g.sync()
        sx, sy, sz = src
        u = g.field_view(0)[sz - c:sz + c, sy - c:sy + c, sx - c:sx + c].cpu().numpy()
        g.close()
        del g
        torch.cuda.empty_cache()
        return u

    big = run(1024, 1024, 2100, (512, 512, 1050))
    small = run(200, 200, 200, (100, 100, 100))
    assert np.abs(small).max() > 0
    np.testing.assert_array_equal(big, small)


def test_axis_beyond_the_launch_grid_is_refused(fd):
    """2^20 points along y (the largest axis a description may have) fit the
    default 32-row tiles (32768 of them) but need more than 65535 tiles of 16
    rows: that launch shape is refused instead of launched, and the grid keeps
    its own."""
    import torch
    d, _ = fd.make_desc(fd.FD_MODE_ISO, 1, 1 << 20, 1, 4, 4, 10.0, 10.0, 1e-4)
    nbytes = fd.fd_required_bytes(d)
    arena = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda:0")
    ptr = arena.data_ptr() + (-arena.data_ptr()) % 256
    h = fd.fd_create_grid(d, ptr, nbytes, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(fd.FdError) as e:
        fd.fd_set_launch(h, 64, 16, 64, 3)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    fd.fd_set_launch(h, 32, 32, 64, 3)
    fd.fd_destroy_grid(h)
    d2, _ = fd.make_desc(fd.FD_MODE_ISO, 1, 1, (1 << 20) + 1, 4, 4, 10.0, 10.0, 1e-4)
    with pytest.raises(fd.FdError) as e:
        fd.fd_required_bytes(d2)
    assert e.value.code == fd.FD_ERR_INVALID_ARG


def test_anisotropic_spacing(fd, O):
    shot = iso_shot(40, 36, 33, 4, 50, seed=11, nb=4, dz=7.0)
    (u, up), _ = _run_gpu(fd, shot, 50)
    ur, _, _ = oracle_problem(O, shot).iso_run(shot.v, 50)
    assert max_rel(u, ur) <= 1e-4


def test_receivers_gather_matches_lattice(fd, O):
    shot = iso_shot(48, 40, 30, 4, 30, seed=5, nb=5)
    lattice = synth.receiver_plane(48, 40, 12, stride=3, x0=2, y0=1)
    rng = np.random.default_rng(0)
    scattered = np.stack([rng.integers(0, 48, 50), rng.integers(0, 40, 50), rng.integers(0, 30, 50)],
                         axis=1).astype(np.int32)
    shot.receivers = lattice
    _, tr_lat = _run_gpu(fd, shot, 30)
    shot.receivers = scattered
    (u, _), tr_sc = _run_gpu(fd, shot, 30)
    shot.receivers = lattice
    _, _, trr = oracle_problem(O, shot).iso_run(shot.v, 30)
    assert max_rel(tr_lat, trr) <= 1e-4
    shot.receivers = scattered
    _, _, trs = oracle_problem(O, shot).iso_run(shot.v, 30)
    assert max_rel(tr_sc, trs) <= 1e-4


def test_graph_and_tiles_are_bitwise_identical(fd):
    shot = iso_shot(100, 70, 60, 4, 24, seed=9, nb=8)
    (u0, p0), t0 = _run_gpu(fd, shot, 24)
    (u1, p1), t1 = _run_gpu(fd, shot, 24, set_graph=(8,))
    (u2, p2), t2 = _run_gpu(fd, shot, 24, set_launch=(64, 8, 13, 3))
    (u3, p3), t3 = _run_gpu(fd, shot, 24, set_launch=(128, 8, 60, 3))
    (u4, p4), t4 = _run_gpu(fd, shot, 24, set_launch=(64, 16, 13, 3))
    (u5, p5), t5 = _run_gpu(fd, shot, 24, set_launch=(32, 32, 13, 2))
    for a, b in ((u0, u1), (u0, u2), (u0, u3), (u0, u4), (u0, u5), (p0, p1), (p0, p3), (p0, p4), (p0, p5)):
        np.testing.assert_array_equal(a, b)
    for t in (t2, t4, t5):
        np.testing.assert_array_equal(t0, t)


@pytest.mark.parametrize("launch", [(64, 8, 17, 3), (32, 16, 9, 2), (32, 32, 9, 2)])
def test_radius8_tiles_are_bitwise_identical(fd, O, launch):
    """Radius 8 in other tiles, z chunks and lookaheads, ragged in x, y and z:
    the same values bit for bit, and the oracle's within tolerance."""
    rec = synth.receiver_plane(102, 70, 20, stride=3)
    shot = iso_shot(102, 70, 58, 8, 20, seed=17, nb=8, receivers=rec)
    (u0, p0), t0 = _run_gpu(fd, shot, 20)
    (u1, p1), t1 = _run_gpu(fd, shot, 20, set_launch=launch)
    np.testing.assert_array_equal(u0, u1)
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_array_equal(t0, t1)
    u_ref, _, tr_ref = oracle_problem(O, shot).iso_run(shot.v, 20)
    assert max_rel(u1, u_ref) <= 1e-4 and max_rel(t1, tr_ref) <= 1e-4


def _weighted_grid(fd, shot, w_xy, w_z):
    g = fd.Grid(fd.GridSpec.from_shot(shot), device="cuda:0")
    fd.fd_set_weights(g.h, w_xy, w_z)
    if shot.mode == "vti":
        g.set_model(shot.v, shot.eps, shot.delta)
    else:
        g.set_model(shot.v)
    g.add_source(*shot.src, freq_hz=shot.src_f, t0=shot.src_t0, amp=shot.src_amp, inject_q=shot.src_into_q)
    g.set_receivers(shot.receivers, shot.nsteps)
    return g


def test_optimized_weights_parity(fd, O):
    """Band-optimised weights (Sec. 1; kmax = 2.0 on all axes) installed with
    fd_set_weights: the GPU run matches the oracle run with the oracle's own
    optimised weights, and differs from the Taylor run."""
    shot = iso_shot(48, 40, 36, 4, 60, seed=23, nb=5, receivers=synth.receiver_plane(48, 40, 10, stride=2))
    w = fd.fd_optimized_weights(4, 2.0)
    g = _weighted_grid(fd, shot, w, w)
    g.run(shot.nsteps)
    u, _ = g.state()
    tr = g.traces()
    g.close()
    wo = O.optimized_weights(4, 2.0)
    ur, _, trr = oracle_problem(O, shot, weights_xy=wo, weights_z=wo).iso_run(shot.v, shot.nsteps)
    assert max_rel(u, ur) <= 1e-4 and rel_l2(u, ur) <= 1e-4 and max_rel(tr, trr) <= 1e-4
    (ut, _), _ = _run_gpu(fd, shot, shot.nsteps)
    assert max_rel(ut, ur) > 1e-3


def test_set_weights_errors(fd):
    shot = iso_shot(20, 20, 20, 4, 5, seed=1)
    g = fd.Grid(fd.GridSpec.from_shot(shot), device="cuda:0")
    bad = fd.fd_optimized_weights(4, 2.0)
    bad[2] *= 1.01                                   # no longer exact on quadratics
    with pytest.raises(fd.FdError) as e:
        fd.fd_set_weights(g.h, bad, None)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    g.set_model(shot.v)
    with pytest.raises(fd.FdError) as e:
        fd.fd_set_weights(g.h, fd.fd_optimized_weights(4, 2.0), None)
    assert e.value.code == fd.FD_ERR_BAD_STATE
    g.close()
    v = synth.vti_shot(24, nsteps=2)
    gv = fd.Grid(fd.GridSpec.from_shot(v), device="cuda:0")
    with pytest.raises(fd.FdError) as e:
        fd.fd_set_weights(gv.h, None, fd.fd_optimized_weights(8, 2.0))    # stretched dz
    assert e.value.code == fd.FD_ERR_UNSUPPORTED
    fd.fd_set_weights(gv.h, fd.fd_optimized_weights(12, 2.5), None)
    gv.close()


def test_checkpoint_resume_is_bitwise(fd):
    shot = iso_shot(60, 50, 40, 4, 40, seed=13, nb=6)
    (u_full, p_full), tr_full = _run_gpu(fd, shot, 40)
    g = fd.grid_from_shot(shot, device="cuda:0", nt_cap=40)
    g.run(17)
    cur, prev = g.state()
    n = g.time_index
    g.close()
    g2 = fd.grid_from_shot(shot, device="cuda:0", nt_cap=40)
    fd.fd_set_state(g2.h, cur, prev, ptr_kind=fd.FD_PTR_HOST, time_index=n)
    g2.set_receivers(shot.receivers, 40) if shot.receivers is not None else None
    g2.run(23)
    u2, p2 = g2.state()
    g2.close()
    np.testing.assert_array_equal(u2, u_full)
    np.testing.assert_array_equal(p2, p_full)


def test_error_codes(fd):
    import torch
    shot = iso_shot(20, 20, 20, 4, 5, seed=1)
    g = fd.Grid(fd.GridSpec.from_shot(shot), device="cuda:0")
    with pytest.raises(fd.FdError) as e:
        g.run(1)
    assert e.value.code == fd.FD_ERR_BAD_STATE
    bad = shot.v.copy()
    bad[3, 4, 5] = np.nan
    with pytest.raises(fd.FdError) as e:
        g.set_model(bad)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FdError) as e:
        g.set_model(shot.v * 2.5)       # 2.5x the velocity: dt above the bound
    assert e.value.code == fd.FD_ERR_UNSTABLE_DT
    g.set_model(torch.from_numpy(shot.v).cuda())
    with pytest.raises(fd.FdError) as e:
        g.add_source(20, 0, 0)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    g.set_receivers([[1, 2, 3]], 3)
    g.run(3)
    with pytest.raises(fd.FdError) as e:
        g.run(1)
    assert e.value.code == fd.FD_ERR_OUT_OF_RANGE
    with pytest.raises(fd.FdError) as e:
        g.traces(0, 4)
    assert e.value.code == fd.FD_ERR_OUT_OF_RANGE
    with pytest.raises(fd.FdError) as e:
        g.set_launch(48, 16, 8, 2)
    assert e.value.code == fd.FD_ERR_UNSUPPORTED
    g.run(0)
    g.sync()
    g.close()


@pytest.mark.parametrize("R", [4, 8])
def test_bounded_wait_reports_timeout(fd, O, R):
    """Failure detection without a GPU fault: one CTA is denied one plane's TMA
    copy (the test hook), its bounded wait runs out after about a second, it
    records the timeout and exits; fd_sync reports FD_ERR_TIMEOUT and the
    context keeps working (a fresh grid's run still matches the oracle).  At
    radius 8 the CTA also frees its tensor memory on the way out: a CTA that
    did not would leave the next launches unable to allocate."""
    import time
    shot = iso_shot(64, 32, 40, R, 6, seed=3, nb=4)
    g = fd.grid_from_shot(shot, device="cuda:0")
    with pytest.raises(fd.FdError) as e:
        fd.fd_debug_skip_copy(g.h, 40)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    fd.fd_debug_skip_copy(g.h, 6)         # in the z chunk of CTA (0,0,0), which starts at plane 0
    t0 = time.perf_counter()
    g.run(1)
    with pytest.raises(fd.FdError) as e:
        g.sync()
    assert e.value.code == fd.FD_ERR_TIMEOUT and "timed out" in str(e.value)
    assert 0.5 < time.perf_counter() - t0 < 30.0
    g.close()
    (u, _), tr = _run_gpu(fd, shot, shot.nsteps)
    ur, _, _ = oracle_problem(O, shot).iso_run(shot.v, shot.nsteps)
    assert max_rel(u, ur) <= 1e-4


@pytest.mark.parametrize("R", [4, 8])
def test_full_size_512_one_step_sampled(fd, O, R):
    """The 512^3 layered shot in the benchmark's launch configuration: after 30
    steps, one more GPU step is checked point by point against the oracle's step
    from the same single-precision state."""
    shot = synth.layered_shot(512, R, nsteps=40)
    g = fd.grid_from_shot(shot, device="cuda:0", nt_cap=40)
    g.run(30)
    cur, prev = g.state()
    g.step()
    new, _ = g.state()
    tr = g.traces(30, 1)[0]
    g.close()
    P = oracle_problem(O, shot, receivers=False)
    rng = np.random.default_rng(R)
    sx, sy, sz = shot.src
    pts = [rng.integers(0, 512, size=(3000, 3))]
    pts.append(np.array([[sx + a, sy + b, sz + c] for a in range(-5, 6) for b in (-3, 0, 3) for c in (-4, 0, 4)]))
    pts.append(np.array([[i, j, k] for i in (0, 1, 19, 20, 255, 491, 492, 510, 511)
                         for j in (0, 20, 300, 511) for k in (0, 3, 20, 21, 511)]))
    pts = np.concatenate(pts).astype(np.int32)
    sel = (pts[:, 2], pts[:, 1], pts[:, 0])
    G = np.array([P.sponge_at(int(i), int(j), int(k)) for i, j, k in pts])
    want = P.iso_step_points(shot.v, cur, pts, G * prev[sel].astype(np.float64), 30)
    scale = np.abs(new).max()
    assert scale > 0
    assert np.abs(new[sel] - want).max() <= 2e-6 * scale
    # the receiver plane row of this step is the new level at k = 20
    np.testing.assert_array_equal(tr.reshape(512, 512), new[shot.nb])


@pytest.mark.parametrize("R", [4, 8])
def test_step_from_caller_levels_equals_fd_step(fd, R):
    """fd_step_from: steps between caller-owned pitched levels (out of place,
    and in place with out = prev) equal fd_step on the grid bit for bit, source
    and receivers included; the grid's own levels are left alone."""
    import torch
    rec = synth.receiver_plane(50, 44, 9, stride=2)
    shot = iso_shot(50, 44, 40, R, 12, seed=8, nb=5, src=(25, 22, 20), receivers=rec)
    ref = fd.grid_from_shot(shot, device="cuda:0")
    ref.run(4)
    g = fd.grid_from_shot(shot, device="cuda:0")
    g.run(4)
    own = g.field_view(0).clone()
    a, b = g.field_view(0).clone(), g.field_view(1).clone()
    c = torch.empty_like(a)
    fd.fd_step_from(g.h, a, b, c)      # u^5 into c
    fd.fd_step_from(g.h, c, a, b)      # u^6 into b
    fd.fd_step_from(g.h, b, c, c)      # u^7 in place over u^5
    ref.run(3)
    torch.cuda.synchronize()
    nx = shot.nx
    np.testing.assert_array_equal(c[:, :, :nx].cpu().numpy(), ref.field_view(0)[:, :, :nx].cpu().numpy())
    np.testing.assert_array_equal(b[:, :, :nx].cpu().numpy(), ref.field_view(1)[:, :, :nx].cpu().numpy())
    assert g.time_index == ref.time_index == 7
    np.testing.assert_array_equal(g.traces(), ref.traces())
    assert torch.equal(g.field_view(0), own)
    with pytest.raises(fd.FdError) as e:
        fd.fd_step_from(g.h, a, b, a)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    g.close()
    ref.close()


def test_host_threads_drive_grids_at_once(fd):
    """Four host threads, each creating and running its own grid (radius 4 or
    8, isotropic or VTI) on its own stream at the same time -- first calls,
    launch-attribute and tensor-map caches included -- give the same traces and
    levels bit for bit as the same shots run one after the other."""
    import threading
    import torch
    shots = [iso_shot(40 + 8 * i, 36, 30, 4 if i % 2 == 0 else 8, 20, seed=50 + i, nb=4,
                      receivers=synth.receiver_plane(40 + 8 * i, 36, 6, stride=2)) for i in range(3)]
    v = synth.vti_shot(32, nsteps=20, seed=9, with_model=False)
    v.v = synth.layered_model(32, 32, 32, 9)
    v.eps, v.delta = synth.layered_anisotropy(32, 32, 32, 9)
    shots.append(v)

    def run(shot, stream):
        with torch.cuda.stream(stream):
            g = fd.grid_from_shot(shot, device="cuda:0")
            g.run(shot.nsteps)
            out = (g.state(), g.traces())
            g.close()
        return out

    seq = [run(s, torch.cuda.current_stream()) for s in shots]
    par = [None] * len(shots)
    errs = []

    def worker(i):
        try:
            torch.cuda.set_device(0)
            par[i] = run(shots[i], torch.cuda.Stream())
        except Exception as e:          # surfaced below
            errs.append(e)

    th = [threading.Thread(target=worker, args=(i,)) for i in range(len(shots))]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    for (sa, ta), (sb, tb) in zip(seq, par):
        for a, b in zip(sa, sb):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(ta, tb)
        assert np.abs(ta).max() > 0


@pytest.mark.parametrize("mode,graph,chunk", [("iso", 0, 0), ("iso", 0, 7), ("iso", 4, 5), ("vti", 0, 6)])
def test_run_to_host_streams_the_traces(fd, mode, graph, chunk):
    """fd_run_to_host: the receiver rows it streams to the host while later steps
    compute -- into pinned and into pageable memory, with chunks that do not
    divide the step count, with graphs on -- equal fd_run followed by
    fd_read_receivers bit for bit; a run the trace buffer cannot hold, or one
    without receivers, is refused with nothing enqueued."""
    import torch
    if mode == "iso":
        rec = synth.receiver_plane(52, 40, 7)          # full-rate lattice: 16-byte stores
        shot = iso_shot(52, 40, 36, 4, 60, seed=9, nb=5, src=(26, 20, 18), receivers=rec)
    else:
        shot = synth.vti_shot(40, nsteps=60, seed=4)
        rec = shot.receivers
    ref = fd.grid_from_shot(shot, device="cuda:0", nt_cap=60)
    ref.run(56)
    want = ref.traces()
    g = fd.grid_from_shot(shot, device="cuda:0", nt_cap=60)
    if graph:
        g.set_graph(graph)
    g.run(3)
    pinned = torch.empty((33, len(rec)), dtype=torch.float32).pin_memory()
    g.run_to_host(33, pinned, chunk)
    assert g.time_index == 36
    page = np.empty((20, len(rec)), np.float32)
    fd.fd_run_to_host(g.h, 20, page, chunk)
    assert g.time_index == 56
    np.testing.assert_array_equal(pinned.numpy(), want[3:36])
    np.testing.assert_array_equal(page, want[36:56])
    np.testing.assert_array_equal(g.traces(), want)
    fd.fd_run_to_host(g.h, 0, None, chunk)             # nothing to do
    with pytest.raises(fd.FdError) as e:
        fd.fd_run_to_host(g.h, 5, page, chunk)          # rows 56..60: the buffer holds 60
    assert e.value.code == fd.FD_ERR_OUT_OF_RANGE
    assert g.time_index == 56
    g.close()
    ref.close()
    bare = fd.grid_from_shot(shot, device="cuda:0", receivers=False)
    with pytest.raises(fd.FdError) as e:
        fd.fd_run_to_host(bare.h, 2, page, 0)
    assert e.value.code == fd.FD_ERR_BAD_STATE
    assert bare.time_index == 0
    bare.close()


@pytest.mark.parametrize("mode,R,launch", [("iso", 4, None), ("iso", 4, (64, 16, 17, 3)), ("iso", 8, None),
                                           ("iso", 8, (64, 8, 17, 3)),
                                           ("vti", 12, None), ("vti", 12, (64, 8, 17, 2))])
@pytest.mark.parametrize("lat", [dict(stride=1), dict(stride=1, x0=1, nrx=37), dict(stride=1, x0=4, nrx=6, nry=3),
                                 dict(stride=2, x0=3, y0=1), dict(stride=3, x0=2, y0=2),
                                 dict(stride=5, x0=4, y0=7, nrx=1, nry=1)])
def test_lattice_receivers_record_the_new_level(fd, mode, R, launch, lat):
    """The fused receiver lattice -- 16-byte stores where a thread's 4 points are
    4 aligned receivers, single stores otherwise (offset and ragged lattices,
    strides 2, 3, 5, one receiver) -- records after every step exactly the new
    level (p for VTI) at its points, in lattice order, in the two-row forms (the
    defaults) and the one-row forms."""
    import torch
    n = 40
    rec = synth.receiver_plane(n + (13 if mode == "iso" else 0), n - 2 if mode == "iso" else n, 9, **lat)
    if mode == "iso":
        shot = iso_shot(n + 13, n - 2, 30, R, 6, seed=3, nb=4, src=(8, 4, 10), receivers=rec)
    else:
        shot = synth.vti_shot(n, nsteps=6, seed=3)
        shot.src = (8, 4, 10)      # within three steps of every lattice's points
        shot.receivers = rec
    g = fd.grid_from_shot(shot, device="cuda:0", nt_cap=6)
    if launch:
        g.set_launch(*launch)
    for t in range(6):
        g.step()
        torch.cuda.synchronize()
        f = g.field_view(0)[:, :, :shot.nx].cpu().numpy()
        np.testing.assert_array_equal(g.traces(t, 1)[0], f[rec[:, 2], rec[:, 1], rec[:, 0]])
    assert np.count_nonzero(g.traces()) > 0
    g.close()
