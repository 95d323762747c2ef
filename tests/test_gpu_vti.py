"""VTI sweep (Eqs. 1-2, R_xy = 12, R_z = 8, stretched dz) on the GPU against
the FP64 oracle, through the C ABI.  Tolerances as in test_gpu_iso."""
import numpy as np
import pytest

from paper_1410_1387_gb300 import synth
from tests.helpers import max_rel, oracle_problem, rel_l2

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


def vti_small(nx, ny, nz, steps, seed, nb=5, into_q=False, rxy=12, rz=8):
    s = synth.vti_shot(max(nx, ny, nz), nsteps=steps, seed=seed, r_xy=rxy, r_z=rz, with_model=False)
    s.nx, s.ny, s.nz = nx, ny, nz
    s.nb = nb
    s.src = (nx // 2, ny // 3, nz // 2)
    s.src_into_q = into_q
    s.dzk = synth.stretched_dz(nz, s.h, seed)
    s.receivers = synth.receiver_plane(nx, ny, max(nz // 4, 0), stride=2)
    s.v = synth.layered_model(nx, ny, nz, seed)
    s.eps, s.delta = synth.layered_anisotropy(nz, ny, nx, seed)
    return s


def _run(fd, shot, steps):
    g = fd.grid_from_shot(shot, device="cuda:0", nt_cap=steps)
    g.run(steps)
    st = g.state()
    tr = g.traces()
    g.close()
    return st, tr


@pytest.mark.parametrize("shape,steps", [((70, 45, 50), 50), ((33, 90, 41), 40), ((9, 5, 20), 20)])
def test_vti_parity(fd, O, shape, steps):
    shot = vti_small(*shape, steps=steps, seed=21)
    (p, pp, q, qp), tr = _run(fd, shot, steps)
    P = oracle_problem(O, shot)
    pr, ppr, qr, qpr, trr = P.vti_run(shot.v, shot.eps, shot.delta, steps)
    assert max_rel(p, pr) <= 1e-4 and rel_l2(p, pr) <= 1e-4
    assert max_rel(q, qr) <= 1e-4
    G = P.sponge_field()
    assert max_rel(G * pp, ppr) <= 1e-4 and max_rel(G * qp, qpr) <= 1e-4
    assert max_rel(tr, trr) <= 1e-4


def test_vti_reduces_to_iso_on_gpu(fd):
    """eps = delta = 0, source into p and q, radius (4, 4), uniform dz = h:
    p and q equal the isotropic radius-4 run."""
    n, steps = 48, 40
    shot = vti_small(n, n, n, steps, seed=4, nb=6, into_q=True, rxy=4, rz=4)
    shot.dzk = None
    shot.dz = shot.h
    shot.eps = np.zeros_like(shot.v)
    shot.delta = np.zeros_like(shot.v)
    shot.dt = 0.5 * synth.COURANT_LIMIT[4] * shot.h / synth.V_MAX_LAYERED
    (p, _, q, _), tr = _run(fd, shot, steps)
    iso = synth.Shot(name="iso", nx=n, ny=n, nz=n, r_xy=4, r_z=4, h=shot.h, dt=shot.dt, nsteps=steps,
                     nb=shot.nb, src=shot.src, receivers=shot.receivers)
    iso.v = shot.v
    (u, _), tri = _run(fd, iso, steps)
    assert max_rel(p, u) <= 1e-5 and max_rel(q, u) <= 1e-5
    assert max_rel(tr, tri) <= 1e-5


def test_vti_optimized_weights(fd, O):
    """The paper's operator with band-optimised weights (R_xy = 12 at kmax 2.5,
    R_z = 8 at kmax 2.3, uniform dz) against the oracle with its own optimised
    weights."""
    from tests.test_gpu_iso import _weighted_grid
    shot = vti_small(40, 36, 32, 30, seed=6, nb=4)
    shot.dzk, shot.dz = None, shot.h
    g = _weighted_grid(fd, shot, fd.fd_optimized_weights(12, 2.5), fd.fd_optimized_weights(8, 2.3))
    g.run(shot.nsteps)
    p, _, q, _ = g.state()
    tr = g.traces()
    g.close()
    P = oracle_problem(O, shot, weights_xy=O.optimized_weights(12, 2.5), weights_z=O.optimized_weights(8, 2.3))
    pr, _, qr, _, trr = P.vti_run(shot.v, shot.eps, shot.delta, shot.nsteps)
    assert max_rel(p, pr) <= 1e-4 and max_rel(q, qr) <= 1e-4 and max_rel(tr, trr) <= 1e-4


def test_vti_rejects_eps_below_delta(fd):
    shot = vti_small(20, 20, 20, 5, seed=2)
    shot.delta[4, 5, 6] = shot.eps[4, 5, 6] + 0.01
    g = fd.Grid(fd.GridSpec.from_shot(shot), device="cuda:0")
    with pytest.raises(fd.FdError) as e:
        g.set_model(shot.v, shot.eps, shot.delta)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    g.close()


def test_vti_full_size_512_one_step_sampled(fd, O):
    shot = synth.vti_shot(512, nsteps=30)
    g = fd.grid_from_shot(shot, device="cuda:0", nt_cap=30)
    g.run(24)
    p, pp, q, qp = g.state()
    g.step()
    p1, _, q1, _ = g.state()
    g.close()
    P = oracle_problem(O, shot, receivers=False)
    rng = np.random.default_rng(5)
    sx, sy, sz = shot.src
    pts = [rng.integers(0, 512, size=(2000, 3))]
    pts.append(np.array([[sx + a, sy + b, sz + c] for a in range(-13, 14, 2) for b in (-12, 0, 12)
                         for c in (-9, -1, 0, 8)]))
    pts.append(np.array([[i, j, k] for i in (0, 11, 12, 500, 511) for j in (0, 256, 511)
                         for k in (0, 7, 8, 256, 503, 511)]))
    pts = np.concatenate(pts).astype(np.int32)
    sel = (pts[:, 2], pts[:, 1], pts[:, 0])
    G = np.array([P.sponge_at(int(i), int(j), int(k)) for i, j, k in pts])
    wp, wq = P.vti_step_points(shot.v, shot.eps, shot.delta, p, q, pts, G * pp[sel], G * qp[sel], 24)
    assert np.abs(p1[sel] - wp).max() <= 2e-6 * np.abs(p1).max()
    assert np.abs(q1[sel] - wq).max() <= 2e-6 * np.abs(q1).max()


VTI_TILES = [(64, 8, 2), (64, 8, 3), (32, 16, 2), (32, 32, 2)]


@pytest.mark.parametrize("shape", [(70, 45, 50), (33, 90, 41), (97, 66, 23)])
def test_vti_tiles_are_bitwise_identical(fd, shape):
    """Every VTI tile built into the library -- the one-row register forms and
    the two-row form whose q queues live in tensor memory (32 x 32) -- gives the
    same levels and traces bit for bit, with stretched dz, ragged x and y and
    several z chunks (the per-point arithmetic and its order are shared)."""
    steps = 30
    shot = vti_small(*shape, steps=steps, seed=31)
    ref = None
    for tx, ty, la in VTI_TILES:
        for zc in (shape[2], 16):
            g = fd.grid_from_shot(shot, device="cuda:0", nt_cap=steps)
            g.set_launch(tx, ty, zc, la)
            g.run(steps)
            out = (g.state(), g.traces())
            g.close()
            if ref is None:
                ref = out
                assert np.abs(out[1]).max() > 0
                continue
            for a, b in zip(out[0], ref[0]):
                np.testing.assert_array_equal(a, b)
            np.testing.assert_array_equal(out[1], ref[1])


@pytest.mark.parametrize("tile", [(64, 8, 2), (32, 32, 2)])
def test_vti_bounded_wait_reports_timeout(fd, O, tile):
    """Failure detection in the VTI sweep without a fault: CTA (0,0,0) is denied
    one plane's copy of p^n (the test hook), its bounded wait runs out, it
    records the timeout and exits -- in the 32 x 32 form after freeing its
    tensor memory, or the next launches could not allocate -- and fd_sync
    reports FD_ERR_TIMEOUT; a fresh grid in the same context, in the same tile,
    still matches the oracle."""
    import time
    tx, ty, la = tile
    shot = vti_small(48, 40, 36, steps=12, seed=7)
    g = fd.grid_from_shot(shot, device="cuda:0")
    g.set_launch(tx, ty, 36, la)
    fd.fd_debug_skip_copy(g.h, 5)
    t0 = time.perf_counter()
    g.run(1)
    with pytest.raises(fd.FdError) as e:
        g.sync()
    assert e.value.code == fd.FD_ERR_TIMEOUT and "timed out" in str(e.value)
    assert 0.5 < time.perf_counter() - t0 < 30.0
    g.close()
    g = fd.grid_from_shot(shot, device="cuda:0", nt_cap=shot.nsteps)
    g.set_launch(tx, ty, 36, la)
    g.run(shot.nsteps)
    p, _, q, _ = g.state()
    g.close()
    pr, _, qr, _, _ = oracle_problem(O, shot).vti_run(shot.v, shot.eps, shot.delta, shot.nsteps)
    assert max_rel(p, pr) <= 1e-4 and max_rel(q, qr) <= 1e-4
