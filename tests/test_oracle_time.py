"""Pins of the oracle's time stepping (Eq. 3 with the source, damping layer and
receivers) to facts outside the oracle.

* plane-wave dispersion: a discrete plane wave with sin^2(w dt/2) = (v dt/2)^2
  sum_a K(k_a) is advanced exactly (isotropic, and the 2x2 VTI system);
* discrete energy conservation without damping or source;
* a dense-matrix NumPy recurrence (literal Cerjan damping, source, receivers)
  on a tiny grid;
* closed forms with v = 0: the injected source sums as sum_m (N-m) dt^2 s_m / V,
  the damping layer decays a constant as G^n;
* VTI with eps = delta = 0 and the source in p and q equals the isotropic run;
* the leapfrog stability boundary at 0.99 / 1.01 times the Courant limit.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from tests.test_oracle_weights import _moment_solve


def _K(theta, R):
    """Symbol of the exact rational stencil: -(c_0 + 2 sum c_l cos(l theta))."""
    c = [float(w) for w in _moment_solve(R)]
    return -(c[0] + 2 * sum(c[l] * math.cos(l * theta) for l in range(1, R + 1)))


def test_iso_plane_wave_dispersion(O):
    R, n, steps = 4, 40, 3
    h, v = 10.0, 2000.0
    dt = 0.4 * O.iso_courant_limit(R) * h / v
    th = np.array([0.7, 0.4, 1.1])             # k_a h
    lam = (v * dt / h) ** 2 * sum(_K(t, R) for t in th)
    w = 2.0 * math.asin(math.sqrt(lam) / 2.0) / dt
    i = np.arange(n)
    phase = (th[2] * i[:, None, None] + th[1] * i[None, :, None] + th[0] * i[None, None, :])
    u0 = np.cos(phase)
    um1 = np.cos(phase + w * dt)
    P = O.Problem(n, n, n, r_xy=R, h=h, dt=dt)
    vv = np.full((n, n, n), v)
    u, up, _ = P.iso_run(vv, steps, u=u0, uprev=um1, traces=False)
    s = slice(R * steps, n - R * steps)
    np.testing.assert_allclose(u[s, s, s], np.cos(phase - steps * w * dt)[s, s, s], atol=2e-12)
    np.testing.assert_allclose(up[s, s, s], np.cos(phase - (steps - 1) * w * dt)[s, s, s], atol=2e-12)


def test_iso_plane_wave_dispersion_custom_weights(O):
    """The same closed form with caller-supplied weights (band-optimised, and
    different on x-y and z): the symbol is the one of those weights."""
    R, n, steps = 4, 40, 3
    h, v = 10.0, 2000.0
    dt = 0.35 * O.iso_courant_limit(R) * h / v
    wxy, wz = O.optimized_weights(R, 2.0), O.optimized_weights(R, 1.2)
    K = lambda c, t: -(c[0] + 2 * sum(c[l] * math.cos(l * t) for l in range(1, R + 1)))  # noqa: E731
    th = np.array([0.7, 0.4, 1.1])             # k_a h
    lam = (v * dt / h) ** 2 * (K(wxy, th[0]) + K(wxy, th[1]) + K(wz, th[2]))
    w = 2.0 * math.asin(math.sqrt(lam) / 2.0) / dt
    i = np.arange(n)
    phase = (th[2] * i[:, None, None] + th[1] * i[None, :, None] + th[0] * i[None, None, :])
    P = O.Problem(n, n, n, r_xy=R, h=h, dt=dt, weights_xy=wxy, weights_z=wz)
    u, up, _ = P.iso_run(np.full((n, n, n), v), steps, u=np.cos(phase), uprev=np.cos(phase + w * dt),
                         traces=False)
    s = slice(R * steps, n - R * steps)
    np.testing.assert_allclose(u[s, s, s], np.cos(phase - steps * w * dt)[s, s, s], atol=2e-12)
    # Taylor weights passed explicitly give the default run exactly
    u0 = np.cos(phase)
    a = O.Problem(n, n, n, r_xy=R, h=h, dt=dt).iso_run(np.full((n, n, n), v), 2, u=u0, traces=False)[0]
    tw = O.taylor_weights(R)
    b = O.Problem(n, n, n, r_xy=R, h=h, dt=dt, weights_xy=tw, weights_z=tw).iso_run(
        np.full((n, n, n), v), 2, u=u0, traces=False)[0]
    assert np.array_equal(a, b)


def test_vti_plane_wave_dispersion(O):
    rxy, rz, n, steps = 4, 2, 36, 2
    h, dz = 10.0, 8.0
    vz, eps, delta = 2500.0, 0.2, 0.08
    dt = 4e-4
    th = np.array([0.6, 0.9, 0.5])     # k_x h, k_y h, k_z dz
    Kh = (_K(th[0], rxy) + _K(th[1], rxy)) / h ** 2
    Kz = _K(th[2], rz) / dz ** 2
    kx, kn, kz = vz ** 2 * (1 + 2 * eps) * dt ** 2, vz ** 2 * (1 + 2 * delta) * dt ** 2, vz ** 2 * dt ** 2
    M = np.array([[kx * Kh, kz * Kz], [kn * Kh, kz * Kz]])
    lam, vec = np.linalg.eig(M)
    m = int(np.argmax(lam.real))
    lam, (P0, Q0) = lam[m].real, vec[:, m].real
    w = 2.0 * math.asin(math.sqrt(lam) / 2.0) / dt
    i = np.arange(n)
    phase = (th[2] * i[:, None, None] + th[1] * i[None, :, None] + th[0] * i[None, None, :])
    Pb = O.Problem(n, n, n, r_xy=rxy, r_z=rz, h=h, dz=dz, dt=dt)
    shp = (n, n, n)
    p, pp, q, qp, _ = Pb.vti_run(np.full(shp, vz), np.full(shp, eps), np.full(shp, delta), steps,
                                 p=P0 * np.cos(phase), pprev=P0 * np.cos(phase + w * dt),
                                 q=Q0 * np.cos(phase), qprev=Q0 * np.cos(phase + w * dt),
                                 traces=False)
    s = slice(rxy * steps, n - rxy * steps)
    np.testing.assert_allclose(p[s, s, s], (P0 * np.cos(phase - steps * w * dt))[s, s, s], atol=1e-11)
    np.testing.assert_allclose(q[s, s, s], (Q0 * np.cos(phase - steps * w * dt))[s, s, s], atol=1e-11)


def test_energy_conservation(O):
    R, n, steps = 4, 24, 200
    h = 10.0
    rng = np.random.default_rng(2)
    v = rng.uniform(1500.0, 3000.0, size=(n, n, n))
    dt = 0.5 * O.iso_courant_limit(R) * h / v.max()
    i = np.arange(n) - n / 2
    g = np.exp(-(i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2) / 8.0)
    P = O.Problem(n, n, n, r_xy=R, h=h, dt=dt)

    def energy(un1, un):
        return (np.sum((un1 - un) ** 2 / (v * v * dt * dt)) - np.sum(un1 * P.iso_laplacian(un)))

    u, up = g.copy(), g.copy()
    u1, u0, _ = P.iso_run(v, 1, u=u, uprev=up, traces=False)
    E0 = energy(u1, u0)
    assert E0 > 0
    u, up, _ = P.iso_run(v, steps, u=u1, uprev=u0, n0=1, traces=False)
    E1 = energy(u, up)
    assert abs(E1 - E0) <= 1e-10 * E0
    assert np.abs(u).max() > 1e-3   # the pulse is still on the grid


def _brute_iso(nx, ny, nz, R, h, dz, dt, v, nb, a, src, f, t0, amp, vol, rec, nsteps):
    """Dense-matrix NumPy recurrence with literal Cerjan damping of both levels."""
    c = [float(w) for w in _moment_solve(R)]
    N = nx * ny * nz
    A = np.zeros((N, N))
    lin = lambda i, j, k: i + nx * (j + ny * k)  # noqa: E731
    G = np.ones(N)
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        r = lin(i, j, k)
        A[r, r] += c[0] * (2.0 / h ** 2 + 1.0 / dz ** 2)
        for l in range(1, R + 1):
            for (di, dj, dk, w) in [(l, 0, 0, h), (-l, 0, 0, h), (0, l, 0, h), (0, -l, 0, h),
                                    (0, 0, l, dz), (0, 0, -l, dz)]:
                ii, jj, kk = i + di, j + dj, k + dk
                if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                    A[r, lin(ii, jj, kk)] += c[l] / w ** 2
        g = 1.0
        for (x, n_) in ((i, nx), (j, ny), (k, nz)):
            d = nb - x if x < nb else (x - (n_ - nb - 1) if x >= n_ - nb else 0)
            g *= math.exp(-(a * d) ** 2)
        G[r] = g
    kap = (v.ravel() * dt) ** 2
    u = np.zeros(N)
    up = np.zeros(N)
    tr = np.zeros((nsteps, len(rec)))
    for n in range(nsteps):
        tau = n * dt - t0
        s = amp * (1 - 2 * (math.pi * f * tau) ** 2) * math.exp(-(math.pi * f * tau) ** 2)
        un = 2 * u - up + kap * (A @ u)
        un[lin(*src)] += dt * dt * s / vol
        un *= G
        u = u * G
        tr[n] = [un[lin(*r)] for r in rec]
        up, u = u, un
    return u.reshape(nz, ny, nx), up.reshape(nz, ny, nx), tr


def test_brute_force_recurrence(O):
    nx, ny, nz, R = 9, 8, 7, 2
    h, dz = 10.0, 12.0
    rng = np.random.default_rng(4)
    v = rng.uniform(1500.0, 2500.0, size=(nz, ny, nx))
    dt = 1.5e-3
    nb, a = 2, 0.2
    src, f, t0, amp = (4, 3, 3), 15.0, 1.0 / 15.0, 3.0
    rec = [(1, 1, 1), (4, 3, 3), (8, 7, 6), (0, 5, 2)]
    nsteps = 40
    bu, bup, btr = _brute_iso(nx, ny, nz, R, h, dz, dt, v, nb, a, src, f, t0, amp, h * h * dz, rec, nsteps)
    P = O.Problem(nx, ny, nz, r_xy=R, h=h, dz=dz, dt=dt, nb=nb, sponge_a=a, src=src, src_f=f,
                  src_t0=t0, src_amp=amp, receivers=rec)
    u, up, tr = P.iso_run(v, nsteps)
    scale = np.abs(bu).max()
    assert scale > 0
    np.testing.assert_allclose(u, bu, atol=1e-13 * scale, rtol=0)
    np.testing.assert_allclose(up, bup, atol=1e-13 * scale, rtol=0)
    np.testing.assert_allclose(tr, btr, atol=1e-13 * scale, rtol=0)


def test_source_closed_form(O):
    # v = 0: no coupling, u^N(src) = sum_{m<N} (N - m) dt^2 s(m dt - t0) / V
    n, N = 5, 60
    h, dz, dt, f, t0, amp = 10.0, 10.0, 1e-3, 15.0, 1.0 / 15.0, 2.0
    P = O.Problem(n, n, n, r_xy=2, h=h, dz=dz, dt=dt, src=(2, 2, 2), src_f=f, src_t0=t0,
                  src_amp=amp, receivers=[(2, 2, 2)])
    u, up, tr = P.iso_run(np.zeros((n, n, n)), N)
    rk = lambda t: (1 - 2 * (math.pi * f * t) ** 2) * math.exp(-(math.pi * f * t) ** 2)  # noqa: E731
    want = sum((N - m) * dt * dt * amp * rk(m * dt - t0) / (h * h * dz) for m in range(N))
    assert u[2, 2, 2] == pytest.approx(want, rel=1e-13)
    assert np.count_nonzero(u) == 1
    # trace row m holds u^{m+1} at the receiver
    want_tr = [sum((M - m) * dt * dt * amp * rk(m * dt - t0) / (h * h * dz) for m in range(M))
               for M in range(1, N + 1)]
    np.testing.assert_allclose(tr[:, 0], want_tr, rtol=1e-12)
    # Ricker: unit peak at t0, zero crossings at t0 +- 1/(pi f sqrt 2)
    assert O.ricker(0.0, f) == 1.0
    assert abs(O.ricker(1.0 / (math.pi * f * math.sqrt(2.0)), f)) < 1e-15


def test_sponge_closed_form(O):
    # v = 0, u^0 = u^{-1} = 1: the undamped solution stays 1, Cerjan gives G^n
    nx, ny, nz = 12, 9, 10
    nb, a, N = 3, 0.3, 7
    P = O.Problem(nx, ny, nz, r_xy=2, h=1.0, dt=1.0, nb=nb, sponge_a=a)
    one = np.ones((nz, ny, nx))
    u, up, _ = P.iso_run(np.zeros_like(one), N, u=one, uprev=one, traces=False)
    G = P.sponge_field()
    np.testing.assert_allclose(u, G ** N, rtol=1e-14)
    np.testing.assert_allclose(up, G ** N, rtol=1e-14)
    # the layer: d counted from the inner edge, 1 at the innermost layer cell
    assert O.sponge_axis(nb - 1, nx, nb, a) == pytest.approx(math.exp(-a * a), rel=1e-15)
    assert O.sponge_axis(0, nx, nb, a) == pytest.approx(math.exp(-(a * nb) ** 2), rel=1e-15)
    assert O.sponge_axis(nx - 1, nx, nb, a) == O.sponge_axis(0, nx, nb, a)
    assert O.sponge_axis(nx - nb, nx, nb, a) == O.sponge_axis(nb - 1, nx, nb, a)
    assert O.sponge_axis(nb, nx, nb, a) == 1.0 and O.sponge_axis(nx - nb - 1, nx, nb, a) == 1.0


def test_vti_reduces_to_iso(O):
    n, R, steps = 20, 4, 30
    h = 10.0
    rng = np.random.default_rng(8)
    v = rng.uniform(1500.0, 3000.0, size=(n, n, n))
    dt = 0.5 * O.iso_courant_limit(R) * h / v.max()
    rec = [(3, 4, 5), (10, 10, 10)]
    kw = dict(r_xy=R, r_z=R, h=h, dt=dt, nb=4, sponge_a=0.05, src=(9, 10, 11), receivers=rec)
    Pi = O.Problem(n, n, n, **kw)
    u, up, tri = Pi.iso_run(v, steps)
    Pv = O.Problem(n, n, n, src_into_q=True, **kw)
    z = np.zeros_like(v)
    p, pp, q, qp, trv = Pv.vti_run(v, z, z, steps)
    scale = np.abs(u).max()
    np.testing.assert_allclose(p, u, atol=1e-13 * scale, rtol=0)
    np.testing.assert_allclose(q, u, atol=1e-13 * scale, rtol=0)
    np.testing.assert_allclose(trv, tri, atol=1e-13 * scale, rtol=0)


@pytest.mark.parametrize("factor,grows", [(0.99, False), (1.01, True)])
def test_stability_boundary(O, factor, grows):
    R, n, steps = 4, 48, 300
    h, v = 10.0, 2000.0
    dt = factor * O.iso_courant_limit(R) * h / v
    u0 = np.random.default_rng(9).standard_normal((n, n, n))
    P = O.Problem(n, n, n, r_xy=R, h=h, dt=dt)
    u, _, _ = P.iso_run(np.full((n, n, n), v), steps, u=u0, uprev=u0, traces=False)
    m = np.abs(u).max()
    if grows:
        assert m > 1e6
    else:
        assert m < 1e3


def test_step_points_match_run(O):
    nx, ny, nz, R = 21, 17, 15, 4
    h = 10.0
    rng = np.random.default_rng(12)
    v = rng.uniform(1500.0, 4500.0, size=(nz, ny, nx)).astype(np.float32)
    dt = 0.5 * O.iso_courant_limit(R) * h / 4500.0
    P = O.Problem(nx, ny, nz, r_xy=R, h=h, dt=dt, nb=3, sponge_a=0.1, src=(10, 8, 7))
    u, up, _ = P.iso_run(v, 25, traces=False)
    u32 = u.astype(np.float32)
    u1, _, _ = P.iso_run(v, 1, u=u32.astype(np.float64), uprev=up, n0=25, traces=False)
    pts = np.array([[i, j, k] for k in (0, 7, 14) for j in (0, 8, 16) for i in (0, 10, 20)], np.int32)
    got = P.iso_step_points(v, u32, pts, up[pts[:, 2], pts[:, 1], pts[:, 0]], 25)
    np.testing.assert_allclose(got, u1[pts[:, 2], pts[:, 1], pts[:, 0]], rtol=1e-13, atol=1e-20)


def test_vti_step_points_match_run(O):
    nx, ny, nz = 30, 28, 26
    h = 10.0
    rng = np.random.default_rng(13)
    vz = rng.uniform(1500.0, 3000.0, size=(nz, ny, nx)).astype(np.float32)
    eps = rng.uniform(0.0, 0.2, size=vz.shape).astype(np.float32)
    delta = (eps * rng.uniform(0, 1, size=vz.shape)).astype(np.float32)
    dzk = h * (1 + 0.1 * np.sin(np.arange(nz - 1)))
    P = O.Problem(nx, ny, nz, r_xy=12, r_z=8, h=h, dzk=dzk, dt=3e-4, nb=3, sponge_a=0.1,
                  src=(15, 14, 13))
    p, pp, q, qp, _ = P.vti_run(vz, eps, delta, 20, traces=False)
    p32, q32 = p.astype(np.float32), q.astype(np.float32)
    p1, _, q1, _, _ = P.vti_run(vz, eps, delta, 1, p=p32, pprev=pp, q=q32, qprev=qp, n0=20, traces=False)
    pts = np.array([[i, j, k] for k in (0, 13, 25) for j in (0, 14, 27) for i in (0, 15, 29)], np.int32)
    sel = (pts[:, 2], pts[:, 1], pts[:, 0])
    gp, gq = P.vti_step_points(vz, eps, delta, p32, q32, pts, pp[sel], qp[sel], 20)
    np.testing.assert_allclose(gp, p1[sel], rtol=1e-12, atol=1e-20)
    np.testing.assert_allclose(gq, q1[sel], rtol=1e-12, atol=1e-20)


def test_receivers_sample_new_level(O):
    n, R, steps = 14, 2, 12
    rec = [(3, 4, 5), (7, 7, 7), (0, 13, 6)]
    P = O.Problem(n, n, n, r_xy=R, h=10.0, dt=1e-3, nb=2, sponge_a=0.1, src=(7, 7, 7), receivers=rec)
    v = np.full((n, n, n), 2000.0)
    _, _, tr = P.iso_run(v, steps)
    u = up = None
    for s in range(steps):
        u, up, _ = P.iso_run(v, 1, u=u, uprev=up, n0=s, traces=False)
        np.testing.assert_array_equal(tr[s], [u[k, j, i] for (i, j, k) in rec])


def test_vti_receivers_sample_new_p(O):
    """VTI traces are p^{n+1} at the receivers (p, the field the paper records;
    with eps != delta q differs from it)."""
    n, steps = 16, 10
    rec = [(3, 4, 5), (8, 8, 9), (0, 15, 6)]
    P = O.Problem(n, n, n, r_xy=4, r_z=2, h=10.0, dt=5e-4, nb=2, sponge_a=0.1, src=(8, 8, 8), receivers=rec)
    v = np.full((n, n, n), 2000.0)
    eps, delta = np.full_like(v, 0.2), np.full_like(v, 0.05)
    *_, tr = P.vti_run(v, eps, delta, steps)
    p = pp = q = qp = None
    for s in range(steps):
        p, pp, q, qp, _ = P.vti_run(v, eps, delta, 1, p=p, pprev=pp, q=q, qprev=qp, n0=s, traces=False)
        np.testing.assert_array_equal(tr[s], [p[k, j, i] for (i, j, k) in rec])
    pr, qr = np.array([p[k, j, i] for (i, j, k) in rec]), np.array([q[k, j, i] for (i, j, k) in rec])
    assert np.all(pr != 0) and np.all(np.abs(pr - qr) > 1e-3 * np.abs(pr))


def test_fractions_helper_consistent():
    assert _moment_solve(1) == [Fraction(-2), Fraction(1)]
