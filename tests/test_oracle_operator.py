"""Pins of the oracle's spatial operators (Eqs. 4-5) without the time loop.

* polynomial exactness: L x^a y^b z^c equals the analytic Laplacian at points at
  least R cells from the boundary for per-axis degree <= 2R+1, and fails at 2R+2
  (so the stencil order is what Eq. 4 asks, not lower);
* the VTI operators split: Hp sees only x-y, Dq only z (Eqs. 1-2, 4-5), with the
  stretched-z rows exact up to degree 2R_z;
* brute force: a dense matrix assembled tap by tap on a tiny grid (zero halo),
  checked to be symmetric, reproduces the oracle's L.
"""
import itertools

import numpy as np
import pytest


def _coords(n, h, c):
    return (np.arange(n) - c) * h


def _poly_field(nx, ny, nz, h, dz, a, b, cdeg):
    x = _coords(nx, h, nx // 2)
    y = _coords(ny, h, ny // 2)
    z = _coords(nz, dz, nz // 2)
    return (z[:, None, None] ** cdeg) * (y[None, :, None] ** b) * (x[None, None, :] ** a), x, y, z


def _d2(t, p):
    return p * (p - 1) * t ** (p - 2) if p >= 2 else np.zeros_like(t)


@pytest.mark.parametrize("R", [4, 8])
def test_iso_polynomial_exactness(O, R):
    n = 2 * R + 6
    h, dz = 0.5, 0.75
    P = O.Problem(n, n, n, r_xy=R, h=h, dz=dz, dt=1.0)
    sl = slice(R, n - R)
    for (a, b, c) in [(2 * R + 1, 0, 0), (0, 2 * R, 1), (1, 2, 2 * R + 1), (R, R + 1, 3), (2, 2, 2)]:
        u, x, y, z = _poly_field(n, n, n, h, dz, a, b, c)
        Lu = P.iso_laplacian(u)
        exact = (_d2(z, c)[:, None, None] * (y ** b)[None, :, None] * (x ** a)[None, None, :]
                 + (z ** c)[:, None, None] * _d2(y, b)[None, :, None] * (x ** a)[None, None, :]
                 + (z ** c)[:, None, None] * (y ** b)[None, :, None] * _d2(x, a)[None, None, :])
        err = np.abs(Lu[sl, sl, sl] - exact[sl, sl, sl]).max()
        scale = np.abs(exact[sl, sl, sl]).max() + np.abs(u[sl, sl, sl]).max() / h ** 2
        assert err <= 1e-11 * scale, (a, b, c, err, scale)


@pytest.mark.parametrize("R", [2, 4])
def test_iso_order_is_not_higher(O, R):
    # degree 2R+2 along x breaks exactness: the truncation term is nonzero
    n = 2 * R + 6
    P = O.Problem(n, n, n, r_xy=R, h=1.0, dt=1.0)
    u, x, y, z = _poly_field(n, n, n, 1.0, 1.0, 2 * R + 2, 0, 0)
    Lu = P.iso_laplacian(u)
    sl = slice(R, n - R)
    exact = np.broadcast_to(_d2(x, 2 * R + 2)[None, None, :], u.shape)
    assert np.abs(Lu[sl, sl, sl] - exact[sl, sl, sl]).max() > 1e-3


def test_vti_operators_split_and_exactness(O):
    nx = ny = 30
    nz = 24
    rxy, rz = 12, 4
    h = 2.0
    rng = np.random.default_rng(3)
    dzk = 1.5 * (1.0 + rng.uniform(-0.1, 0.1, size=nz - 1))
    P = O.Problem(nx, ny, nz, r_xy=rxy, r_z=rz, h=h, dzk=dzk, dt=1.0)
    zc = np.concatenate([[0.0], np.cumsum(dzk)])
    x = _coords(nx, h, nx // 2)
    y = _coords(ny, h, ny // 2)
    zz = zc - zc[nz // 2]
    # p = x^5 y^3 (no z), q = z^(2 rz) (no x, y)
    p = np.broadcast_to((y ** 3)[None, :, None] * (x ** 5)[None, None, :], (nz, ny, nx)).copy()
    q = np.broadcast_to((zz ** (2 * rz))[:, None, None], (nz, ny, nx)).copy()
    Hp, Dq = P.vti_operators(p, q)
    sx = slice(rxy, nx - rxy)
    szi = slice(rz, nz - rz)
    hp_exact = (y ** 3)[None, :, None] * _d2(x, 5)[None, None, :] + _d2(y, 3)[None, :, None] * (x ** 5)[None, None, :]
    np.testing.assert_allclose(Hp[:, sx, sx], np.broadcast_to(hp_exact, Hp.shape)[:, sx, sx],
                               rtol=1e-9, atol=1e-6)
    dq_exact = _d2(zz, 2 * rz)[:, None, None]
    np.testing.assert_allclose(Dq[szi], np.broadcast_to(dq_exact, Dq.shape)[szi], rtol=1e-8, atol=1e-6)
    # Hp ignores q and z structure, Dq ignores p
    Hp2, Dq2 = P.vti_operators(p, np.zeros_like(q))
    np.testing.assert_array_equal(Hp2, Hp)
    assert np.abs(Dq2).max() == 0.0


def _dense_laplacian(nx, ny, nz, R, h, dz, c):
    """Assemble L tap by tap: row (i,j,k), column of each in-grid neighbour."""
    N = nx * ny * nz
    A = np.zeros((N, N))
    lin = lambda i, j, k: i + nx * (j + ny * k)  # noqa: E731
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        r = lin(i, j, k)
        A[r, r] += c[0] * (2.0 / h ** 2 + 1.0 / dz ** 2)
        for l in range(1, R + 1):
            for (di, dj, dk, w) in [(l, 0, 0, h), (-l, 0, 0, h), (0, l, 0, h), (0, -l, 0, h),
                                    (0, 0, l, dz), (0, 0, -l, dz)]:
                ii, jj, kk = i + di, j + dj, k + dk
                if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                    A[r, lin(ii, jj, kk)] += c[l] / w ** 2
    return A


@pytest.mark.parametrize("R,shape", [(2, (7, 6, 5)), (4, (8, 8, 8)), (4, (3, 9, 5))])
def test_dense_brute_force_laplacian(O, R, shape):
    nx, ny, nz = shape
    h, dz = 3.0, 2.0
    c = O.taylor_weights(R)
    A = _dense_laplacian(nx, ny, nz, R, h, dz, c)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-15)
    u = np.random.default_rng(1).standard_normal((nz, ny, nx))
    P = O.Problem(nx, ny, nz, r_xy=R, h=h, dz=dz, dt=1.0)
    np.testing.assert_allclose(P.iso_laplacian(u).ravel(), A @ u.ravel(), rtol=1e-13, atol=1e-13)
    # -L is positive definite with zero ghosts (needed by the energy argument)
    assert np.linalg.eigvalsh(-A).min() > 0
