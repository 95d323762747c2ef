"""Pins of the oracle's misfit gradient (discrete adjoint of the damped
leapfrog): central finite differences in FP64 along random directions, the
misfit itself against the oracle's forward run, and linearity checks."""
import numpy as np
import pytest


def _case(O, R=2, n=(13, 11, 12), nb=3, steps=45):
    nx, ny, nz = n
    rng = np.random.default_rng(31)
    v = rng.uniform(1800.0, 2600.0, size=(nz, ny, nx))
    h = 10.0
    dt = 0.45 * O.iso_courant_limit(R) * h / v.max()
    rec = [(i, j, 4) for j in (2, 5, 8) for i in (2, 6, 10)]
    P = O.Problem(nx, ny, nz, r_xy=R, h=h, dt=dt, nb=nb, sponge_a=0.08, src=(6, 5, 6), src_f=25.0,
                  src_t0=0.03, receivers=rec)
    vtrue = v.copy()
    vtrue[4:8, 3:8, 4:9] *= 1.08
    _, _, dobs = P.iso_run(vtrue, steps)
    return P, v, dobs, steps


def test_misfit_matches_forward_traces(O):
    P, v, dobs, steps = _case(O)
    _, _, tr = P.iso_run(v, steps)
    J, _ = P.iso_misfit_grad(v, dobs, steps, grad=False)
    assert J == pytest.approx(0.5 * np.sum((tr - dobs) ** 2), rel=1e-12)
    assert J > 0
    J0, _ = P.iso_misfit_grad(v, tr, steps, grad=False)
    assert J0 == 0.0


@pytest.mark.parametrize("R", [2, 4])
def test_gradient_central_differences(O, R):
    P, v, dobs, steps = _case(O, R=R)
    J, g = P.iso_misfit_grad(v, dobs, steps)
    rng = np.random.default_rng(R)
    for _ in range(3):
        d = rng.standard_normal(v.shape)
        eps = 1e-3
        Jp, _ = P.iso_misfit_grad(v + eps * d, dobs, steps, grad=False)
        Jm, _ = P.iso_misfit_grad(v - eps * d, dobs, steps, grad=False)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(g * d))
        assert an == pytest.approx(fd, rel=2e-6, abs=1e-12 * abs(J))


def test_gradient_localised_and_linear_in_residual(O):
    P, v, dobs, steps = _case(O)
    _, _, tr = P.iso_run(v, steps)
    # J = 1/2 |r|^2 with r = tr - dobs: scaling the residual by s scales the gradient by s
    J1, g1 = P.iso_misfit_grad(v, tr - (tr - dobs), steps)
    J2, g2 = P.iso_misfit_grad(v, tr - 2.0 * (tr - dobs), steps)
    assert J2 == pytest.approx(4.0 * J1, rel=1e-12)
    np.testing.assert_allclose(g2, 2.0 * g1, rtol=1e-10, atol=1e-14 * np.abs(g1).max())
