"""Pins of the oracle's stencil weights (Eqs. 4-5) to facts outside the oracle.

* textbook centred weights (tests/golden/central_d2_weights.txt, Fornberg 1988),
* the Taylor moment conditions, solved exactly in rationals here (a different
  characterisation from the oracle's closed form),
* the variable-spacing z weights: exactness on polynomials up to degree 2R_z on
  stretched nodes, and reduction to the uniform weights on uniform nodes,
* the band-optimised weights (Sec. 1, after Holberg 1987): the two consistency
  constraints, optimality of the band error computed by adaptive quadrature
  (vanishing directional derivatives, and scipy's SLSQP reaching the same
  weights from the Taylor start), the Taylor weights as the band shrinks
  (quadratically), and a band error far below Taylor's.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "central_d2_weights.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        out[int(parts[0])] = [Fraction(p) for p in parts[1:]]
    return out


def _moment_solve(R):
    """Exact weights from the moment conditions: the symmetric stencil
    sum_l c_l (u_l + u_-l) + c_0 u_0 must reproduce u'' for x^(2m), m = 0..R,
    i.e. c_0 + 2 sum c_l = 0 and 2 sum_l c_l l^(2m) = (2m)(2m-1) 0^(2m-2)."""
    n = R + 1
    A = [[Fraction(0)] * n for _ in range(n)]
    b = [Fraction(0)] * n
    for m in range(n):
        for l in range(n):
            if l == 0:
                A[m][l] = Fraction(1 if m == 0 else 0)
            else:
                A[m][l] = Fraction(2 * l ** (2 * m))
        b[m] = Fraction(2) if m == 1 else Fraction(0)
    # Gaussian elimination in exact arithmetic
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col] / A[col][col]
                A[r] = [a - f * c for a, c in zip(A[r], A[col])]
                b[r] -= f * b[col]
    return [b[i] / A[i][i] for i in range(n)]


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_textbook_weights(O, R):
    want = _golden()[R]
    got = O.taylor_weights(R)
    np.testing.assert_allclose(got, [float(w) for w in want], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("R", [1, 2, 4, 6, 8, 12])
def test_moment_conditions_exact(O, R):
    exact = _moment_solve(R)
    got = O.taylor_weights(R)
    np.testing.assert_allclose(got, [float(w) for w in exact], rtol=1e-13, atol=1e-16)


def test_exact_solve_matches_golden():
    g = _golden()
    for R in (1, 2, 3, 4):
        assert _moment_solve(R) == g[R]


@pytest.mark.parametrize("R", [4, 8, 12])
def test_nyquist_symbol_is_stencil_symbol_at_pi(O, R):
    # symbol of the exact rational stencil at theta = pi: -(c_0 + 2 sum c_l cos(l pi))
    c = _moment_solve(R)
    sym = -(c[0] + 2 * sum(c[l] * (-1) ** l for l in range(1, R + 1)))
    assert O.nyquist_symbol(R) == pytest.approx(float(sym), rel=1e-14)


def test_courant_limit_literals(O):
    from paper_1410_1387_gb300.synth import COURANT_LIMIT
    for R, lim in COURANT_LIMIT.items():
        assert O.iso_courant_limit(R) == pytest.approx(lim, rel=1e-14)
    assert O.iso_courant_limit(1) == pytest.approx(1 / math.sqrt(3), rel=1e-15)  # textbook 7-point


@pytest.mark.parametrize("R", [2, 4, 8])
def test_lagrange_uniform_nodes_reduce_to_taylor(O, R):
    dz = 7.5
    z = dz * np.arange(-R, R + 1, dtype=np.float64)
    w = O.lagrange_d2(z, R)
    c = O.taylor_weights(R)
    want = np.concatenate([c[:0:-1], c]) / dz ** 2
    np.testing.assert_allclose(w, want, rtol=1e-9, atol=1e-12 / dz ** 2)


@pytest.mark.parametrize("R", [2, 4, 8])
def test_lagrange_stretched_polynomial_exactness(O, R):
    rng = np.random.default_rng(5)
    sp = 1.0 + rng.uniform(-0.3, 0.3, size=2 * R)
    z = np.concatenate([[0.0], np.cumsum(sp)])
    for k in (0, R, 2 * R):          # one-sided, centred, one-sided
        w = O.lagrange_d2(z, k)
        zc = z - z[k]
        for m in range(0, 2 * R + 1):
            got = float(np.sum(w * zc ** m))
            want = m * (m - 1) * 0.0 ** (m - 2) if m >= 2 else 0.0
            scale = float(np.sum(np.abs(w * zc ** m))) + 1.0
            assert abs(got - want) <= 1e-10 * scale, (k, m, got, want)


def test_z_table_rows(O):
    nz, Rz = 24, 4
    rng = np.random.default_rng(11)
    dzk = 10.0 * (1.0 + rng.uniform(-0.1, 0.1, size=nz - 1))
    tab = O.z_table(nz, Rz, dzk)
    z = np.concatenate([[0.0], np.cumsum(dzk)])
    # interior row k: nodes z[k-Rz..k+Rz]
    k = 11
    np.testing.assert_allclose(tab[k], O.lagrange_d2(z[k - Rz:k + Rz + 1], Rz), rtol=1e-12)
    # ghost rows continue the end spacing
    zg = np.concatenate([dzk[0] * np.arange(-Rz, 0), z[:Rz + 1]])
    np.testing.assert_allclose(tab[0], O.lagrange_d2(zg, Rz), rtol=1e-12)
    # uniform table equals the Taylor weights / dz^2 on every row
    tu = O.z_table(nz, Rz, None, dz=10.0)
    c = O.taylor_weights(Rz)
    np.testing.assert_allclose(tu, np.tile(np.concatenate([c[:0:-1], c]) / 100.0, (nz, 1)),
                               rtol=1e-9, atol=1e-14)


# ---------------------------------------------------------------------------
# band-optimised weights
# ---------------------------------------------------------------------------

def _band_error(O, c, kmax):
    """int_0^kmax (-S(k)/k^2 - 1)^2 dk by adaptive quadrature (independent of
    the oracle's Simpson sampling)."""
    from scipy import integrate
    return integrate.quad(lambda k: (O.symbol_ratio(c, k)[0] - 1.0) ** 2, 0.0, kmax, limit=400,
                          epsabs=1e-18, epsrel=1e-12)[0]


def _null_direction(R, rng):
    """A weight perturbation that keeps both constraints (sum l^2 d_l = 0,
    d_0 = -2 sum d_l)."""
    d = np.zeros(R + 1)
    d[1:] = rng.standard_normal(R)
    l2 = np.arange(1, R + 1) ** 2
    d[1:] -= (l2 @ d[1:]) / (l2 @ l2) * l2
    d[0] = -2.0 * d[1:].sum()
    return d


@pytest.mark.parametrize("R,kmax", [(2, 1.5), (4, 2.0), (8, 2.3), (12, 2.5)])
def test_optimized_weights_constraints(O, R, kmax):
    c = O.optimized_weights(R, kmax)
    assert abs(c[0] + 2.0 * c[1:].sum()) <= 1e-12 * np.abs(c).sum()
    assert abs((np.arange(1, R + 1) ** 2) @ c[1:] - 1.0) <= 1e-12
    assert abs(O.symbol_ratio(c, 0.0)[0] - 1.0) <= 1e-12


@pytest.mark.parametrize("R,kmax", [(4, 2.0), (8, 2.3)])
def test_optimized_weights_are_optimal(O, R, kmax):
    c = O.optimized_weights(R, kmax)
    e0 = _band_error(O, c, kmax)
    rng = np.random.default_rng(R)
    for _ in range(3):
        d = _null_direction(R, rng)
        h = 1e-3 * np.abs(c).max() / np.abs(d).max()
        ep, em = _band_error(O, c + h * d, kmax), _band_error(O, c - h * d, kmax)
        slope, curv = (ep - em) / (2 * h), (ep + em - 2 * e0) / h ** 2
        assert curv > 0 and abs(slope) <= 1e-6 * curv * np.abs(c).max()


def test_optimized_weights_match_slsqp(O):
    from scipy import optimize
    R, kmax = 4, 2.0
    c = O.optimized_weights(R, kmax)
    l2 = np.arange(1, R + 1) ** 2
    res = optimize.minimize(lambda x: _band_error(O, np.concatenate([[-2.0 * x.sum()], x]), kmax),
                            O.taylor_weights(R)[1:], method="SLSQP",
                            constraints=[{"type": "eq", "fun": lambda x: l2 @ x - 1.0}],
                            options={"ftol": 1e-16, "maxiter": 500})
    assert res.success
    assert np.abs(res.x - c[1:]).max() <= 1e-5 * np.abs(c).max()


def test_optimized_weights_tend_to_taylor(O):
    t = O.taylor_weights(4)
    dev = [np.abs(O.optimized_weights(4, km) - t).max() / np.abs(t).max() for km in (1.0, 0.5, 0.25)]
    assert dev[2] < 1e-3
    # quadratic in the band edge: halving kmax divides the deviation by ~4
    assert 3.5 < dev[0] / dev[1] < 4.5 and 3.5 < dev[1] / dev[2] < 4.5


@pytest.mark.parametrize("R,kmax", [(4, 2.0), (12, 2.5)])
def test_optimized_band_error_below_taylor(O, R, kmax):
    c, t = O.optimized_weights(R, kmax), O.taylor_weights(R)
    assert _band_error(O, c, kmax) < 0.05 * _band_error(O, t, kmax)
    k = np.linspace(1e-4, kmax, 2000)
    assert np.abs(O.symbol_ratio(c, k) - 1).max() < np.abs(O.symbol_ratio(t, k) - 1).max()
