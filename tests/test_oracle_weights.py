"""Pins of the oracle's stencil weights (Eqs. 4-5) to facts outside the oracle.

* textbook centred weights (tests/golden/central_d2_weights.txt, Fornberg 1988),
* the Taylor moment conditions, solved exactly in rationals here (a different
  characterisation from the oracle's closed form),
* the variable-spacing z weights: exactness on polynomials up to degree 2R_z on
  stretched nodes, and reduction to the uniform weights on uniform nodes.
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
