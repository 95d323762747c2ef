"""The pins catch plausible mistakes: each entry below plants one (a dropped
term, a wrong sign, index or factor, a transposed operand, a copy-paste slip)
in a copy of oracle.c, builds the copy aside, and runs the oracle's pin tests
against it (FD_ORACLE_LIB); every copy must fail at least one pin.  The source
file itself is never touched."""
import concurrent.futures
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = ["tests/test_oracle_weights.py", "tests/test_oracle_operator.py", "tests/test_oracle_time.py",
        "tests/test_oracle_adjoint.py"]

MUTATIONS = [
    # x-y stencil: centre weight counted once instead of for both axes
    ("2.0 * cw[0] * at(u, c, i, j, k);\n    for", "cw[0] * at(u, c, i, j, k);\n    for"),
    # x-y stencil: off-by-one neighbour
    ("at(u, c, i - l, j, k) +\n", "at(u, c, i - l + 1, j, k) +\n"),
    # leapfrog: sign of the older level
    ("un[p] = 2.0 * cur[p] - prv[p]", "un[p] = 2.0 * cur[p] + prv[p]"),
    # source: dt instead of dt^2
    ("return c->dt * c->dt * s / c->src_volume;", "return c->dt * s / c->src_volume;"),
    # damping applied to the new level only
    ("un[idx(c, i, j, k)] *= g;\n                        cur[idx(c, i, j, k)] *= g;", "un[idx(c, i, j, k)] *= g;"),
    # z stencil scaled by h instead of dz
    ("return s / (c->dz * c->dz);", "return s / (c->h * c->h);"),
    # VTI: kappa_x in the q equation
    ("qn[m] = 2.0 * qc[m] - qp[m] + kn * Hp", "qn[m] = 2.0 * qc[m] - qp[m] + kx * Hp"),
    # VTI: kappa_n on Dq
    ("+ kn * Hp + v2 * Dq;\n                }", "+ kn * Hp + kn * Dq;\n                }"),
    # receivers sample the old level
    ("                    un[idx(c, c->rec[3 * r]", "                    cur[idx(c, c->rec[3 * r]"),
    # Taylor weights: factorial ratio off by one
    ("ratio *= (double)(R - l + m) / (double)(R + m);", "ratio *= (double)(R - l + m + 1) / (double)(R + m);"),
    # Lagrange second derivative: a node left in the product
    ("if (m != j && m != a && m != b) prod", "if (m != j && m != a) prod"),
    # ghost planes below the grid: wrong spacing
    ("if (k <= 0) return dzk[0] * (double)k;", "if (k <= 0) return dzk[1] * (double)k;"),
    # damping layer: distance off by one on the far side
    ("else if (i >= n - nb) d = i - (n - nb - 1);", "else if (i >= n - nb) d = i - (n - nb);"),
    # VTI: v instead of v^2
    ("double v2 = vz[m] * vz[m] * c->dt * c->dt;", "double v2 = vz[m] * c->dt * c->dt;"),
    # per-plane z weights applied reversed
    ("for (int l = -c->r_z; l <= c->r_z; ++l) s += w[l + c->r_z] * at(u, c, i, j, k + l);",
     "for (int l = -c->r_z; l <= c->r_z; ++l) s += w[c->r_z - l] * at(u, c, i, j, k + l);"),
    # adjoint: sign of the older-level term
    ("be[m] = -G[m] * al[m];", "be[m] = G[m] * al[m];"),
    # adjoint: damping factor dropped on the older-level term
    ("aln[m] = 2.0 * G[m] * al[m] + Lw + G[m] * be[m];", "aln[m] = 2.0 * G[m] * al[m] + Lw + be[m];"),
    # gradient: dt instead of dt^2 in dK/dv
    ("grad_v[m] = gk[m] * 2.0 * v[m] * c->dt * c->dt;", "grad_v[m] = gk[m] * 2.0 * v[m] * c->dt;"),
    # gradient: residual of the wrong step injected
    ("res[(size_t)(n - 1) * (size_t)c->nrec + (size_t)r];", "res[(size_t)n * (size_t)c->nrec + (size_t)r];"),
    # caller weights: x-y weights copied into z (copy-paste slip)
    ("for (int l = 0; l <= c->r_z; ++l) cz[l] = c->cz[l];", "for (int l = 0; l <= c->r_z; ++l) cz[l] = c->cxy[l];"),
    # VTI: delta in place of epsilon in kappa_x
    ("double kx = v2 * (1.0 + 2.0 * eps[m]);", "double kx = v2 * (1.0 + 2.0 * delta[m]);"),
    # VTI: source injected into q as well, whatever the setting
    ("if (c->src_into_q) qn[idx(c, c->sx, c->sy, c->sz)] += st;", "qn[idx(c, c->sx, c->sy, c->sz)] += st;"),
    # Ricker: factor 2 dropped from the polynomial
    ("return (1.0 - 2.0 * a) * exp(-a);", "return (1.0 - a) * exp(-a);"),
    # source sampled one step late
    ("or_ricker((double)n * c->dt - c->src_t0, c->src_f);", "or_ricker((double)(n + 1) * c->dt - c->src_t0, c->src_f);"),
    # damping: exp(-a d) instead of exp(-(a d)^2)
    ("return exp(-ad * ad);", "return exp(-ad);"),
    # VTI: the q equation takes Hp for Dq
    ("qn[m] = 2.0 * qc[m] - qp[m] + kn * Hp + v2 * Dq;", "qn[m] = 2.0 * qc[m] - qp[m] + kn * Hp + v2 * Hp;"),
    # receivers: x and y of the receiver swapped
    ("traces[(size_t)s * (size_t)c->nrec + (size_t)r] =\n                    un[idx(c, c->rec[3 * r], c->rec[3 * r + 1],",
     "traces[(size_t)s * (size_t)c->nrec + (size_t)r] =\n                    un[idx(c, c->rec[3 * r + 1], c->rec[3 * r],"),
    # VTI: traces sample q instead of p
    ("                    pn[idx(c, c->rec[3 * r], c->rec[3 * r + 1], c->rec[3 * r + 2])];",
     "                    qn[idx(c, c->rec[3 * r], c->rec[3 * r + 1], c->rec[3 * r + 2])];"),
    # VTI damping: the older level of q left undamped
    ("pn[m] *= g; pc[m] *= g; qn[m] *= g; qc[m] *= g;", "pn[m] *= g; pc[m] *= g; qn[m] *= g;"),
    # x-y stencil: one y neighbour counted twice (copy-paste slip)
    ("at(u, c, i, j + l, k) + at(u, c, i, j - l, k));", "at(u, c, i, j + l, k) + at(u, c, i, j + l, k));"),
    # VTI: Dq taken of p
    ("double Dq = op_z(c, cz, qc, i, j, k);\n", "double Dq = op_z(c, cz, pc, i, j, k);\n"),
    # VTI: Hp taken of q
    ("double Hp = op_h(c, cw, pc, i, j, k);\n", "double Hp = op_h(c, cw, qc, i, j, k);\n"),
]


def _run(i, before, after, tmp):
    src = open(SRC).read()
    assert src.count(before) >= 1, f"mutation {i}: pattern not found"
    c_path = os.path.join(tmp, f"m{i}.c")
    so_path = os.path.join(tmp, f"m{i}.so")
    with open(c_path, "w") as f:
        f.write(src.replace(before, after, 1))
    b = subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", so_path, c_path, "-lm"],
                       capture_output=True, text=True)
    if b.returncode != 0:
        return i, False, "does not compile: " + b.stderr[-300:]
    env = dict(os.environ, FD_ORACLE_LIB=so_path, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *PINS],
                       capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    return i, r.returncode != 0, r.stdout[-300:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda a: _run(a[0], a[1][0], a[1][1], str(tmp_path)), enumerate(MUTATIONS)))
    missed = [(i, out) for i, caught, out in results if not caught]
    assert not missed, f"planted mistakes no pin caught: {missed}"


@pytest.mark.parametrize("i", [0])
def test_unmutated_copy_passes(tmp_path, i):
    """The harness itself: the unchanged source built the same way passes."""
    idx, caught, out = _run(-1, "#include <math.h>", "#include <math.h>", str(tmp_path))
    assert not caught, out
