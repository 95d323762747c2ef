"""The C ABI without a GPU: libfd.so loads, exports every entry point that
include/fd.h declares, and its pure host calls (layout, sizes, stability
bound, argument validation) behave; the stability bound is cross-checked
against the oracle's, which is computed by independent code."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_1387_gb300 import fd as fdmod
    fdmod.lib()
    return fdmod


def _declared():
    src = open(os.path.join(ROOT, "include", "fd.h")).read()
    return sorted(set(re.findall(r"^int\s+(fd_\w+)\s*\(", src, flags=re.M)))


def test_header_and_binding_agree(fd):
    assert _declared() == sorted(fd.EXPORTS)


def test_library_exports_every_declared_symbol(fd):
    L = fd.lib()
    for name in _declared():
        assert hasattr(L, name), name


def _iso(fd, n=64, R=4, **kw):
    d, keep = fd.make_desc(fd.FD_MODE_ISO, n, n, n, R, R, 10.0, 10.0, 1e-3, **kw)
    return d


def test_layout_and_bytes(fd):
    d = _iso(fd, 70)
    L = fd.fd_layout(d)
    assert L.pitch == 96 and L.nfields == 2 and L.nmodel == 1
    assert L.field_bytes == 96 * 70 * 70 * 4
    assert fd.fd_required_bytes(d) == 3 * L.field_bytes
    dv, keep = fd.make_desc(fd.FD_MODE_VTI, 33, 5, 7, 12, 8, 10.0, 0.0, 1e-4, dz_k=np.full(6, 9.0))
    Lv = fd.fd_layout(dv)
    assert Lv.pitch == 64 and Lv.nfields == 4 and Lv.nmodel == 3
    assert Lv.field_bytes == (64 * 5 * 7 * 4 + 255) // 256 * 256


@pytest.mark.parametrize("R", [4, 8])
def test_stability_limit_matches_oracle(fd, O, R):
    d = _iso(fd, 64, R)
    dt = fd.fd_stability_limit(d, 2000.0)
    assert dt == pytest.approx(O.iso_courant_limit(R) * 10.0 / 2000.0, rel=1e-12)


def test_vti_stability_limit_matches_oracle_tables(fd, O):
    nz = 40
    dzk = 10.0 * (1 + 0.1 * np.sin(np.arange(nz - 1)))
    d, keep = fd.make_desc(fd.FD_MODE_VTI, 32, 32, nz, 12, 8, 10.0, 0.0, 1e-4, dz_k=dzk)
    dt = fd.fd_stability_limit(d, 4725.0, 0.25)
    sxy = O.nyquist_symbol(12)
    zrow = np.abs(O.z_table(nz, 8, dzk)).sum(axis=1).max()
    rho = 1.5 * 2 * sxy / 100.0 + zrow
    assert dt == pytest.approx(2.0 / (4725.0 * np.sqrt(rho)), rel=1e-9)


def test_vti_workload_dt_is_half_the_bound(fd):
    from paper_1410_1387_gb300 import synth
    s = synth.vti_shot(512, with_model=False)
    d, keep = fd.make_desc(fd.FD_MODE_VTI, s.nx, s.ny, s.nz, 12, 8, s.h, s.h, s.dt, dz_k=s.dzk)
    bound = fd.fd_stability_limit(d, synth.V_MAX_LAYERED, 0.25)
    assert 0.45 * bound < s.dt < 0.55 * bound


@pytest.mark.parametrize("kw,code", [
    (dict(mode=0, nx=0), -1), (dict(mode=0, nx=8, r=3), -8), (dict(mode=0, nx=8, dt=-1.0), -1),
    (dict(mode=1, nx=8, r=8), -8), (dict(mode=7, nx=8), -1),
])
def test_invalid_descriptions(fd, kw, code):
    r = kw.get("r", 4)
    mode = kw["mode"]
    rz = 8 if (mode == 1 and r == 12) else r
    d, keep = fd.make_desc(mode, kw["nx"], 8, 8, r, rz, 10.0, 10.0, kw.get("dt", 1e-3))
    with pytest.raises(fd.FdError) as e:
        fd.fd_required_bytes(d)
    assert e.value.code == code
    assert fd.fd_last_error()


@pytest.mark.parametrize("R,kmax", [(1, 1.0), (4, 2.0), (8, 2.3), (12, 2.5), (4, 3.14159)])
def test_optimized_weights_match_oracle(fd, O, R, kmax):
    """The library's band-optimised weights (Gauss-Legendre quadrature, Householder
    QR) against the oracle's (Simpson sampling, SVD least squares)."""
    a = fd.fd_optimized_weights(R, kmax)
    b = O.optimized_weights(R, kmax)
    assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()


@pytest.mark.parametrize("R,kmax", [(0, 1.0), (13, 1.0), (4, 0.0), (4, 3.2), (4, float("nan"))])
def test_optimized_weights_reject_bad_arguments(fd, R, kmax):
    with pytest.raises(fd.FdError) as e:
        fd.fd_optimized_weights(max(R, 0), kmax)
    assert e.value.code == fd.FD_ERR_INVALID_ARG


def test_no_fallback_when_library_missing(monkeypatch):
    from paper_1410_1387_gb300 import fd as fdmod
    monkeypatch.setattr(fdmod, "LIB_PATH", "/nonexistent/libfd.so")
    monkeypatch.setattr(fdmod, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        fdmod.lib()
