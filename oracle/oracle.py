"""ctypes front end of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` are the only users.  Nothing in the CUDA
library imports this module, and this module imports nothing from the library.

Every function takes and returns plain NumPy float64 arrays of shape
``(nz, ny, nx)`` (C order, so x is fastest, as in the C code).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, OpenMP, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(ctypes.Structure):
    """Mirror of ``or_cfg`` in oracle.c."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("r_xy", ctypes.c_int), ("r_z", ctypes.c_int),
        ("h", ctypes.c_double), ("dz", ctypes.c_double),
        ("ztab", ctypes.POINTER(ctypes.c_double)),
        ("dt", ctypes.c_double),
        ("nb", ctypes.c_int), ("sponge_a", ctypes.c_double),
        ("src_on", ctypes.c_int), ("sx", ctypes.c_int), ("sy", ctypes.c_int), ("sz", ctypes.c_int),
        ("src_f", ctypes.c_double), ("src_t0", ctypes.c_double), ("src_amp", ctypes.c_double),
        ("src_into_q", ctypes.c_int), ("src_volume", ctypes.c_double),
        ("nrec", ctypes.c_int), ("rec", ctypes.POINTER(ctypes.c_int)),
        ("cxy", ctypes.POINTER(ctypes.c_double)), ("cz", ctypes.POINTER(ctypes.c_double)),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    """The oracle's library; FD_ORACLE_LIB names another build of oracle.c to load
    instead (the mutation test loads copies with planted mistakes this way)."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(os.environ.get("FD_ORACLE_LIB") or build())
            L.or_taylor_weights.argtypes = [ctypes.c_int, _D]
            L.or_lagrange_d2.argtypes = [_D, ctypes.c_int, ctypes.c_int, _D]
            L.or_z_table.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double, _D]
            L.or_nyquist_symbol.argtypes = [ctypes.c_int]
            L.or_nyquist_symbol.restype = ctypes.c_double
            L.or_iso_courant_limit.argtypes = [ctypes.c_int]
            L.or_iso_courant_limit.restype = ctypes.c_double
            L.or_ricker.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_ricker.restype = ctypes.c_double
            L.or_sponge_axis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.or_sponge_axis.restype = ctypes.c_double
            P = ctypes.POINTER(Cfg)
            L.or_iso_laplacian.argtypes = [P, _D, _D]
            L.or_vti_operators.argtypes = [P, _D, _D, _D, _D]
            L.or_iso_run.argtypes = [P, _D, _D, _D, ctypes.c_int, ctypes.c_int, _D]
            L.or_vti_run.argtypes = [P, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int, _D]
            L.or_iso_step_points.argtypes = [P, _F, _F, ctypes.c_int, _I, _D, ctypes.c_int, _D]
            L.or_vti_step_points.argtypes = [P, _F, _F, _F, _F, _F, ctypes.c_int, _I, _D, _D,
                                             ctypes.c_int, _D, _D]
            L.or_iso_misfit_grad.argtypes = [P, _D, _D, ctypes.c_int, _D, _D]
            L.or_sponge_at.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.or_sponge_at.restype = ctypes.c_double
            L.or_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# coefficient and scalar helpers
# --------------------------------------------------------------------------

def taylor_weights(R: int) -> np.ndarray:
    """c_0..c_R of the order-2R central second-derivative stencil (Eq. 4)."""
    c = np.zeros(R + 1)
    if lib().or_taylor_weights(R, _dp(c)) != 0:
        raise ValueError(f"bad radius {R}")
    return c


def symbol_ratio(c, k):
    """-S(k) / k^2 of the unit-grid stencil c (S(k) = c_0 + 2 sum c_l cos(l k)),
    1 for the exact second derivative; its k -> 0 limit is sum_l l^2 c_l."""
    c = np.asarray(c, dtype=np.float64)
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    out = np.empty_like(k)
    small = np.abs(k) < 1e-6
    l = np.arange(1, len(c))
    kk = k[~small][:, None]
    out[~small] = (4.0 * np.sin(0.5 * l * kk) ** 2 / kk ** 2) @ c[1:]
    out[small] = (l ** 2) @ c[1:]
    return out


def optimized_weights(R: int, kmax: float, samples: int = 4001) -> np.ndarray:
    """Band-optimised second-derivative weights (Sec. 1 notes that the weights
    can be optimised, after Holberg 1987; it gives no method).  Read here as:
    c_0..c_R exact on constants and quadratics (c_0 = -2 sum c_l,
    sum l^2 c_l = 1) minimising int_0^kmax (-S(k)/k^2 - 1)^2 dk, the squared
    relative error of the numerical phase velocity squared.  Solved as a
    linear least-squares problem in c_2..c_R (c_1 from the quadratic
    constraint) on `samples` equispaced wavenumbers with Simpson weights."""
    if R < 1 or not (0.0 < kmax <= np.pi):
        raise ValueError("radius >= 1 and 0 < kmax <= pi")
    c = np.zeros(R + 1)
    if R == 1:
        c[:] = [-2.0, 1.0]
        return c
    n = samples if samples % 2 == 1 else samples + 1
    k = np.linspace(0.0, kmax, n)
    w = np.ones(n)
    w[1:-1:2], w[2:-1:2] = 4.0, 2.0
    w *= (k[1] - k[0]) / 3.0
    # phi_l(k) = -S_l(k) / k^2 of the unit stencil "c_l = 1": 4 sin^2(l k/2) / k^2
    phi = np.empty((n, R))
    for l in range(1, R + 1):
        e = np.zeros(R + 1)
        e[l] = 1.0
        phi[:, l - 1] = symbol_ratio(e, k)
    ls = np.arange(2, R + 1)
    A = phi[:, 1:] - phi[:, [0]] * (ls ** 2)[None, :]
    b = 1.0 - phi[:, 0]
    sw = np.sqrt(w)[:, None]
    x = np.linalg.lstsq(A * sw, b * sw[:, 0], rcond=None)[0]
    c[2:] = x
    c[1] = 1.0 - (ls ** 2) @ x
    c[0] = -2.0 * c[1:].sum()
    return c


def lagrange_d2(z, k: int) -> np.ndarray:
    """Second-derivative weights at node z[k] from all nodes z (Eq. 5)."""
    z = _c64(z)
    w = np.zeros(len(z))
    if lib().or_lagrange_d2(_dp(z), len(z), k, _dp(w)) != 0:
        raise ValueError("bad nodes")
    return w


def z_table(nz: int, Rz: int, dzk=None, dz: float = 1.0) -> np.ndarray:
    """(nz, 2Rz+1) table of per-plane z weights (Eq. 5); dzk = nz-1 spacings."""
    tab = np.zeros((nz, 2 * Rz + 1))
    if dzk is not None:
        dzk = _c64(dzk)
        assert dzk.shape == (nz - 1,)
        ptr = _dp(dzk)
    else:
        ptr = None
    if lib().or_z_table(nz, Rz, ptr, dz, _dp(tab)) != 0:
        raise ValueError("bad z table arguments")
    return tab


def nyquist_symbol(R: int) -> float:
    return lib().or_nyquist_symbol(R)


def iso_courant_limit(R: int) -> float:
    """Largest stable v*dt/h of the 3D isotropic scheme with dx = dy = dz."""
    return lib().or_iso_courant_limit(R)


def ricker(t: float, f: float) -> float:
    return lib().or_ricker(t, f)


def sponge_axis(i: int, n: int, nb: int, a: float) -> float:
    return lib().or_sponge_axis(i, n, nb, a)


# --------------------------------------------------------------------------
# configuration
# --------------------------------------------------------------------------

class Problem:
    """Keeps a ``Cfg`` and the arrays it points to alive together."""

    def __init__(self, nx, ny, nz, *, r_xy, r_z=None, h, dz=None, dzk=None, dt,
                 nb=0, sponge_a=0.0, src=None, src_f=15.0, src_t0=None, src_amp=1.0,
                 src_into_q=False, src_volume=None, receivers=None, weights_xy=None, weights_z=None):
        r_z = r_xy if r_z is None else r_z
        dz = h if dz is None else dz
        self.shape = (nz, ny, nx)
        self.ztab = None
        if dzk is not None:
            self.ztab = z_table(nz, r_z, dzk)
        rec = np.zeros((0, 3), dtype=np.int32) if receivers is None else np.asarray(receivers, np.int32)
        self.rec = np.ascontiguousarray(rec.reshape(-1, 3), dtype=np.int32)
        c = Cfg()
        c.nx, c.ny, c.nz = nx, ny, nz
        c.r_xy, c.r_z = r_xy, r_z
        c.h, c.dz = h, dz
        c.ztab = _dp(self.ztab) if self.ztab is not None else None
        c.dt = dt
        c.nb, c.sponge_a = nb, sponge_a
        if src is not None:
            c.src_on = 1
            c.sx, c.sy, c.sz = src
            c.src_f = src_f
            c.src_t0 = (1.0 / src_f) if src_t0 is None else src_t0
            c.src_amp = src_amp
            c.src_into_q = int(bool(src_into_q))
            if src_volume is None:
                if dzk is not None:
                    k = src[2]
                    dzk_a = np.asarray(dzk, dtype=np.float64)
                    lo = dzk_a[k - 1] if k >= 1 else dzk_a[0]
                    hi = dzk_a[k] if k <= nz - 2 else dzk_a[-1]
                    src_volume = h * h * 0.5 * (lo + hi)
                else:
                    src_volume = h * h * dz
            c.src_volume = src_volume
        c.nrec = len(self.rec)
        c.rec = self.rec.ctypes.data_as(_I) if len(self.rec) else None
        # optional stencil weights (default: Taylor, Eq. 4); z weights need a uniform dz
        self.wxy = None if weights_xy is None else _c64(weights_xy)
        self.wz = None if weights_z is None else _c64(weights_z)
        if self.wxy is not None:
            assert self.wxy.shape == (r_xy + 1,)
            c.cxy = _dp(self.wxy)
        if self.wz is not None:
            assert self.wz.shape == (r_z + 1,) and dzk is None
            c.cz = _dp(self.wz)
        self.cfg = c

    @property
    def nrec(self):
        return len(self.rec)

    # ---- operators ---------------------------------------------------------
    def iso_laplacian(self, u):
        u = _c64(u)
        out = np.zeros(self.shape)
        lib().or_iso_laplacian(ctypes.byref(self.cfg), _dp(u), _dp(out))
        return out

    def vti_operators(self, p, q):
        p, q = _c64(p), _c64(q)
        hp, dq = np.zeros(self.shape), np.zeros(self.shape)
        lib().or_vti_operators(ctypes.byref(self.cfg), _dp(p), _dp(q), _dp(hp), _dp(dq))
        return hp, dq

    def sponge_at(self, i, j, k):
        return lib().or_sponge_at(ctypes.byref(self.cfg), i, j, k)

    def sponge_field(self):
        nz, ny, nx = self.shape
        c = self.cfg
        gx = np.array([sponge_axis(i, nx, c.nb, c.sponge_a) for i in range(nx)])
        gy = np.array([sponge_axis(j, ny, c.nb, c.sponge_a) for j in range(ny)])
        gz = np.array([sponge_axis(k, nz, c.nb, c.sponge_a) for k in range(nz)])
        return gz[:, None, None] * gy[None, :, None] * gx[None, None, :]

    # ---- time stepping -----------------------------------------------------
    def iso_run(self, v, nsteps, u=None, uprev=None, n0=0, traces=True):
        """Advance (u^{n0}, u^{n0-1}) by nsteps.  Returns (u, uprev, traces)."""
        v = _c64(v)
        u = np.zeros(self.shape) if u is None else _c64(u).copy()
        uprev = np.zeros(self.shape) if uprev is None else _c64(uprev).copy()
        tr = np.zeros((nsteps, max(self.nrec, 0))) if traces else None
        rc = lib().or_iso_run(ctypes.byref(self.cfg), _dp(v), _dp(u), _dp(uprev), n0, nsteps,
                              _dp(tr) if tr is not None and tr.size else None)
        if rc != 0:
            raise RuntimeError(f"or_iso_run failed: {rc}")
        return u, uprev, tr

    def vti_run(self, vz, eps, delta, nsteps, p=None, pprev=None, q=None, qprev=None, n0=0,
                traces=True):
        vz, eps, delta = _c64(vz), _c64(eps), _c64(delta)
        z = lambda a: np.zeros(self.shape) if a is None else _c64(a).copy()  # noqa: E731
        p, pprev, q, qprev = z(p), z(pprev), z(q), z(qprev)
        tr = np.zeros((nsteps, self.nrec)) if traces else None
        rc = lib().or_vti_run(ctypes.byref(self.cfg), _dp(vz), _dp(eps), _dp(delta),
                              _dp(p), _dp(pprev), _dp(q), _dp(qprev), n0, nsteps,
                              _dp(tr) if tr is not None and tr.size else None)
        if rc != 0:
            raise RuntimeError(f"or_vti_run failed: {rc}")
        return p, pprev, q, qprev, tr

    def iso_misfit_grad(self, v, dobs, nsteps, grad=True):
        """(J, dJ/dv) of the run from rest against data dobs (nsteps, nrec)."""
        v = _c64(v)
        dobs = _c64(dobs).reshape(nsteps, self.nrec)
        J = ctypes.c_double()
        g = np.zeros(self.shape) if grad else None
        rc = lib().or_iso_misfit_grad(ctypes.byref(self.cfg), _dp(v), _dp(dobs), nsteps, ctypes.byref(J),
                                      _dp(g) if grad else None)
        if rc != 0:
            raise RuntimeError("or_iso_misfit_grad failed")
        return J.value, g

    def iso_step_points(self, v32, u32, pts, uprev_pts, n):
        """u^{n+1} at the cells pts (M, 3) [ix, iy, iz] from float32 state u^n."""
        v32 = np.ascontiguousarray(v32, np.float32)
        u32 = np.ascontiguousarray(u32, np.float32)
        pts = np.ascontiguousarray(pts, np.int32)
        up = _c64(uprev_pts)
        out = np.zeros(len(pts))
        rc = lib().or_iso_step_points(ctypes.byref(self.cfg), v32.ctypes.data_as(_F),
                                      u32.ctypes.data_as(_F), len(pts), pts.ctypes.data_as(_I),
                                      _dp(up), n, _dp(out))
        if rc != 0:
            raise RuntimeError("or_iso_step_points failed")
        return out

    def vti_step_points(self, vz32, eps32, delta32, p32, q32, pts, pprev_pts, qprev_pts, n):
        f = lambda a: np.ascontiguousarray(a, np.float32)  # noqa: E731
        vz32, eps32, delta32, p32, q32 = f(vz32), f(eps32), f(delta32), f(p32), f(q32)
        pts = np.ascontiguousarray(pts, np.int32)
        pp, qp = _c64(pprev_pts), _c64(qprev_pts)
        op, oq = np.zeros(len(pts)), np.zeros(len(pts))
        F = lambda a: a.ctypes.data_as(_F)  # noqa: E731
        rc = lib().or_vti_step_points(ctypes.byref(self.cfg), F(vz32), F(eps32), F(delta32),
                                      F(p32), F(q32), len(pts), pts.ctypes.data_as(_I),
                                      _dp(pp), _dp(qp), n, _dp(op), _dp(oq))
        if rc != 0:
            raise RuntimeError("or_vti_step_points failed")
        return op, oq


def num_threads() -> int:
    return lib().or_num_threads()
