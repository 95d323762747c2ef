"""Thin ctypes binding of ``libfd.so`` (the C ABI in ``include/fd.h``).

The ``fd_*`` functions here carry the C names and only marshal arguments; the
``Grid`` class strings them together for one shot, with PyTorch allocating the
device arena and trace buffer and providing the stream.  Every step of the
time loop runs in the library's CUDA kernels: there is no other code path, and
importing this module fails loudly when the library is not built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfd.so")

FD_OK = 0
FD_ERR_INVALID_ARG = -1
FD_ERR_UNSTABLE_DT = -2
FD_ERR_OUT_OF_RANGE = -3
FD_ERR_BAD_STATE = -4
FD_ERR_CUDA = -5
FD_ERR_TIMEOUT = -6
FD_ERR_NO_MEMORY = -7
FD_ERR_UNSUPPORTED = -8
FD_MODE_ISO = 0
FD_MODE_VTI = 1
FD_PTR_HOST = 0
FD_PTR_DEVICE = 1

# every entry point declared in include/fd.h
EXPORTS = [
    "fd_required_bytes", "fd_layout", "fd_stability_limit", "fd_create_grid", "fd_set_model",
    "fd_add_source", "fd_add_source_series", "fd_set_receivers", "fd_step", "fd_step_from", "fd_run",
    "fd_set_graph", "fd_read_receivers", "fd_run_to_host", "fd_get_state", "fd_set_state", "fd_field",
    "fd_set_launch", "fd_time_index", "fd_sync", "fd_destroy_grid", "fd_last_error",
    "fd_iso_step_static",
    "fd_batch_create", "fd_batch_set_launch", "fd_batch_set_graph", "fd_batch_add", "fd_batch_remove",
    "fd_batch_steps_left", "fd_batch_run", "fd_batch_destroy",
    "fd_set_injection", "fd_adjoint_source", "fd_grad_accumulate",
    "fd_set_z_window", "fd_halo_exchange", "fd_step_planes", "fd_optimized_weights", "fd_set_weights",
    "fd_debug_skip_copy",
]


class FdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class fd_desc(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("r_xy", ctypes.c_int), ("r_z", ctypes.c_int),
        ("h", ctypes.c_double), ("dz", ctypes.c_double),
        ("dz_k", ctypes.POINTER(ctypes.c_double)),
        ("dt", ctypes.c_double),
        ("sponge_width", ctypes.c_int), ("sponge_a", ctypes.c_double),
    ]


class fd_layout_t(ctypes.Structure):
    _fields_ = [
        ("pitch", ctypes.c_int), ("nfields", ctypes.c_int), ("nmodel", ctypes.c_int),
        ("field_bytes", ctypes.c_size_t), ("arena_bytes", ctypes.c_size_t),
    ]


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


def lib() -> ctypes.CDLL:
    """Load libfd.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() first "
                               "(there is no fallback path)")
        L = ctypes.CDLL(LIB_PATH)
        D = ctypes.POINTER(fd_desc)
        sig = {
            "fd_required_bytes": [D, ctypes.POINTER(ctypes.c_size_t)],
            "fd_layout": [D, ctypes.POINTER(fd_layout_t)],
            "fd_stability_limit": [D, _d, _d, ctypes.POINTER(ctypes.c_double)],
            "fd_create_grid": [D, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)],
            "fd_set_model": [_vp, _vp, _vp, _vp, _i],
            "fd_add_source": [_vp, _i, _i, _i, _d, _d, _d, _i],
            "fd_add_source_series": [_vp, _i, _i, _i, _vp, _i, _i],
            "fd_set_receivers": [_vp, _vp, _i, _vp, _i],
            "fd_step": [_vp],
            "fd_step_from": [_vp, _vp, _vp, _vp],
            "fd_run": [_vp, _i],
            "fd_set_graph": [_vp, _i],
            "fd_read_receivers": [_vp, _i, _i, _vp, _i],
            "fd_run_to_host": [_vp, _i, _vp, _i],
            "fd_get_state": [_vp, _vp, _vp, _vp, _vp, _i, ctypes.POINTER(_i)],
            "fd_set_state": [_vp, _vp, _vp, _vp, _vp, _i, _i],
            "fd_field": [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_i)],
            "fd_set_launch": [_vp, _i, _i, _i, _i],
            "fd_time_index": [_vp, ctypes.POINTER(_i)],
            "fd_sync": [_vp],
            "fd_destroy_grid": [_vp],
            "fd_last_error": [ctypes.c_char_p, ctypes.c_size_t],
            "fd_iso_step_static": [D, _vp, _vp, _vp, _i, _i, _i, _i, _d, _d, _d, _vp, _vp],
            "fd_batch_create": [_vp, ctypes.POINTER(_vp)],
            "fd_batch_set_launch": [_vp, _i, _i, _i, _i, _i],
            "fd_batch_set_graph": [_vp, _i],
            "fd_batch_add": [_vp, _vp, _i],
            "fd_batch_remove": [_vp, _vp],
            "fd_batch_steps_left": [_vp, _vp, ctypes.POINTER(_i)],
            "fd_batch_run": [_vp, _i, ctypes.POINTER(_i)],
            "fd_batch_destroy": [_vp],
            "fd_set_injection": [_vp, _vp, _i, _vp, _i],
            "fd_adjoint_source": [_vp, _vp, _vp, _i, _vp, ctypes.POINTER(ctypes.c_double)],
            "fd_grad_accumulate": [_vp, _vp, _vp, _vp],
            "fd_set_z_window": [_vp, _i, _i],
            "fd_halo_exchange": [_vp, _vp, _i],
            "fd_step_planes": [_vp, _i, _i, _i],
            "fd_optimized_weights": [_i, _d, _vp],
            "fd_set_weights": [_vp, _vp, _vp],
            "fd_debug_skip_copy": [_vp, _i],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def fd_last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().fd_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def _check(rc: int) -> None:
    if rc != FD_OK:
        raise FdError(rc, fd_last_error())


def _ptr(x):
    """Raw address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


# ---- one function per C entry point -------------------------------------------

def make_desc(mode, nx, ny, nz, r_xy, r_z, h, dz, dt, sponge_width=0, sponge_a=0.0, dz_k=None):
    """Build an fd_desc; the returned tuple keeps dz_k alive alongside it."""
    d = fd_desc()
    d.mode, d.nx, d.ny, d.nz, d.r_xy, d.r_z = mode, nx, ny, nz, r_xy, r_z
    d.h, d.dz, d.dt = h, dz, dt
    d.sponge_width, d.sponge_a = sponge_width, sponge_a
    keep = None
    if dz_k is not None:
        keep = np.ascontiguousarray(dz_k, dtype=np.float64)
        d.dz_k = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return d, keep


def fd_required_bytes(d: fd_desc) -> int:
    out = ctypes.c_size_t()
    _check(lib().fd_required_bytes(ctypes.byref(d), ctypes.byref(out)))
    return out.value


def fd_layout(d: fd_desc) -> fd_layout_t:
    out = fd_layout_t()
    _check(lib().fd_layout(ctypes.byref(d), ctypes.byref(out)))
    return out


def fd_stability_limit(d: fd_desc, vmax: float, eps_max: float = 0.0) -> float:
    out = ctypes.c_double()
    _check(lib().fd_stability_limit(ctypes.byref(d), vmax, eps_max, ctypes.byref(out)))
    return out.value


def fd_create_grid(d: fd_desc, arena, arena_bytes: int, stream: int) -> int:
    out = _vp()
    _check(lib().fd_create_grid(ctypes.byref(d), _ptr(arena), arena_bytes, stream, ctypes.byref(out)))
    return out.value


def fd_set_model(g, vz, eps=None, delta=None, ptr_kind=FD_PTR_DEVICE) -> None:
    _check(lib().fd_set_model(g, _ptr(vz), _ptr(eps), _ptr(delta), ptr_kind))


def fd_add_source(g, ix, iy, iz, freq_hz, t0, amp, inject_q=0) -> None:
    _check(lib().fd_add_source(g, ix, iy, iz, freq_hz, t0, amp, int(inject_q)))


def fd_add_source_series(g, ix, iy, iz, s, nt, inject_q=0) -> None:
    _check(lib().fd_add_source_series(g, ix, iy, iz, _ptr(s), nt, int(inject_q)))


def fd_set_receivers(g, idx, nrec, trace_dev, nt_cap) -> None:
    _check(lib().fd_set_receivers(g, _ptr(idx), nrec, _ptr(trace_dev), nt_cap))


def fd_step(g) -> None:
    _check(lib().fd_step(g))


def fd_step_from(g, cur, prev, out) -> None:
    _check(lib().fd_step_from(g, _ptr(cur), _ptr(prev), _ptr(out)))


def fd_run(g, nsteps: int) -> None:
    _check(lib().fd_run(g, nsteps))


def fd_set_graph(g, steps: int) -> None:
    _check(lib().fd_set_graph(g, steps))


def fd_set_launch(g, tx, ty, zchunk, lookahead) -> None:
    _check(lib().fd_set_launch(g, tx, ty, zchunk, lookahead))


def fd_read_receivers(g, t_begin, t_count, dst, dst_kind) -> None:
    _check(lib().fd_read_receivers(g, t_begin, t_count, _ptr(dst), dst_kind))


def fd_run_to_host(g, nsteps, host_dst, chunk_steps=0) -> None:
    _check(lib().fd_run_to_host(g, nsteps, _ptr(host_dst), chunk_steps))


def fd_get_state(g, cur=None, prev=None, q_cur=None, q_prev=None, ptr_kind=FD_PTR_HOST) -> int:
    n = _i()
    _check(lib().fd_get_state(g, _ptr(cur), _ptr(prev), _ptr(q_cur), _ptr(q_prev), ptr_kind,
                              ctypes.byref(n)))
    return n.value


def fd_set_state(g, cur=None, prev=None, q_cur=None, q_prev=None, ptr_kind=FD_PTR_HOST,
                 time_index=0) -> None:
    _check(lib().fd_set_state(g, _ptr(cur), _ptr(prev), _ptr(q_cur), _ptr(q_prev), ptr_kind,
                              time_index))


def fd_field(g, which: int):
    p, pitch = _vp(), _i()
    _check(lib().fd_field(g, which, ctypes.byref(p), ctypes.byref(pitch)))
    return p.value, pitch.value


def fd_time_index(g) -> int:
    n = _i()
    _check(lib().fd_time_index(g, ctypes.byref(n)))
    return n.value


def fd_sync(g) -> None:
    _check(lib().fd_sync(g))


def fd_destroy_grid(g) -> None:
    _check(lib().fd_destroy_grid(g))


def fd_iso_step_static(d: fd_desc, u_cur, u_prev, kappa, n, src=None, freq_hz=15.0, t0=None,
                       amp=1.0, status=None, stream=0) -> None:
    """One isotropic step with no device allocation (see include/fd.h).
    `status`: optional device int32 tensor that receives FD_OK or FD_ERR_TIMEOUT."""
    sx, sy, sz = (-1, -1, -1) if src is None else src
    t0 = 1.0 / freq_hz if t0 is None else t0
    _check(lib().fd_iso_step_static(ctypes.byref(d), _ptr(u_cur), _ptr(u_prev), _ptr(kappa), n,
                                    sx, sy, sz, freq_hz, t0, amp, _ptr(status), stream))


def fd_set_injection(g, idx, nrec, values_dev, nt_cap) -> None:
    _check(lib().fd_set_injection(g, _ptr(idx), nrec, _ptr(values_dev), nt_cap))


def fd_adjoint_source(g, traces, dobs, nt, inj) -> float:
    J = ctypes.c_double()
    _check(lib().fd_adjoint_source(g, _ptr(traces), _ptr(dobs), nt, _ptr(inj), ctypes.byref(J)))
    return J.value


def fd_grad_accumulate(g, z, a, grad) -> None:
    _check(lib().fd_grad_accumulate(g, _ptr(z), _ptr(a), _ptr(grad)))


def fd_optimized_weights(radius: int, kmax: float) -> np.ndarray:
    """Band-optimised unit-grid second-derivative weights c_0..c_radius."""
    out = np.zeros(radius + 1, dtype=np.float64)
    _check(lib().fd_optimized_weights(radius, kmax, out.ctypes.data))
    return out


def fd_set_weights(g, w_xy=None, w_z=None) -> None:
    a = None if w_xy is None else np.ascontiguousarray(w_xy, dtype=np.float64)
    b = None if w_z is None else np.ascontiguousarray(w_z, dtype=np.float64)
    _check(lib().fd_set_weights(g, _ptr(a), _ptr(b)))


def fd_debug_skip_copy(g, plane: int) -> None:
    _check(lib().fd_debug_skip_copy(g, plane))


def fd_set_z_window(g, kg0: int, nz_global: int) -> None:
    _check(lib().fd_set_z_window(g, kg0, nz_global))


def fd_halo_exchange(lower, upper, planes: int) -> None:
    _check(lib().fd_halo_exchange(lower, upper, planes))


def fd_step_planes(g, k_begin: int, k_end: int, complete: bool) -> None:
    _check(lib().fd_step_planes(g, k_begin, k_end, int(bool(complete))))


def fd_batch_create(stream: int) -> int:
    out = _vp()
    _check(lib().fd_batch_create(stream, ctypes.byref(out)))
    return out.value


def fd_batch_set_launch(b, radius, tx, ty, zchunk, lookahead) -> None:
    _check(lib().fd_batch_set_launch(b, radius, tx, ty, zchunk, lookahead))


def fd_batch_set_graph(b, steps: int) -> None:
    _check(lib().fd_batch_set_graph(b, steps))


def fd_batch_add(b, g, nsteps: int) -> None:
    _check(lib().fd_batch_add(b, g, nsteps))


def fd_batch_remove(b, g) -> None:
    _check(lib().fd_batch_remove(b, g))


def fd_batch_steps_left(b, g) -> int:
    n = _i()
    _check(lib().fd_batch_steps_left(b, g, ctypes.byref(n)))
    return n.value


def fd_batch_run(b, max_steps: int) -> int:
    n = _i()
    _check(lib().fd_batch_run(b, max_steps, ctypes.byref(n)))
    return n.value


def fd_batch_destroy(b) -> None:
    _check(lib().fd_batch_destroy(b))


# ---- one shot on the GPU ---------------------------------------------------------

@dataclass
class GridSpec:
    mode: int
    nx: int
    ny: int
    nz: int
    r_xy: int
    r_z: int
    h: float
    dz: float
    dt: float
    sponge_width: int = 0
    sponge_a: float = 0.0
    dz_k: np.ndarray | None = None

    @classmethod
    def from_shot(cls, s) -> "GridSpec":
        return cls(mode=FD_MODE_VTI if s.mode == "vti" else FD_MODE_ISO, nx=s.nx, ny=s.ny, nz=s.nz,
                   r_xy=s.r_xy, r_z=s.r_z, h=s.h, dz=s.dz if s.dz is not None else s.h, dt=s.dt,
                   sponge_width=s.nb, sponge_a=s.sponge_a if s.nb else 0.0, dz_k=s.dzk)

    def desc(self):
        return make_desc(self.mode, self.nx, self.ny, self.nz, self.r_xy, self.r_z, self.h, self.dz,
                         self.dt, self.sponge_width, self.sponge_a, self.dz_k)


class Grid:
    """A grid handle with its torch-allocated arena (and trace buffer) on one device."""

    def __init__(self, spec: GridSpec, device=None, stream=None):
        import torch
        self.torch = torch
        self.spec = spec
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        self._desc, self._keep = spec.desc()
        self.layout = fd_layout(self._desc)
        nbytes = self.layout.arena_bytes
        with torch.cuda.device(self.device):
            self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            off = (-self.arena.data_ptr()) % 256
            self.arena_ptr = self.arena.data_ptr() + off
            self.h = fd_create_grid(self._desc, self.arena_ptr, nbytes, self.stream.cuda_stream)
        self.trace = None
        self.nrec = 0

    # model / source / receivers -------------------------------------------------
    def set_model(self, vz, eps=None, delta=None):
        """Dense (nz, ny, nx) float32 arrays: numpy (host path) or CUDA tensors."""
        torch = self.torch
        if isinstance(vz, torch.Tensor):
            args = [vz.contiguous()] + [None if a is None else a.contiguous() for a in (eps, delta)]
            with torch.cuda.device(self.device):
                fd_set_model(self.h, *args, ptr_kind=FD_PTR_DEVICE)
        else:
            args = [np.ascontiguousarray(vz, np.float32)] + \
                   [None if a is None else np.ascontiguousarray(a, np.float32) for a in (eps, delta)]
            with torch.cuda.device(self.device):
                fd_set_model(self.h, *args, ptr_kind=FD_PTR_HOST)

    def add_source(self, ix, iy, iz, freq_hz=15.0, t0=None, amp=1.0, inject_q=False):
        t0 = 1.0 / freq_hz if t0 is None else t0
        fd_add_source(self.h, ix, iy, iz, freq_hz, t0, amp, inject_q)

    def set_receivers(self, idx, nt_cap: int):
        torch = self.torch
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(-1, 3))
        self.nrec = len(idx)
        with torch.cuda.device(self.device):
            self.trace = torch.zeros((max(nt_cap, 1), max(self.nrec, 1)), dtype=torch.float32,
                                     device=self.device)
        fd_set_receivers(self.h, idx, self.nrec, self.trace, nt_cap)

    # stepping ----------------------------------------------------------------------
    def step(self):
        with self.torch.cuda.device(self.device):
            fd_step(self.h)

    def run(self, nsteps: int):
        with self.torch.cuda.device(self.device):
            fd_run(self.h, nsteps)

    def step_planes(self, k_begin: int, k_end: int, complete: bool):
        """Part of a step: planes [k_begin, k_end) (see fd_step_planes)."""
        with self.torch.cuda.device(self.device):
            fd_step_planes(self.h, k_begin, k_end, complete)

    def set_graph(self, steps: int):
        fd_set_graph(self.h, steps)

    def set_launch(self, tx, ty, zchunk, lookahead):
        fd_set_launch(self.h, tx, ty, zchunk, lookahead)

    def sync(self):
        with self.torch.cuda.device(self.device):
            fd_sync(self.h)

    @property
    def time_index(self) -> int:
        return fd_time_index(self.h)

    def run_to_host(self, nsteps: int, out=None, chunk_steps: int = 0):
        """nsteps steps with their receiver rows streamed to host memory while
        later steps compute (fd_run_to_host); returns the (nsteps, nrec) rows
        (`out` if given: pinned memory lets the copies run asynchronously)."""
        torch = self.torch
        if out is None:
            out = torch.empty((nsteps, max(self.nrec, 1)), dtype=torch.float32).pin_memory()
        with torch.cuda.device(self.device):
            fd_run_to_host(self.h, nsteps, out, chunk_steps)
        return out

    # read back --------------------------------------------------------------------
    def traces(self, t_begin=0, t_count=None) -> np.ndarray:
        if t_count is None:
            t_count = self.time_index - t_begin
        out = np.empty((t_count, self.nrec), dtype=np.float32)
        with self.torch.cuda.device(self.device):
            fd_read_receivers(self.h, t_begin, t_count, out, FD_PTR_HOST)
        return out

    def state(self):
        """(cur, prev[, q_cur, q_prev]) as dense (nz, ny, nx) float32 numpy arrays."""
        s = self.spec
        shape = (s.nz, s.ny, s.nx)
        arrs = [np.empty(shape, np.float32) for _ in range(4 if s.mode == FD_MODE_VTI else 2)]
        with self.torch.cuda.device(self.device):
            fd_get_state(self.h, *arrs, ptr_kind=FD_PTR_HOST)
        return tuple(arrs)

    def field_view(self, which: int = 0):
        """A (nz, ny, pitch) torch view of a stored level (valid until the next step)."""
        torch = self.torch
        ptr, pitch = fd_field(self.h, which)
        s = self.spec
        off = ptr - self.arena.data_ptr()
        nbytes = s.nz * s.ny * pitch * 4
        return self.arena[off:off + nbytes].view(torch.float32).view(s.nz, s.ny, pitch)

    def model_view(self, m: int = 0):
        """A (nz, ny, pitch) torch view of model buffer m (kappa; VTI: kx, kn, kz)."""
        torch = self.torch
        s, lay = self.spec, self.layout
        off = self.arena_ptr - self.arena.data_ptr() + (lay.nfields + m) * lay.field_bytes
        nbytes = s.nz * s.ny * lay.pitch * 4
        return self.arena[off:off + nbytes].view(torch.float32).view(s.nz, s.ny, lay.pitch)

    def close(self):
        if getattr(self, "h", None):
            with self.torch.cuda.device(self.device):
                fd_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_from_shot(shot, device=None, nt_cap=None, model=True, receivers=True) -> Grid:
    """Grid for a ``synth.Shot`` with its model, source and receivers set."""
    g = Grid(GridSpec.from_shot(shot), device=device)
    if model:
        g.set_model(shot.v, shot.eps, shot.delta) if shot.mode == "vti" else g.set_model(shot.v)
    if shot.src is not None:
        g.add_source(*shot.src, freq_hz=shot.src_f, t0=shot.src_t0, amp=shot.src_amp,
                     inject_q=shot.src_into_q)
    if receivers and shot.receivers is not None and len(shot.receivers):
        g.set_receivers(shot.receivers, shot.nsteps if nt_cap is None else nt_cap)
    return g
