"""Velocity gradient of a receiver misfit by the discrete adjoint, with
checkpoint-and-recompute, over the C ABI; and a ``torch.autograd.Function``.

For J = 1/2 sum_n sum_r (u^{n+1}(x_r) - dobs[n][r])^2 of an isotropic shot:

* forward: ``fd_run`` in segments of C steps, saving the stored pair
  (u^n, u_prev) at n = 0, C, 2C, ... (dense copies on the device);
* ``fd_adjoint_source`` turns the traces and data into the adjoint's injection
  rows (kappa(x_r) r, reversed in time) and J;
* backward, segment by segment from the last: restore the checkpoint, recompute
  the C forward levels u^n of the segment with ``fd_step_from`` (each written
  straight into a segment buffer, no copies), then run the adjoint grid one
  step per level (the same sweep kernel,
  fed by the injection lattice: z_n = G (2 z_{n+1} - G z_{n+2} + K L z_{n+1} +
  K R^T r_{n-1})) and accumulate dJ/dv += 2 dt z_{n+1} (L u^n) / sqrt(K) with
  ``fd_grad_accumulate``.

Memory: 2 N/C checkpoint fields + C - 1 segment levels + 2 grids.
"""
from __future__ import annotations

import numpy as np

from . import fd


class AdjointSolver:
    """Misfit and gradient of one isotropic shot geometry (``synth.Shot``:
    grid, radius, spacing, dt, damping, source, receiver lattice)."""

    def __init__(self, shot, checkpoint_every: int = 50, device=None):
        import torch
        self.torch = torch
        self.shot = shot
        self.C = int(checkpoint_every)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.spec = fd.GridSpec.from_shot(shot)
        self.N = shot.nsteps
        self.rec = np.ascontiguousarray(np.asarray(shot.receivers, np.int32).reshape(-1, 3))
        self.nrec = len(self.rec)
        self._state = None

    def _grid(self, v):
        g = fd.Grid(self.spec, device=self.device)
        g.set_model(v)
        return g

    def forward(self, v, dobs):
        """J for the dense (nz, ny, nx) velocity v against dobs (N, nrec), both
        CUDA float32 tensors.  Keeps what backward() needs."""
        torch = self.torch
        s, N, C = self.shot, self.N, self.C
        v = v.detach().contiguous()
        F = self._grid(v)
        if s.src is not None:
            F.add_source(*s.src, freq_hz=s.src_f, t0=s.src_t0, amp=s.src_amp)
        F.set_receivers(self.rec, N)
        shape = (s.nz, s.ny, s.nx)
        cps = []
        for n0 in range(0, N, C):
            cur = torch.empty(shape, device=self.device)
            prev = torch.empty(shape, device=self.device)
            with torch.cuda.device(self.device):
                fd.fd_get_state(F.h, cur, prev, ptr_kind=fd.FD_PTR_DEVICE)
            cps.append((n0, cur, prev))
            F.run(min(C, N - n0))
        inj = torch.empty((N, self.nrec), device=self.device)
        with torch.cuda.device(self.device):
            J = fd.fd_adjoint_source(F.h, F.trace, dobs.contiguous(), N, inj)
        self._state = (v, F, cps, inj)
        return J, F.trace

    def backward(self):
        """dJ/dv (dense, like v) for the last forward()."""
        torch = self.torch
        v, F, cps, inj = self._state
        s, N, C = self.shot, self.N, self.C
        A = self._grid(v)
        fd.fd_set_injection(A.h, self.rec, self.nrec, inj, N)
        pitch = F.layout.pitch
        grad = torch.zeros((s.nz, s.ny, pitch), device=self.device)
        seg = torch.empty((max(C - 1, 1), s.nz, s.ny, pitch), device=self.device)
        with torch.cuda.device(self.device):
            for n0, cur, prev in reversed(cps):
                ln = min(C, N - n0)
                fd.fd_set_state(F.h, cur, prev, ptr_kind=fd.FD_PTR_DEVICE, time_index=n0)
                levels = [F.field_view(0)]             # u^{n0}, in F's own buffer
                older = F.field_view(1)                # its stored older level
                for j in range(1, ln):
                    fd.fd_step_from(F.h, levels[-1], older, seg[j - 1])
                    older = levels[-1]
                    levels.append(seg[j - 1])
                for n in range(n0 + ln - 1, n0 - 1, -1):
                    fd.fd_step(A.h)                                   # z_{n+1}
                    fd.fd_grad_accumulate(F.h, A.field_view(0), levels[n - n0], grad)
        A.close()
        F.close()
        self._state = None
        return grad[:, :, :s.nx].contiguous()


class WaveMisfit:
    """``WaveMisfit.apply(v, dobs, solver)`` -> J (a 0-d tensor); J.backward()
    fills v.grad through the adjoint."""

    _fn = None

    @classmethod
    def apply(cls, v, dobs, solver):
        import torch
        if cls._fn is None:
            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, vv, dd, sv):
                    J, _ = sv.forward(vv, dd)
                    ctx.solver = sv
                    return torch.tensor(J, dtype=torch.float64, device=vv.device)

                @staticmethod
                def backward(ctx, gJ):
                    gv = ctx.solver.backward()
                    return (gv * gJ.to(gv.dtype)), None, None

            cls._fn = _F
        return cls._fn.apply(v, dobs, solver)
