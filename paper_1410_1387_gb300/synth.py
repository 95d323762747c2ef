"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds none of the method's arithmetic: it draws velocity and
anisotropy models, z spacings, receiver lattices and shot lists from a seed,
and states the time steps of the named workloads as literals.  Both the CUDA
path and the CPU oracle receive what it returns as plain inputs.

The paper's benchmark case is not specified (Sec. 4 says only "representative
synthetic test case"), so the shapes below are the workloads this project is
measured on: a 64^3 constant-velocity parity case, a 512^3 layered single shot,
and a 512^3 layered VTI shot.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Largest stable Courant number v*dt/h of the 3D isotropic leapfrog scheme with
# the order-2R Taylor stencil and dx = dy = dz (2 / sqrt(3 sigma_R), where
# sigma_R is the stencil's symbol at the Nyquist frequency).  Literals; a test
# pins them against the oracle and against the growth of the Nyquist mode.
COURANT_LIMIT = {4: 0.45285552331841994, 8: 0.42370633104984806, 12: 0.41192031573908844}

# Velocity ceiling of the layered models: 4500 m/s plus the 5 % cell noise.
V_MAX_LAYERED = 4500.0 * 1.05


@dataclass
class Shot:
    """One isotropic or VTI shot: grid, radii, spacings, source, receivers, model."""
    name: str
    nx: int
    ny: int
    nz: int
    r_xy: int
    r_z: int
    h: float
    dt: float
    nsteps: int
    mode: str = "iso"                 # "iso" or "vti"
    dz: float | None = None           # uniform dz (defaults to h)
    dzk: np.ndarray | None = None     # VTI: nz-1 plane spacings
    nb: int = 0                       # damping-layer width
    sponge_a: float = 0.015
    src: tuple[int, int, int] | None = None
    src_f: float = 15.0
    src_t0: float = 1.0 / 15.0
    src_amp: float = 1.0
    src_into_q: bool = False
    receivers: np.ndarray | None = None   # (M, 3) int32 [ix, iy, iz]
    v: np.ndarray | None = None           # (nz, ny, nx) float32: v (iso) or v_z (vti)
    eps: np.ndarray | None = None
    delta: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return self.nx * self.ny * self.nz


def receiver_plane(nx: int, ny: int, k: int, stride: int = 1, x0: int = 0, y0: int = 0,
                   nrx: int | None = None, nry: int | None = None) -> np.ndarray:
    """Receivers on a regular lattice of plane k, row-major (y outer, x inner)."""
    nrx = (nx - x0 + stride - 1) // stride if nrx is None else nrx
    nry = (ny - y0 + stride - 1) // stride if nry is None else nry
    ys, xs = np.meshgrid(y0 + stride * np.arange(nry), x0 + stride * np.arange(nrx), indexing="ij")
    out = np.empty((nry * nrx, 3), dtype=np.int32)
    out[:, 0] = xs.ravel()
    out[:, 1] = ys.ravel()
    out[:, 2] = k
    return out


def layered_model(nx: int, ny: int, nz: int, seed: int, nlayers: int = 10,
                  vmin: float = 1500.0, vmax: float = 4500.0, noise: float = 0.05) -> np.ndarray:
    """Layered velocity (nz, ny, nx) float32: nlayers layers with boundaries at
    sorted uniform depths, layer speeds uniform in [vmin, vmax], then every
    cell scaled by 1 + U(-noise, noise)."""
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.integers(1, max(nz, 2), size=nlayers - 1))
    speeds = rng.uniform(vmin, vmax, size=nlayers)
    layer_of_k = np.searchsorted(cuts, np.arange(nz), side="right")
    vk = speeds[layer_of_k].astype(np.float32)
    v = np.empty((nz, ny, nx), dtype=np.float32)
    for k in range(nz):
        v[k] = vk[k] * (1.0 + rng.uniform(-noise, noise, size=(ny, nx))).astype(np.float32)
    return v


def layered_anisotropy(nz: int, ny: int, nx: int, seed: int, nlayers: int = 10,
                       eps_max: float = 0.25):
    """Per-layer Thomsen parameters: eps ~ U[0, eps_max], delta ~ U[0, eps]."""
    rng = np.random.default_rng(seed + 7919)
    cuts = np.sort(rng.integers(1, max(nz, 2), size=nlayers - 1))
    e = rng.uniform(0.0, eps_max, size=nlayers)
    d = rng.uniform(0.0, 1.0, size=nlayers) * e
    lk = np.searchsorted(cuts, np.arange(nz), side="right")
    eps = np.broadcast_to(e[lk].astype(np.float32)[:, None, None], (nz, ny, nx)).copy()
    delta = np.broadcast_to(d[lk].astype(np.float32)[:, None, None], (nz, ny, nx)).copy()
    return eps, delta


def stretched_dz(nz: int, h: float, seed: int, amp: float = 0.10) -> np.ndarray:
    """nz-1 smoothly varying plane spacings h (1 + amp sin(2 pi k / nz + phase))."""
    rng = np.random.default_rng(seed + 104729)
    phase = rng.uniform(0.0, 2.0 * np.pi)
    k = np.arange(nz - 1, dtype=np.float64)
    return h * (1.0 + amp * np.sin(2.0 * np.pi * k / max(nz - 1, 1) + phase))


def random_model(nx: int, ny: int, nz: int, seed: int, lo: float = 1500.0, hi: float = 4500.0):
    """Cell-wise uniform random velocity (a rough model for parity tests)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(nz, ny, nx)).astype(np.float32)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def parity_shot_64() -> Shot:
    """64^3 constant v = 2000 m/s, h = 10 m, radius 4, 200 steps, Ricker 15 Hz at
    the centre cell, zero boundary, no damping layer.  dt is half the stability
    limit: 0.5 * COURANT_LIMIT[4] * 10 / 2000 = 1.1321388082960499e-3 s."""
    n = 64
    s = Shot(name="iso64_r4", nx=n, ny=n, nz=n, r_xy=4, r_z=4, h=10.0,
             dt=1.1321388082960499e-3, nsteps=200, nb=0, src=(32, 32, 32),
             receivers=receiver_plane(n, n, 32, nry=1, y0=32))
    s.v = np.full((n, n, n), 2000.0, dtype=np.float32)
    return s


def layered_shot(n: int = 512, R: int = 4, nsteps: int = 1000, seed: int = 1,
                 with_model: bool = True) -> Shot:
    """Single large shot: n^3 layered model (10 layers, 1500-4500 m/s, +-5 %
    noise), h = 10 m, 20-cell damping layer inside the grid, Ricker 15 Hz at
    (n/2, n/2, 30) (10 cells below the layer), an n x n receiver plane at k = 20
    (the first plane below the layer).  dt = 0.5 * limit * h / v_max."""
    h = 10.0
    dt = 0.5 * COURANT_LIMIT[R] * h / V_MAX_LAYERED
    nb = 20 if n > 60 else max(2, n // 6)
    s = Shot(name=f"iso{n}_r{R}_layered", nx=n, ny=n, nz=n, r_xy=R, r_z=R, h=h, dt=dt,
             nsteps=nsteps, nb=nb, src=(n // 2, n // 2, nb + 10 if n > 60 else n // 2),
             receivers=receiver_plane(n, n, nb))
    if with_model:
        s.v = layered_model(n, n, n, seed)
    return s


def vti_shot(n: int = 512, nsteps: int = 1000, seed: int = 3, r_xy: int = 12, r_z: int = 8,
             with_model: bool = True) -> Shot:
    """The paper's operator (Sec. 4: R_xy = 12, R_z = 8): n^3 layered v_z as the
    isotropic shot, per-layer eps in [0, 0.25] and delta in [0, eps], smoothly
    stretched dz_k (+-10 %), damping layer, source and receivers as above.
    dt = 0.5 times a bound on the stability limit (v_max, eps_max = 0.25,
    dz_min = 0.9 h): 3.6986e-4 s at h = 10 m."""
    h = 10.0
    nb = 20 if n > 60 else max(2, n // 6)
    s = Shot(name=f"vti{n}_r{r_xy}_{r_z}", nx=n, ny=n, nz=n, r_xy=r_xy, r_z=r_z, h=h,
             dt=VTI_DT_H10, nsteps=nsteps, mode="vti", nb=nb,
             src=(n // 2, n // 2, nb + 10 if n > 60 else n // 2),
             receivers=receiver_plane(n, n, nb))
    s.dzk = stretched_dz(n, h, seed)
    if with_model:
        s.v = layered_model(n, n, n, seed)
        s.eps, s.delta = layered_anisotropy(n, n, n, seed)
    return s


def survey_shots(count: int = 64, seed: int = 2024, n_lo: int = 96, n_hi: int = 320,
                 steps_lo: int = 300, steps_hi: int = 1500, radii=(4,), with_model: bool = True):
    """Independent shots of a survey: cubic grids n ~ U{n_lo..n_hi}, step counts
    ~ U{steps_lo..steps_hi}, radius drawn from `radii`, each with its own seeded
    layered model, damping layer, source and surface receivers (as
    ``layered_shot``)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    steps = rng.integers(steps_lo, steps_hi + 1, size=count)
    rs = rng.choice(np.asarray(radii), size=count)
    out = []
    for i in range(count):
        s = layered_shot(int(ns[i]), int(rs[i]), nsteps=int(steps[i]), seed=seed * 1000 + i,
                         with_model=with_model)
        s.name = f"survey{seed}_{i}_n{ns[i]}_r{rs[i]}"
        out.append(s)
    return out


def gradient_shot(n: int = 256, nsteps: int = 2000, seed: int = 5, amp: float = 0.10, sigma: float = 15.0):
    """Gradient workload: an n^3 layered background (radius 4, damping layer,
    source 10 cells below it) with receivers on every 2nd cell of the first
    plane below the damping layer ((n/2)^2 of them), and the true model =
    background x (1 + amp exp(-|x - c|^2 / (2 sigma^2))), a Gaussian anomaly at
    the centre.  Returns (background shot, true velocity)."""
    s = layered_shot(n, 4, nsteps=nsteps, seed=seed)
    s.receivers = receiver_plane(n, n, s.nb, stride=2)
    c = (n - 1) / 2.0
    ax = (np.arange(n) - c) ** 2
    bump = np.exp(-(ax[:, None, None] + ax[None, :, None] + ax[None, None, :]) / (2.0 * sigma * sigma))
    vtrue = (s.v * (1.0 + amp * bump)).astype(np.float32)
    s.name = f"grad{n}_r4"
    return s, vtrue


@dataclass
class Request:
    """One shot request of a served stream."""
    rid: int
    arrival: float          # seconds after the stream starts
    n: int                  # cubic grid size
    steps: int
    radius: int
    seed: int


def poisson_requests(count: int = 1000, rate: float = 20.0, seed: int = 77, n_lo: int = 128,
                     n_hi: int = 400, steps_lo: int = 500, steps_hi: int = 2000, radii=(4, 8)):
    """A Poisson stream: exponential inter-arrival times of mean 1/rate, grid
    sizes, step counts and radii drawn uniformly."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    st = rng.integers(steps_lo, steps_hi + 1, size=count)
    rs = rng.choice(np.asarray(radii), size=count)
    return [Request(i, float(t[i]), int(ns[i]), int(st[i]), int(rs[i]), seed * 100003 + i)
            for i in range(count)]


def request_shot(req: Request, receiver_stride: int = 4) -> Shot:
    """The shot of a request, without its model: layered-shot geometry, every
    `receiver_stride`-th cell of the surface plane as receivers."""
    s = layered_shot(req.n, req.radius, nsteps=req.steps, seed=req.seed, with_model=False)
    s.receivers = receiver_plane(req.n, req.n, s.nb, stride=receiver_stride)
    s.name = f"req{req.rid}"
    return s


def layered_model_device(n: int, seed: int, device, nlayers: int = 10, vmin: float = 1500.0,
                         vmax: float = 4500.0, noise: float = 0.05):
    """Layered model drawn on the GPU (torch's seeded Philox generator) so that a
    server need not build large models on the host: layer cuts and speeds as
    ``layered_model``, cell noise from torch.rand."""
    import torch
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.integers(1, max(n, 2), size=nlayers - 1))
    speeds = rng.uniform(vmin, vmax, size=nlayers)
    vk = torch.as_tensor(speeds[np.searchsorted(cuts, np.arange(n), side="right")], dtype=torch.float32,
                         device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    r = torch.rand((n, n, n), generator=gen, device=device, dtype=torch.float32)
    return vk[:, None, None] * (1.0 + noise * (2.0 * r - 1.0))


# 0.5 * 2 / sqrt(v_max^2 (1.5 * 2 sigma_12 + sigma_8 / 0.81)) * h at h = 10 m,
# v_max = 4725 m/s (sigma_R as in COURANT_LIMIT).  A literal; a test checks it
# against the oracle's stability bound for the generated tables.
VTI_DT_H10 = 3.6986e-4
