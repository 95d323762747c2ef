"""Shared helpers of the GPU parity tests: oracle problems built from the same
seeded shot descriptions that the GPU path receives."""
import numpy as np

from paper_1410_1387_gb300 import synth


def oracle_problem(O, shot, receivers=True, **kw):
    return O.Problem(shot.nx, shot.ny, shot.nz, r_xy=shot.r_xy, r_z=shot.r_z, h=shot.h,
                     dz=shot.dz, dzk=shot.dzk, dt=shot.dt, nb=shot.nb,
                     sponge_a=shot.sponge_a if shot.nb else 0.0, src=shot.src, src_f=shot.src_f,
                     src_t0=shot.src_t0, src_amp=shot.src_amp, src_into_q=shot.src_into_q,
                     receivers=shot.receivers if receivers else None, **kw)


def iso_shot(nx, ny, nz, R, nsteps, seed, nb=0, src=None, receivers=None, layered=True,
             h=10.0, dz=None):
    vmax = synth.V_MAX_LAYERED if layered else 4500.0
    dzv = h if dz is None else dz
    # the stability bound with dz != h: rho = sigma (2/h^2 + 1/dz^2)
    lim = synth.COURANT_LIMIT[R] * np.sqrt(3.0 / (2.0 + (h / dzv) ** 2))
    s = synth.Shot(name="t", nx=nx, ny=ny, nz=nz, r_xy=R, r_z=R, h=h, dz=dzv,
                   dt=0.5 * lim * h / vmax, nsteps=nsteps, nb=nb,
                   src=src if src is not None else (nx // 2, ny // 2, nz // 2),
                   receivers=receivers)
    s.v = synth.layered_model(nx, ny, nz, seed) if layered else synth.random_model(nx, ny, nz, seed)
    return s


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def max_rel(a, b):
    m = np.abs(b).max()
    return np.abs(a - b).max() / (m if m > 0 else 1.0)
