"""Adjoint and velocity gradient on the GPU (FP32): the dot-product test
<Fs, y> = <s, F^T y> to 1e-5 relative, agreement with the oracle's FP64
gradient, central finite differences, checkpoint-interval independence, and
the torch.autograd.Function."""
import numpy as np
import pytest

from paper_1410_1387_gb300 import synth
from tests.helpers import oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_1387_gb300 import adjoint, fd
    return fd, adjoint


def small_shot(n=(40, 36, 32), steps=90, seed=4, anomaly=False, R=4):
    nx, ny, nz = n
    s = synth.layered_shot(max(n), R, nsteps=steps, seed=seed, with_model=False)
    s.nx, s.ny, s.nz = nx, ny, nz
    s.nb = 5
    s.src = (nx // 2, ny // 2, 9)
    s.src_f, s.src_t0 = 25.0, 0.04
    s.receivers = synth.receiver_plane(nx, ny, 6, stride=2, x0=1, y0=1)
    v = synth.layered_model(nx, ny, nz, seed)
    if anomaly:
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        bump = np.exp(-((x - nx / 2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2) / (2 * 5.0 ** 2))
        v = (v * (1.0 + 0.1 * bump)).astype(np.float32)
    s.v = v
    return s


def test_dot_product(mods):
    import torch
    fd, adjoint = mods
    s = small_shot()
    N, nrec = s.nsteps, len(s.receivers)
    rng = np.random.default_rng(1)
    src = rng.standard_normal(N).astype(np.float32)
    F = fd.Grid(fd.GridSpec.from_shot(s), device="cuda:0")
    F.set_model(s.v)
    fd.fd_add_source_series(F.h, *s.src, src, N, 0)
    F.set_receivers(s.receivers, N)
    F.run(N)
    d = F.traces().astype(np.float64)
    y = rng.standard_normal((N, nrec)).astype(np.float32)
    yd = torch.from_numpy(y).cuda()
    inj = torch.empty_like(yd)
    fd.fd_adjoint_source(F.h, yd, torch.zeros_like(yd), N, inj)
    kap = F.model_view(0)[s.src[2], s.src[1], s.src[0]].item()
    A = fd.Grid(fd.GridSpec.from_shot(s), device="cuda:0")
    A.set_model(s.v)
    fd.fd_set_injection(A.h, np.asarray(s.receivers, np.int32), nrec, inj, N)
    A.set_receivers([list(s.src)], N)
    A.run(N)
    z = A.traces()[:, 0].astype(np.float64)
    c = s.dt ** 2 / (s.h * s.h * s.h)
    ft_y = c / kap * z[::-1]                  # (F^T y)_n = c z_{n+1}(src) / K(src)
    lhs = float(np.sum(d * y))
    rhs = float(np.sum(src.astype(np.float64) * ft_y))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))
    assert abs(lhs) > 0
    F.close()
    A.close()


def _data(fd, s_true):
    g = fd.grid_from_shot(s_true, device="cuda:0")
    g.run(s_true.nsteps)
    tr = g.traces()
    g.close()
    return tr


@pytest.mark.parametrize("R", [4, 8])
def test_gradient_matches_oracle(mods, O, R):
    import torch
    fd, adjoint = mods
    true = small_shot(anomaly=True, R=R)
    dobs = _data(fd, true)
    bg = small_shot(R=R)
    solver = adjoint.AdjointSolver(bg, checkpoint_every=20)
    J, _ = solver.forward(torch.from_numpy(bg.v).cuda(), torch.from_numpy(dobs).cuda())
    g = solver.backward().cpu().numpy().astype(np.float64)
    Jo, go = oracle_problem(O, bg).iso_misfit_grad(bg.v.astype(np.float64), dobs.astype(np.float64), bg.nsteps)
    assert J == pytest.approx(Jo, rel=1e-4)
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    cos = float(np.sum(g * go) / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert rel <= 2e-3 and cos >= 0.99999, (rel, cos)


def test_checkpoint_interval_does_not_change_the_gradient(mods):
    import torch
    fd, adjoint = mods
    true = small_shot(anomaly=True, steps=60)
    dobs = torch.from_numpy(_data(fd, true)).cuda()
    bg = small_shot(steps=60)
    v = torch.from_numpy(bg.v).cuda()
    grads = []
    for C in (7, 25, 60):
        sv = adjoint.AdjointSolver(bg, checkpoint_every=C)
        sv.forward(v, dobs)
        grads.append(sv.backward().cpu().numpy())
    np.testing.assert_array_equal(grads[0], grads[1])
    np.testing.assert_array_equal(grads[0], grads[2])


def test_finite_differences_and_autograd(mods):
    import torch
    fd, adjoint = mods
    true = small_shot(anomaly=True)
    dobs = torch.from_numpy(_data(fd, true)).cuda()
    bg = small_shot()
    v = torch.from_numpy(bg.v).cuda().requires_grad_(True)
    sv = adjoint.AdjointSolver(bg, checkpoint_every=30)
    J = adjoint.WaveMisfit.apply(v, dobs, sv)
    J.backward()
    g = v.grad.detach().double()
    # smooth direction (a wide Gaussian) so that FP32 noise does not dominate the difference
    nz, ny, nx = bg.v.shape
    z, y, x = torch.meshgrid(torch.arange(nz), torch.arange(ny), torch.arange(nx), indexing="ij")
    d = torch.exp(-((x - 15.0) ** 2 + (y - 20.0) ** 2 + (z - 14.0) ** 2) / (2 * 8.0 ** 2)).cuda()
    eps = 2.0
    Jp, _ = adjoint.AdjointSolver(bg).forward(v.detach() + eps * d, dobs)
    Jm, _ = adjoint.AdjointSolver(bg).forward(v.detach() - eps * d, dobs)
    fdiff = (Jp - Jm) / (2 * eps)
    an = float((g * d.double()).sum())
    assert an == pytest.approx(fdiff, rel=1e-2)
