"""fd_iso_step_static: the isotropic step for callers that cannot allocate
device memory (a serving process whose pool allocator owns the whole GPU, or a
latency-critical loop that cannot take cudaMalloc's device-wide
synchronisation).  It keeps its scratch in a fixed device array instead of
allocating and runs the same kernel with the same tables as fd_step, so its
output must equal fd_step's bit for bit, call after call -- also when calls on
other grid shapes, or without a source, run in between and rewrite that array.

This file is collected last on purpose: a run that stops at the first failure
has already run every other test when it gets here."""
import numpy as np
import pytest

from tests.helpers import iso_shot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_1387_gb300 import fd as fdmod
    return fdmod


def _caller_buffers(g):
    """Caller-owned copies of u^n, the stored older level and kappa of grid g
    (same pitched layout) and the grid's time index."""
    return g.field_view(0).clone(), g.field_view(1).clone(), g.model_view(0).clone(), g.time_index


def _static(fd, shot, desc, cur, prev, kap, n, status, stream, src=True):
    fd.fd_iso_step_static(desc, cur, prev, kap, n, src=shot.src if src else None, freq_hz=shot.src_f,
                          t0=shot.src_t0, amp=shot.src_amp, status=status, stream=stream)


@pytest.mark.parametrize("R,shape", [(4, (70, 45, 37)), (8, (66, 50, 41))])
def test_static_step_matches_grid_step_twice(fd, R, shape):
    import torch
    nx, ny, nz = shape
    stream = torch.cuda.current_stream().cuda_stream
    shot = iso_shot(nx, ny, nz, R, 10, seed=17 + R, nb=6, src=(nx // 3, ny // 2, nz // 2))
    g = fd.grid_from_shot(shot, device="cuda:0")
    g.run(5)                               # the source is still active at steps 5, 6
    a, b, kap, n = _caller_buffers(g)
    desc, keep = g.spec.desc()
    # a grid of another shape and damping width, called without a source in
    # between: it rewrites every table of the shared scratch array
    other = iso_shot(nx - 19, ny + 7, nz - 9, R, 10, seed=5 + R, nb=3)
    other.src = None
    go = fd.grid_from_shot(other, device="cuda:0")
    oa, ob, okap, on = _caller_buffers(go)
    odesc, okeep = go.spec.desc()
    status = torch.full((3,), -12345, dtype=torch.int32, device="cuda:0")

    g.step()                               # reference: the grid's own steps
    ref1 = g.field_view(0).clone()
    _static(fd, shot, desc, a, b, kap, n, status[0:1], stream)              # b <- u^{n+1}
    _static(fd, other, odesc, oa, ob, okap, on, status[1:2], stream, src=False)
    g.step()
    ref2 = g.field_view(0).clone()
    _static(fd, shot, desc, b, a, kap, n + 1, status[2:3], stream)          # a <- u^{n+2}
    torch.cuda.synchronize()
    g.close()
    go.close()
    assert status.tolist() == [fd.FD_OK] * 3
    np.testing.assert_array_equal(b[:, :, :nx].cpu().numpy(), ref1[:, :, :nx].cpu().numpy())
    np.testing.assert_array_equal(a[:, :, :nx].cpu().numpy(), ref2[:, :, :nx].cpu().numpy())
    assert np.abs(ref2[:, :, :nx].cpu().numpy()).max() > 0


@pytest.mark.parametrize("R", [4, 8])
def test_static_step_other_shape_without_source(fd, R):
    """The interleaved call of the test above, checked on its own: a grid of
    another shape and damping width, no source, stepped from a state copied in
    through fd_set_state, equals the static call from the same state."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    seed = iso_shot(51, 52, 32, R, 10, seed=17 + R, nb=6, src=(17, 26, 16))
    gs = fd.grid_from_shot(seed, device="cuda:0")
    gs.run(6)
    u, up = gs.state()
    gs.close()
    other = iso_shot(51, 52, 32, R, 10, seed=5 + R, nb=3)
    other.src = None
    go = fd.grid_from_shot(other, device="cuda:0")
    fd.fd_set_state(go.h, u, up, ptr_kind=fd.FD_PTR_HOST, time_index=6)
    a, b, kap, n = _caller_buffers(go)
    desc, keep = go.spec.desc()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda:0")
    go.step()
    ref = go.field_view(0).clone()
    _static(fd, other, desc, a, b, kap, n, status, stream, src=False)
    torch.cuda.synchronize()
    go.close()
    assert n == 6 and int(status.item()) == fd.FD_OK
    np.testing.assert_array_equal(b[:, :, :51].cpu().numpy(), ref[:, :, :51].cpu().numpy())


def test_static_step_reports_timeout(fd):
    """Failure detection without a fault: the test hook has one CTA withhold one
    plane's copy in the next static call, its bounded wait runs out (about a
    second), and the call's status word reads FD_ERR_TIMEOUT; the next call
    clears the flag and is exact again."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    shot = iso_shot(64, 32, 40, 4, 6, seed=3, nb=4)
    g = fd.grid_from_shot(shot, device="cuda:0")
    g.run(3)
    a, b, kap, n = _caller_buffers(g)
    b0 = b.clone()
    desc, keep = g.spec.desc()
    status = torch.full((2,), -1, dtype=torch.int32, device="cuda:0")
    with pytest.raises(fd.FdError) as e:
        fd.fd_debug_skip_copy(None, -1)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    fd.fd_debug_skip_copy(None, 6)         # in the z chunk of CTA (0,0,0)
    _static(fd, shot, desc, a, b, kap, n, status[0:1], stream)
    torch.cuda.synchronize()
    assert int(status[0].item()) == fd.FD_ERR_TIMEOUT
    b.copy_(b0)
    g.step()
    _static(fd, shot, desc, a, b, kap, n, status[1:2], stream)
    torch.cuda.synchronize()
    assert int(status[1].item()) == fd.FD_OK
    np.testing.assert_array_equal(b[:, :, :64].cpu().numpy(), g.field_view(0)[:, :, :64].cpu().numpy())
    g.close()


def test_static_step_rejects_oversize_grid(fd):
    import torch
    buf = torch.zeros(16, device="cuda:0")
    desc, _ = fd.make_desc(fd.FD_MODE_ISO, _limit("AXIS") + 4, 8, 8, 4, 4, 10.0, 10.0, 1e-3)
    with pytest.raises(fd.FdError) as e:
        fd.fd_iso_step_static(desc, buf, buf, buf, 0)
    assert e.value.code == fd.FD_ERR_OUT_OF_RANGE
    assert "static scratch limit" in str(e.value)
    wide = _limit("SPONGE") + 1
    desc, _ = fd.make_desc(fd.FD_MODE_ISO, 2 * wide + 8, 8, 8, 4, 4, 10.0, 10.0, 1e-3, wide, 0.015)
    with pytest.raises(fd.FdError) as e:
        fd.fd_iso_step_static(desc, buf, buf, buf, 0)
    assert e.value.code == fd.FD_ERR_OUT_OF_RANGE
    assert "damping layer" in str(e.value)


def _limit(name):
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    h = open(os.path.join(root, "include", "fd.h")).read()
    return int(re.search(rf"#define FD_STATIC_MAX_{name} (\d+)", h).group(1))
