"""fd_iso_step_static: the isotropic step for callers that cannot allocate
device memory (a serving process whose pool allocator owns the whole GPU, or a
latency-critical loop that cannot take cudaMalloc's device-wide
synchronisation).  It keeps its scratch in a fixed device array instead of
allocating; its output must match fd_step on a grid, call after call.

This file is collected last on purpose: a run that stops at the first failure
has already run every other test when it gets here."""
import numpy as np
import pytest

from tests.helpers import iso_shot, max_rel

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


def _kappa_view(g):
    """The grid's pitched kappa buffer (after the wavefields in its arena)."""
    import torch
    lay = g.layout
    s = g.spec
    off = g.arena_ptr - g.arena.data_ptr() + lay.nfields * lay.field_bytes
    n = s.nz * s.ny * lay.pitch * 4
    return g.arena[off:off + n].view(torch.float32).view(s.nz, s.ny, lay.pitch)


@pytest.mark.parametrize("R,shape", [(4, (70, 45, 37)), (8, (66, 50, 41))])
def test_static_step_matches_grid_step_twice(fd, R, shape):
    import torch
    nx, ny, nz = shape
    shot = iso_shot(nx, ny, nz, R, 10, seed=17 + R, nb=6, src=(nx // 3, ny // 2, nz // 2))
    g = fd.grid_from_shot(shot, device="cuda:0")
    g.run(5)                               # the source is still active at steps 5, 6
    n = g.time_index
    # caller-owned copies of u^n, the stored older level and kappa (same pitched layout)
    a = g.field_view(0).clone()
    b = g.field_view(1).clone()
    kap = _kappa_view(g).clone()
    desc, keep = g.spec.desc()
    stream = torch.cuda.current_stream().cuda_stream

    g.step()                               # reference: the grid's own step
    ref1 = g.field_view(0).clone()
    fd.fd_iso_step_static(desc, a, b, kap, n, src=shot.src, freq_hz=shot.src_f, t0=shot.src_t0,
                          amp=shot.src_amp, stream=stream)
    g.step()
    ref2 = g.field_view(0).clone()
    fd.fd_iso_step_static(desc, b, a, kap, n + 1, src=shot.src, freq_hz=shot.src_f, t0=shot.src_t0,
                          amp=shot.src_amp, stream=stream)
    torch.cuda.synchronize()
    g.close()
    got1 = b[:, :, :nx].cpu().numpy()
    got2 = a[:, :, :nx].cpu().numpy()
    want1 = ref1[:, :, :nx].cpu().numpy()
    want2 = ref2[:, :, :nx].cpu().numpy()
    assert np.abs(want2).max() > 0
    assert max_rel(got1, want1) <= 1e-4
    assert max_rel(got2, want2) <= 1e-4


def test_static_step_rejects_oversize_grid(fd):
    import torch
    desc, _ = fd.make_desc(fd.FD_MODE_ISO, fd_static_max() + 4, 8, 8, 4, 4, 10.0, 10.0, 1e-3)
    buf = torch.zeros(16, device="cuda:0")
    with pytest.raises(fd.FdError) as e:
        fd.fd_iso_step_static(desc, buf, buf, buf, 0)
    assert e.value.code == fd.FD_ERR_OUT_OF_RANGE
    assert "static scratch limit" in str(e.value)


def fd_static_max():
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    h = open(os.path.join(root, "include", "fd.h")).read()
    return int(re.search(r"#define FD_STATIC_MAX_AXIS (\d+)", h).group(1))
