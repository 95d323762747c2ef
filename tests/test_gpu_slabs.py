"""One shot cut into z slabs on one GPU, ghost planes exchanged by the library
after every step: every level and every trace equals the unsplit grid's bit
for bit (isotropic R = 4 and 8 with the damping layer across the cuts, VTI with
uniform dz), and the exchange rejects slabs that do not fit together."""
import numpy as np
import pytest

from paper_1410_1387_gb300 import slabs, synth
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


def _compare(fd, shot, nslabs):
    ref = fd.grid_from_shot(shot, device="cuda:0")
    ref.run(shot.nsteps)
    st_ref, tr_ref = ref.state(), ref.traces()
    ss = slabs.SlabShot(shot, nslabs, device="cuda:0")
    ss.run(shot.nsteps)
    ss.sync()
    st, tr = ss.state(), ss.traces()
    for a, b in zip(st, st_ref):
        assert np.array_equal(a, b)
    assert np.array_equal(tr, tr_ref)
    assert np.abs(st_ref[0]).max() > 0 and np.abs(tr_ref).max() > 0
    ss.close()
    ref.close()


@pytest.mark.parametrize("R,nslabs", [(4, 3), (4, 2), (8, 2)])
def test_iso_slabs_bitwise(fd, R, nslabs):
    nz = 80 if R == 4 else 72
    rec = synth.receiver_plane(64, 48, 30, stride=2)
    shot = iso_shot(64, 48, nz, R, 60, seed=21, nb=10, src=(32, 24, nz // 2 - 1), receivers=rec)
    _compare(fd, shot, nslabs)


def test_vti_slabs_bitwise(fd):
    s = synth.vti_shot(48, nsteps=40, seed=4, with_model=False)
    s.dzk, s.dz, s.nb = None, s.h, 6
    s.src = (24, 20, 23)
    s.receivers = synth.receiver_plane(48, 48, 10, stride=3)
    s.v = synth.layered_model(48, 48, 48, 4)
    s.eps, s.delta = synth.layered_anisotropy(48, 48, 48, 4)
    _compare(fd, s, 2)


def test_exchange_rejects_mismatched_slabs(fd):
    shot = iso_shot(32, 32, 40, 4, 4, seed=2, nb=4)
    ss = slabs.SlabShot(shot, 2, device="cuda:0")
    lo, up = ss.grids
    with pytest.raises(fd.FdError) as e:
        fd.fd_halo_exchange(lo.h, up.h, 3)            # fewer planes than the radius
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FdError) as e:
        fd.fd_halo_exchange(up.h, lo.h, 4)            # wrong order: windows do not overlap
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FdError) as e:
        fd.fd_halo_exchange(lo.h, lo.h, 4)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    lo.run(1)
    with pytest.raises(fd.FdError) as e:
        fd.fd_halo_exchange(lo.h, up.h, 4)            # different time indices
    assert e.value.code == fd.FD_ERR_BAD_STATE
    with pytest.raises(fd.FdError) as e:
        fd.fd_set_z_window(lo.h, 30, 40)              # 24 planes from 30 overrun 40
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    ss.close()
    vs = synth.vti_shot(32, nsteps=2, seed=1)
    g = fd.grid_from_shot(vs, device="cuda:0")
    with pytest.raises(fd.FdError) as e:
        fd.fd_set_z_window(g.h, 0, 64)                # stretched dz
    assert e.value.code == fd.FD_ERR_UNSUPPORTED
    g.close()
