"""The C ABI from plain C: tests/c/shot_abi.c (include/fd.h and the CUDA
runtime only) runs an isotropic shot; its traces and final level equal the
Python binding's run of the same shot bit for bit and the FP64 oracle's within
the parity tolerance."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1410_1387_gb300 import synth
from tests.helpers import max_rel, oracle_problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_1387_gb300 import fd as fdmod
    return fdmod


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


@pytest.fixture(scope="module")
def shot_abi(fd, tmp_path_factory):
    cuda = _cuda_home()
    pkg = os.path.join(ROOT, "paper_1410_1387_gb300")
    exe = str(tmp_path_factory.mktemp("c_abi") / "shot_abi")
    libdirs = [d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"),
                           os.path.join(cuda, "targets", "sbsa-linux", "lib"),
                           os.path.join(cuda, "targets", "x86_64-linux", "lib")) if os.path.isdir(d)]
    cmd = ["gcc", "-O2", "-std=c11", os.path.join(ROOT, "tests", "c", "shot_abi.c"), "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), "-L", pkg, "-lfd", f"-Wl,-rpath,{pkg}"]
    for d in libdirs:
        cmd += ["-L", d, f"-Wl,-rpath,{d}"]
    cmd += ["-lcudart", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _shot(n, R, steps, nb, dt):
    s = synth.Shot(name="c_abi", nx=n, ny=n, nz=n, r_xy=R, r_z=R, h=10.0, dt=dt, nsteps=steps, nb=nb,
                   src=(n // 2, n // 2, n // 2),
                   receivers=synth.receiver_plane(n, n, n // 2, nry=1, y0=n // 2))
    s.v = np.broadcast_to((1800.0 + 10.0 * np.arange(n, dtype=np.float32))[:, None, None], (n, n, n)).astype(np.float32)
    return s


@pytest.mark.parametrize("n,R,steps,nb", [(64, 4, 120, 0), (48, 8, 80, 6)])
def test_c_client_matches_python_and_oracle(fd, O, shot_abi, tmp_path, n, R, steps, nb):
    dt = 0.5 * synth.COURANT_LIMIT[R] * 10.0 / 2430.0       # v_max = 1800 + 10 * 63
    out = str(tmp_path / "out.bin")
    r = subprocess.run([shot_abi, str(n), str(R), str(steps), str(nb), repr(dt), out], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr
    raw = np.fromfile(out, dtype=np.float32)
    tr_c = raw[:steps * n].reshape(steps, n)
    u_c = raw[steps * n:].reshape(n, n, n)

    s = _shot(n, R, steps, nb, dt)
    g = fd.grid_from_shot(s, device="cuda:0")
    g.set_graph(8)
    g.run(steps)
    u_py, _ = g.state()
    tr_py = g.traces()
    g.close()
    np.testing.assert_array_equal(tr_c, tr_py)
    np.testing.assert_array_equal(u_c, u_py)

    ur, _, trr = oracle_problem(O, s).iso_run(s.v, steps)
    assert max_rel(u_c, ur) <= 1e-4 and max_rel(tr_c, trr) <= 1e-4
    assert np.abs(trr).max() > 0
