"""Host logic of the default launch shape (no GPU): the wave-fitted z chunk of
launch_shape.h, compiled with the host compiler against the CUDA headers.  It
must end for every grid (an nz of 1 once made the search loop forever), stay
within [min(32, nz), cap] and nz, and at 512^3 pick 7 chunks of 74 planes on
152 SMs x 2 CTAs (radius 4) and x 3 CTAs (radius 8), and 8 of 64 for the VTI
sweep (cap 64, 2 CTAs per SM)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include "launch_shape.h"
#include <cstdio>
int main()
{
    const fdk::Launch shapes[2] = {{64, 16, 0, 3}, {32, 32, 0, 2}};
    const int xs[] = {1, 7, 64, 512, 200003}, ys[] = {1, 33, 512, 70001};
    long bad = 0;
    for (int nz = 1; nz <= 3000; ++nz)
        for (int nx : xs)
            for (int ny : ys)
                for (const fdk::Launch &L : shapes)
                    for (int hi : {96, 64}) {
                        const int z = fdk::wave_zchunk(L, nx, ny, nz, 304, 8, hi);
                        const int lo = nz < 32 ? nz : 32;
                        if (z < lo || z > nz || z > hi) ++bad;
                    }
    printf("%ld %d %d %d %d %d\n", bad, fdk::wave_zchunk(shapes[0], 512, 512, 512, 304, 8),
           fdk::wave_zchunk(shapes[1], 512, 512, 512, 456, 16), fdk::wave_zchunk(shapes[0], 1, 1, 1, 304, 8),
           fdk::wave_zchunk(shapes[0], 320, 320, 320, 304, 8),
           fdk::wave_zchunk(shapes[1], 512, 512, 512, 304, 16, 64));
    return 0;
}
"""


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


def test_wave_zchunk_ends_and_stays_in_bounds(tmp_path):
    inc = _cuda_include()
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")) or not shutil.which("g++"):
        pytest.skip("no CUDA headers or host compiler")
    src = tmp_path / "wz.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "wz"
    b = subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1410_1387_gb300", "csrc"),
                        "-I", inc, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0
    bad, r4, r8, one, c320, vti = map(int, r.stdout.split())
    assert bad == 0
    assert r4 == 74 and r8 == 74          # 7 chunks: 1792 CTAs, 5.9 waves of 304 or 3.9 of 456
    assert one == 1
    assert c320 == 54                     # 6 chunks of 5 x 20 tiles: 600 CTAs, two waves of 304
    assert vti == 64                      # 8 chunks: 2048 CTAs, 6.7 waves of 304


POLICY = r"""
#include "launch_policy.h"
#include <cstdio>
namespace fdk {
// the sweep's own default, as iso_sweep.cu gives it (32 x 32 tiles)
Launch iso_default_launch(int R, int nx, int ny, int nz)
{
    Launch L{32, 32, 0, R == 4 ? 3 : 2};
    L.zchunk = wave_zchunk(L, nx, ny, nz, 456, 2 * R);
    return L;
}
}
int main()
{
    const int cubes[] = {96, 200, 224, 240, 256, 320, 512};
    for (int n : cubes) {
        const fdk::Launch L = fdk::iso_grid_launch(4, n, n, n);
        printf("%d %d %d %d %d\n", n, L.tx, L.ty, L.zchunk, L.lookahead);
    }
    const fdk::Launch L8 = fdk::iso_grid_launch(8, 96, 96, 96);
    printf("8 %d %d %d %d\n", L8.tx, L8.ty, L8.zchunk, L8.lookahead);
    return 0;
}
"""


def test_radius4_grid_launch_policy(tmp_path):
    """The radius-4 default: the two-row 32 x 32 form when the grid's 32 x 32
    tiles times ceil(nz / 32) reach the GPU's CTA slots (152 SMs x 3; the SM
    count falls back to 152 without a GPU), else the one-row 64 x 16 form at
    lookahead 3 with a z chunk in range; radius 8 keeps its own default."""
    inc = _cuda_include()
    lib = os.path.join(os.path.dirname(inc), "lib64")
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")) or not shutil.which("g++") \
            or not os.path.exists(os.path.join(lib, "libcudart.so")):
        pytest.skip("no CUDA headers, runtime or host compiler")
    src = tmp_path / "pol.cpp"
    src.write_text(POLICY)
    exe = tmp_path / "pol"
    b = subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1410_1387_gb300", "csrc"),
                        "-I", inc, str(src), "-o", str(exe), "-L", lib, "-lcudart", "-Wl,-rpath," + lib],
                       capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr
    rows = [list(map(int, l.split())) for l in r.stdout.split("\n") if l.strip()]
    got = {row[0]: tuple(row[1:]) for row in rows[:-1]}
    for n in (96, 200, 224):                   # 27, 343, 343 CTAs at most: below 456 slots
        tx, ty, zc, la = got[n]
        assert (tx, ty, la) == (64, 16, 3) and min(32, n) <= zc <= min(96, n)
    for n in (240, 256, 320, 512):             # 512, 512, 1000, 4096: the two-row form
        assert got[n][:2] == (32, 32) and got[n][3] == 3
    assert got[512][2] == 74
    assert rows[-1][1:3] == [32, 32] and rows[-1][4] == 2
