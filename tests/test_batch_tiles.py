"""Host-side consistency of the batch autotuner (no GPU): every tile it may pick
is one of the (radius, tile, lookahead) combinations compiled into libfd.so
(the FD_ISO_CONFIGS list of the isotropic sweep), and the survey-wide GPU test
covers exactly the radius-4 tiles the autotuner offers."""
import os
import re

from paper_1410_1387_gb300 import batch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _built_configs():
    src = open(os.path.join(ROOT, "paper_1410_1387_gb300", "csrc", "iso_sweep.cu")).read()
    block = src[src.index("#define FD_ISO_CONFIGS"):]
    block = block[:block.index("\n\n")]
    return {tuple(int(v) for v in m) for m in re.findall(r"X\((\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", block)}


def test_autotuner_tiles_are_built():
    built = _built_configs()
    assert built, "no configurations found"
    for r, tiles in batch.TILES.items():
        for tx, ty, la in tiles:
            assert (r, tx, ty, la) in built, (r, tx, ty, la)


def test_survey_test_covers_every_radius4_tile():
    src = open(os.path.join(ROOT, "tests", "test_gpu_batch.py")).read()
    line = next(l for l in src.splitlines() if l.startswith("R4_TILES = "))
    tiles = [tuple(int(v) for v in m) for m in re.findall(r"\((\d+),\s*(\d+),\s*(\d+)\)", line)]
    assert sorted(tiles) == sorted(batch.TILES[4])
