"""bench.py's reference arm (the FP64 oracle timed on the host cores) keeps
the JSON contract on CPU: one line with the metric, unit, value, the oracle's
core count and sample, and an end-to-end entry with no host-device bytes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "24",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "grid-point updates/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["grid"] == [24, 24, 24] and d["config"]["workload"] == "iso512_r4_layered"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0 and e["value"] == d["value"]


def test_l2_note_tracks_the_input_size():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.l2_note(3 * 4 * 512 ** 3).startswith("no flush")
    assert "may stay" in bench.l2_note(3 * 4 * 64 ** 3)


def test_kernel_hash_ignores_comments_and_layout():
    """The recorded DRAM traffic stays valid across comment-only edits of the
    kernel source, and no longer once the code changes."""
    import bench
    a = "int f(int x) { // doubles\n  return 2 * x; /* the\n factor */ }\n"
    b = "int f(int x) {\n\n    return 2 * x;   }"
    c = "int f(int x) { return 3 * x; }"
    assert bench._code_only(a) == bench._code_only(b) != bench._code_only(c)


def test_cpu_leg_samples_like_the_reference_arm():
    """The bench line's cpu_baseline times the oracle as the reference arm does:
    the same step and warm-up counts (capped at 20 and 5) on the same slab rule."""
    sys.path.insert(0, ROOT)
    import bench
    shot = bench.make_shot("iso512_r4", 24, seed=1)
    leg = bench.cpu_leg(shot, 2, 1)
    assert leg["kind"] == "oracle" and leg["cores"] >= 1 and leg["value"] > 0
    assert "2 steps after 1 warm-up steps of a [24, 24, 24] slab" in leg["sample"]
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "24",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    ref = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    assert "2 steps after 1 warm-up steps of a [24, 24, 24] slab" in ref["cpu_baseline"]["sample"]
    long = bench.cpu_leg(shot, 2000, 20)
    assert "20 steps after 5 warm-up steps" in long["sample"]
