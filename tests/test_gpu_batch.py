"""Batched shots (fd_batch_*): every member's traces and final wavefields are
bit-identical to running that shot alone with fd_run (same kernel body, same
per-point summation order), for mixed sizes, radii and step counts, with and
without CUDA graphs, and when members join or leave between runs."""
import numpy as np
import pytest

from paper_1410_1387_gb300 import synth
from tests.helpers import max_rel, oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_1387_gb300 import batch, fd
    return fd, batch


def small_survey(radii=(4, 8), count=6, seed=7):
    shots = synth.survey_shots(count, seed=seed, n_lo=40, n_hi=90, steps_lo=20, steps_hi=60, radii=radii)
    for s in shots:   # smaller damping layer and source depth for the small grids
        s.nb = 6
        s.src = (s.nx // 2, s.ny // 2, 12)
        s.receivers = synth.receiver_plane(s.nx, s.ny, 6, stride=2, x0=1)
    return shots


def test_batch_bitwise_equals_per_shot(fdm):
    fd, batch = fdm
    shots = small_survey()
    tr_b, _, gb, _ = batch.run_batched(shots, keep_grids=True)
    tr_s, _, gs, _ = batch.run_per_shot(shots, keep_grids=True)
    for a, b, x, y in zip(tr_b, tr_s, gb, gs):
        np.testing.assert_array_equal(a, b)
        for u, v in zip(x.state(), y.state()):
            np.testing.assert_array_equal(u, v)
        assert x.time_index == y.time_index
    for g in gb + gs:
        g.close()


def test_batch_graph_and_tiles(fdm):
    fd, batch = fdm
    shots = small_survey(radii=(4,), count=4, seed=11)
    tr0 = batch.run_per_shot(shots)[0]
    tr1 = batch.run_batched(shots, graph_steps=4)[0]
    tr2 = batch.run_batched(shots, graph_steps=3, launch={4: (64, 8, 20, 3)})[0]
    tr3 = batch.run_batched(shots, launch={4: (128, 8, 0, 3)})[0]
    assert batch.traces_equal(tr0, tr1) and batch.traces_equal(tr0, tr2) and batch.traces_equal(tr0, tr3)
    # both radii: the radius-8 members run on a forked stream, inside graphs too
    mixed = small_survey(radii=(4, 8), count=5, seed=14)
    assert len({s.r_xy for s in mixed}) == 2
    tm0 = batch.run_per_shot(mixed)[0]
    tm1 = batch.run_batched(mixed, graph_steps=4)[0]
    assert batch.traces_equal(tm0, tm1)


def test_batch_against_oracle(fdm, O):
    fd, batch = fdm
    shots = small_survey(radii=(8,), count=2, seed=3)
    tr, _, grids, _ = batch.run_batched(shots, keep_grids=True)
    for s, t, g in zip(shots, tr, grids):
        u, _ = g.state()
        ur, _, trr = oracle_problem(O, s).iso_run(s.v, s.nsteps)
        assert max_rel(u, ur) <= 1e-4 and max_rel(t, trr) <= 1e-4
        g.close()


def test_members_join_and_leave(fdm):
    fd, batch = fdm
    a, b_, c = small_survey(radii=(4,), count=3, seed=5)
    solo = [batch.run_per_shot([s])[0][0] for s in (a, b_, c)]
    ga, gb, gc = (fd.grid_from_shot(s) for s in (a, b_, c))
    bt = batch.Batch()
    bt.add(ga, a.nsteps)
    assert bt.run(7) == 7
    bt.add(gb, b_.nsteps)            # joins while a is mid-run
    bt.run(5)
    bt.add(gc, c.nsteps)
    while bt.run(1000):
        if bt.steps_left(ga) == 0 and ga.h in bt.members:
            bt.remove(ga)
    for g, s, want in zip((ga, gb, gc), (a, b_, c), solo):
        assert g.time_index == s.nsteps
        np.testing.assert_array_equal(g.traces(), want)
        g.close()
    bt.close()


def test_batch_errors(fdm):
    fd, batch = fdm
    bt = batch.Batch()
    v = synth.vti_shot(24, nsteps=2)
    gv = fd.grid_from_shot(v)
    with pytest.raises(fd.FdError) as e:
        bt.add(gv, 2)
    assert e.value.code == fd.FD_ERR_UNSUPPORTED
    s = small_survey(radii=(4,), count=1)[0]
    s.receivers = np.array([[1, 2, 3], [5, 1, 7]], np.int32)       # not a lattice
    g = fd.grid_from_shot(s)
    with pytest.raises(fd.FdError) as e:
        bt.add(g, 3)
    assert e.value.code == fd.FD_ERR_UNSUPPORTED
    with pytest.raises(fd.FdError) as e:
        bt.remove(g)
    assert e.value.code == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FdError) as e:
        bt.set_launch(4, 48, 16, 64, 3)
    assert e.value.code == fd.FD_ERR_UNSUPPORTED
    assert bt.run(5) == 0            # no members
    for x in (gv, g):
        x.close()
    bt.close()


def test_autotuner_caches_a_built_choice(fdm, tmp_path):
    fd, batch = fdm
    s = small_survey(radii=(4,), count=1)[0]
    t = batch.Autotuner(path=str(tmp_path / "tune.json"))
    c = t.single(s, steps=4, candidates=[(64, 16, 16, 3), (128, 8, 16, 3), (64, 8, 32, 3)])
    assert c in [(64, 16, 16, 3), (128, 8, 16, 3), (64, 8, 32, 3)]
    t2 = batch.Autotuner(path=str(tmp_path / "tune.json"))
    assert t2.single(s) == c                      # served from the cache
    shots = small_survey(radii=(4,), count=3)
    choice = t.batch(shots, steps=2, zchunks=(16, 32))
    tx, ty, zc, la = choice[4]
    g = fd.grid_from_shot(shots[0])
    g.set_launch(tx, ty, zc, la)                 # a built configuration
    g.close()


# ---------------------------------------------------------------------------
# The 64-shot survey (cubic 96^3..320^3, 300..1500 steps, radius 4) in one batch,
# for every radius-4 tile built into the library, twice each: traces bit for bit
# equal to the per-shot loop's.  Traces stay on the device (10.6 GB per pass).

R4_TILES = [(64, 16, 3), (64, 16, 2), (64, 16, 4), (128, 8, 3), (64, 8, 3), (32, 16, 3), (32, 32, 3), (32, 32, 2)]


@pytest.fixture(scope="module")
def survey(fdm):
    import torch
    fd, batch = fdm
    shots = synth.survey_shots(64, seed=2024)
    ref = []
    for s in shots:                           # the per-shot loop, default launch
        g = fd.grid_from_shot(s)
        g.run(s.nsteps)
        g.sync()
        ref.append(g.trace[:s.nsteps].clone())
        g.close()
    torch.cuda.synchronize()
    return shots, ref


def _survey_batched(fd, batch, shots, launch, graph_steps):
    import torch
    grids = [fd.grid_from_shot(s) for s in shots]
    b = batch.Batch()
    b.set_launch(4, *launch)
    b.set_graph(graph_steps)
    for g, s in zip(grids, shots):
        b.add(g, s.nsteps)
    live = list(grids)
    while live:
        b.run(max(64, min(b.steps_left(g) for g in live)))
        for g in [g for g in live if b.steps_left(g) == 0]:
            b.remove(g)
            live.remove(g)
    torch.cuda.synchronize()
    for g in grids:
        g.sync()
    out = [g.trace[:s.nsteps].clone() for g, s in zip(grids, shots)]
    b.close()
    for g in grids:
        g.close()
    return out


@pytest.mark.parametrize("tile", R4_TILES)
def test_survey_batch_bitwise_every_tile(fdm, survey, tile):
    import torch
    fd, batch = fdm
    shots, ref = survey
    tx, ty, la = tile
    for graph_steps, zchunk in ((16, 64), (0, 0)):
        out = _survey_batched(fd, batch, shots, (tx, ty, zchunk, la), graph_steps)
        bad = [i for i, (a, r) in enumerate(zip(out, ref)) if not torch.equal(a, r)]
        assert not bad, f"tile {tile}, z chunk {zchunk}, graphs {graph_steps}: shots {bad} differ"
        del out


def test_radius4_batch_members_against_oracle(fdm, O):
    """Radius-4 members of a mixed batch, element by element against the FP64
    oracle (wavefield and traces), in the 160-thread tile the batch shares
    with the autotuner's other candidates."""
    fd, batch = fdm
    shots = small_survey(radii=(4,), count=3, seed=19)
    for launch in ({4: (32, 16, 0, 3)}, {4: (64, 16, 24, 3)}):
        tr, _, grids, _ = batch.run_batched(shots, keep_grids=True, graph_steps=5, launch=launch)
        for s, t, g in zip(shots, tr, grids):
            u, _ = g.state()
            ur, _, trr = oracle_problem(O, s).iso_run(s.v, s.nsteps)
            assert np.abs(ur).max() > 0 and np.abs(trr).max() > 0
            assert max_rel(u, ur) <= 1e-4 and max_rel(t, trr) <= 1e-4
            g.close()
