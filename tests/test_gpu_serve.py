"""Continuous-batching server: requests admitted by HBM budget while others
run; each request's traces are bit-identical alone (FIFO loop, one shot at a
time) and in the mix."""
import numpy as np
import pytest

from paper_1410_1387_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_1387_gb300 import serve
    return serve


def small_stream(count=8, rate=200.0, seed=5):
    return synth.poisson_requests(count, rate=rate, seed=seed, n_lo=40, n_hi=80, steps_lo=30, steps_hi=90,
                                  radii=(4, 8))


def test_same_alone_and_in_the_mix(srv):
    reqs = small_stream()
    # a budget that holds about three of these shots at once, so requests queue
    sizes = sorted(srv.shot_bytes(synth.request_shot(r)) for r in reqs)
    budget = sum(sizes[-3:])
    server = srv.ShotServer(budget, steps_per_iter=7, keep_traces=True)
    mixed = server.serve(reqs, realtime=True)
    alone = srv.fifo_loop(reqs, realtime=False, keep_traces=True)
    assert [r.rid for r in mixed] == [r.rid for r in alone] == sorted(r.rid for r in reqs)
    for m, a in zip(mixed, alone):
        np.testing.assert_array_equal(m.traces, a.traces)
        assert np.abs(a.traces).max() > 0
    assert 2 <= server.max_resident < len(reqs)
    s = srv.summary(mixed)
    assert s["shots"] == len(reqs) and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_graphs_and_overlap_keep_results(srv):
    reqs = small_stream(count=5, seed=9)
    budget = 1 << 40
    a = srv.ShotServer(budget, steps_per_iter=16, graph_steps=8, keep_traces=True).serve(reqs, realtime=False)
    b = srv.fifo_loop(reqs, realtime=False, keep_traces=True)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x.traces, y.traces)


def test_request_above_budget_is_refused(srv):
    reqs = small_stream(count=1)
    with pytest.raises(ValueError):
        srv.ShotServer(1024, steps_per_iter=5).serve(reqs, realtime=False)


def test_served_requests_match_the_oracle(srv, O):
    """Served requests against the FP64 oracle, element by element: a stream of
    radius-4 and radius-8 requests runs through the server (a budget that keeps
    about three resident, so the two checked ones share the GPU with others),
    and the traces of one request of each radius are compared with the oracle's
    run of the same shot on the same model (drawn on the GPU, copied back)."""
    import torch
    from tests.helpers import max_rel, oracle_problem
    # grids of 40-56 points (damping layer n // 6, source at the centre) and
    # enough steps for the Ricker pulse (peak at t0 = 1/f, about 150 steps) to
    # cross to the receiver plane
    reqs = synth.poisson_requests(6, rate=200.0, seed=21, n_lo=40, n_hi=56, steps_lo=240, steps_hi=300,
                                  radii=(4, 8))
    assert {r.radius for r in reqs} == {4, 8}
    sizes = sorted(srv.shot_bytes(synth.request_shot(r)) for r in reqs)
    server = srv.ShotServer(sum(sizes[-3:]), steps_per_iter=9, keep_traces=True)
    served = {r.rid: r for r in server.serve(reqs, realtime=True)}
    assert server.max_resident >= 2
    for radius in (4, 8):
        req = next(r for r in reqs if r.radius == radius)
        shot = synth.request_shot(req)
        v = synth.layered_model_device(req.n, req.seed, torch.device("cuda", 0)).cpu().numpy()
        _, _, tr_ref = oracle_problem(O, shot).iso_run(v, shot.nsteps)
        tr = served[req.rid].traces
        assert tr.shape == tr_ref.shape and np.abs(tr_ref).max() > 0
        assert max_rel(tr, tr_ref) <= 1e-4
