"""The multi-rank (replica) path on CPU: two gloo ranks deal a survey between
them identically, cover every shot exactly once, and reduce their timings to
the maximum and the sum, as bench.py does on GPUs."""
import os
import socket

import pytest

from paper_1410_1387_gb300 import dist as fdist


def test_deal_covers_every_shot_once_and_balances():
    costs = [float(n ** 3 * s) for n, s in zip(range(96, 320, 7), range(300, 1500, 37))]
    for world in (1, 2, 3, 8):
        parts = fdist.deal(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, costs, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = fdist.deal(costs, world)[rank]
    elapsed = 1.0 + rank            # stand-in for a rank's measured seconds
    mx = fdist.max_over_ranks(elapsed)
    tot = fdist.sum_over_ranks(sum(costs[i] for i in mine))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mine, mx, tot))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    costs = [5.0, 3.0, 8.0, 1.0, 4.0, 4.0, 2.0]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, mx0, t0), (r1, m1, mx1, t1) = out
    assert sorted(m0 + m1) == list(range(len(costs))) and not set(m0) & set(m1)
    assert mx0 == mx1 == 2.0
    assert t0 == t1 == pytest.approx(sum(costs))
