"""Multi-GPU by replicas: shots are independent, so N processes (one per GPU)
split a survey between them and share nothing but the timing.

``deal`` assigns shots to ranks (largest first, each to the least-loaded rank;
every rank computes the same assignment); ``max_over_ranks`` reduces a
duration to its maximum (the job takes as long as its slowest rank).  Both
work on the gloo (CPU) and nccl (GPU) backends.
"""
from __future__ import annotations


def deal(costs, world: int):
    """Indices of the items each of `world` ranks runs: greedy longest-first
    assignment by cost (deterministic: ties broken by index)."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        out[r].append(i)
        loads[r] += costs[i]
    return [sorted(x) for x in out]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over the ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
