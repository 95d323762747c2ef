"""Multi-process helpers (one process per GPU).

Independent shots are replicas: N processes split a survey between them and
share nothing but the timing.  ``deal`` assigns shots to ranks (largest first,
each to the least-loaded rank; every rank computes the same assignment);
``max_over_ranks`` reduces a duration to its maximum (the job takes as long as
its slowest rank).  One shot split into z slabs over ranks exchanges ghost
planes with its neighbours after every step: ``halo_exchange``.  All work on
the gloo (CPU) and nccl (GPU) backends.
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


def halo_exchange(buf, halo: int, lower, upper, group=None) -> None:
    """Refresh the ghost planes of a z slab from its neighbouring ranks.

    `buf` is the slab's stored planes (a contiguous tensor, planes first): it
    owns planes [halo, n - halo) when it has both neighbours, and its first
    (last) `halo` planes are ghosts of rank `lower`'s (`upper`'s) last (first)
    owned planes.  `lower` / `upper` are ranks or None at the ends of the
    column.  Sends this slab's owned planes next to each cut and receives the
    ghost planes in place; every pair of neighbours must call it together.
    Works on gloo (CPU tensors) and nccl (CUDA tensors) alike."""
    import torch.distributed as dist
    n = buf.shape[0]
    ops = []
    if lower is not None:
        ops.append(dist.P2POp(dist.isend, buf[halo:2 * halo].contiguous(), lower, group))
        ops.append(dist.P2POp(dist.irecv, buf[0:halo], lower, group))
    if upper is not None:
        ops.append(dist.P2POp(dist.isend, buf[n - 2 * halo:n - halo].contiguous(), upper, group))
        ops.append(dist.P2POp(dist.irecv, buf[n - halo:n], upper, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
