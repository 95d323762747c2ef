"""Multi-process helpers (one process per GPU).

Independent shots are replicas: N processes split a survey between them and
share nothing but the timing.  ``deal`` assigns shots to ranks (largest first,
each to the least-loaded rank; every rank computes the same assignment);
``max_over_ranks`` reduces a duration to its maximum (the job takes as long as
its slowest rank).  One shot split into z slabs over ranks exchanges ghost
planes with its neighbours every step: ``halo_exchange_start`` posts the
exchange so that the slab's interior can be updated while it is in flight.
All work on the gloo (CPU tensors, or CUDA tensors staged through host memory)
and nccl (GPU) backends.
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


class _Exchange:
    """A posted ghost-plane exchange; wait() completes it."""

    def __init__(self, finish):
        self._finish = finish

    def wait(self) -> None:
        if self._finish is not None:
            self._finish()
            self._finish = None


def halo_exchange_start(buf, halo: int, lower, upper, group=None) -> _Exchange:
    """Post the refresh of the ghost planes of a z slab from its neighbouring
    ranks; the returned handle's wait() completes it.

    `buf` is the slab's stored planes (a contiguous tensor, planes first): it
    owns planes [halo, n - halo) when it has both neighbours, and its first
    (last) `halo` planes are ghosts of rank `lower`'s (`upper`'s) last (first)
    owned planes.  `lower` / `upper` are ranks or None at the ends of the
    column.  This slab's owned planes next to each cut are sent and the ghost
    planes received in place; every pair of neighbours must take part.

    Work the caller enqueues between this call and wait() overlaps the
    exchange: on nccl (CUDA tensors) the sends and receives run on the
    backend's stream after everything already queued on the current stream,
    and wait() makes the current stream wait for them; on gloo with a CUDA
    buffer the boundary planes are copied to pinned host memory on the current
    stream now, and wait() exchanges them on the host and copies the received
    planes back on that stream; on gloo with a CPU buffer wait() does it all."""
    import torch
    import torch.distributed as dist
    n = buf.shape[0]
    pairs = []          # (peer, slice sent, slice received)
    if lower is not None:
        pairs.append((lower, slice(halo, 2 * halo), slice(0, halo)))
    if upper is not None:
        pairs.append((upper, slice(n - 2 * halo, n - halo), slice(n - halo, n)))
    if not pairs:
        return _Exchange(None)
    staged = buf.is_cuda and dist.get_backend(group) != "nccl"
    if not staged:
        ops = []
        for peer, snd, rcv in pairs:
            ops.append(dist.P2POp(dist.isend, buf[snd].contiguous(), peer, group))
            ops.append(dist.P2POp(dist.irecv, buf[rcv], peer, group))
        if buf.is_cuda:
            works = dist.batch_isend_irecv(ops)
            return _Exchange(lambda: [w.wait() for w in works])
        return _Exchange(lambda: [w.wait() for w in dist.batch_isend_irecv(ops)])
    # gloo and a device buffer: through pinned host memory
    host_send = []
    for peer, snd, rcv in pairs:
        h = torch.empty(buf[snd].shape, dtype=buf.dtype, pin_memory=True)
        h.copy_(buf[snd], non_blocking=True)
        host_send.append(h)
    ready = torch.cuda.Event()
    ready.record()

    def finish():
        ready.synchronize()
        host_recv = [torch.empty(buf[rcv].shape, dtype=buf.dtype, pin_memory=True) for _, _, rcv in pairs]
        ops = []
        for (peer, _, _), hs, hr in zip(pairs, host_send, host_recv):
            ops.append(dist.P2POp(dist.isend, hs, peer, group))
            ops.append(dist.P2POp(dist.irecv, hr, peer, group))
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        for (_, _, rcv), hr in zip(pairs, host_recv):
            buf[rcv].copy_(hr, non_blocking=True)
    return _Exchange(finish)


def halo_exchange(buf, halo: int, lower, upper, group=None) -> None:
    """halo_exchange_start(...).wait(): the ghost planes of `buf` refreshed from
    the neighbouring ranks (gloo or nccl; CPU or CUDA tensors)."""
    halo_exchange_start(buf, halo, lower, upper, group).wait()
