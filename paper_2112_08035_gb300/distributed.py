"""Splitting one job across ranks (one process per GPU).

Packets are independent and every random number is keyed by (seed, packet
id, event), so a job over ids [0, N) splits into contiguous id blocks, one
per rank, with no communication while packets propagate.  The only exchange
is at the end: an element-wise sum of the int64 fixed-point tallies (fluence
grid and totals).  Integer addition is exact and associative, so the reduced
result is bit-identical to a single-GPU run of the whole job, whatever the
number of ranks or the reduction order.
"""
from __future__ import annotations


def shard_range(rank: int, world: int, n: int, base: int = 0):
    """[begin, end) of packet ids for `rank` of `world` (balanced, contiguous)."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad rank / world / n")
    q, r = divmod(n, world)
    begin = base + rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def allreduce_tallies(fluence, totals, group=None):
    """Sum int64 fluence and totals tensors over all ranks in place (the
    exchange step; works with the gloo and nccl backends)."""
    import torch
    import torch.distributed as dist
    for t in (fluence, totals):
        if t is None:
            continue
        if t.dtype != torch.int64:
            raise TypeError("tallies are int64 fixed point")
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return fluence, totals
