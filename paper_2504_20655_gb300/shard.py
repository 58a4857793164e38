"""Splitting the routing path across ranks, one process per GPU (host logic only).

Orders are independent, so a batch splits into contiguous slices of orders, one per
rank; every rank routes its slice on its own GPU with no exchange on the data path, and
the per-order results come together on rank 0 only when a caller asks for them
(`gather_order_results`).  At scale the sources split the same way: every rank produces
the rows of its slice of the sources segment by segment and consumes them into its rows
of the pick submatrix, and one all-gather assembles the full submatrix on every rank
(`all_gather_rows`), the single exchange step of the path.

Nothing here touches a GPU itself: the collectives run on whatever backend the process
group was created with (NCCL with device tensors, gloo with host tensors).
"""
from __future__ import annotations

import numpy as np

from .synth import Orders


def even_slice(n: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous share of n units: the first n % world ranks get
    one unit more than the others."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad split")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_orders(orders: Orders, world: int, rank: int) -> tuple[Orders, int, int]:
    """Rank's contiguous slice of the batch as a batch of its own (offsets from 0), with
    the [lo, hi) range of order indices it covers."""
    lo, hi = even_slice(orders.n, world, rank)
    return orders.subset(np.arange(lo, hi)), lo, hi


def _all_gather_padded(t, world):
    """All-gather of a 1-D or 2-D tensor whose leading size differs across ranks: pad to
    the largest, gather, trim.  Returns the list of every rank's tensor."""
    import torch
    import torch.distributed as dist
    n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(x.item()) for x in sizes]
    big = max(sizes)
    pad = torch.zeros((big,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[:t.shape[0]] = t
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return [p[:s] for p, s in zip(parts, sizes)]


def gather_order_results(cost, perm, status, world: int, rank: int):
    """The results of every rank's slice (cost[n_r], perm[picks_r], status[n_r] tensors,
    in slice order) put together in batch order: (cost, perm, status) tensors on every
    rank, equal to routing the whole batch at once."""
    import torch
    if world == 1:
        return cost, perm, status
    cs = _all_gather_padded(cost, world)
    ps = _all_gather_padded(perm, world)
    ss = _all_gather_padded(status, world)
    return torch.cat(cs), torch.cat(ps), torch.cat(ss)


def all_gather_rows(rows, world: int):
    """Rows of a matrix split by contiguous row slices across ranks (rank r holds rows
    even_slice(n, world, r)): the whole matrix on every rank."""
    import torch
    if world == 1:
        return rows
    return torch.cat(_all_gather_padded(rows, world))
