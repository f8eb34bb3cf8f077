"""Host-side sharding of a replica batch over ranks (one GPU per rank).

Replicas are independent lattices, so a batch splits over ranks with no
exchange during stepping: rank k steps a contiguous range of replicas and
passes the index of its first replica as ``first_replica``, which keeps every
replica on the random stream it has in the unsplit batch.  Only results are
combined afterwards (int64 sums of the totals).
"""
from __future__ import annotations

import numpy as np


def partition(L, world: int) -> list[tuple[int, int]]:
    """Contiguous replica ranges [begin, end), one per rank, balanced by node count.

    Rank k takes the replicas whose node prefix sum falls into the k-th of
    `world` equal slices of the total; ranges may be empty when there are
    fewer replicas than ranks."""
    L = np.asarray(L, dtype=np.int64).reshape(-1)
    if world < 1:
        raise ValueError("world must be >= 1")
    starts = np.concatenate([[0], np.cumsum(L)[:-1]]) if L.size else np.zeros(0, np.int64)
    total = int(L.sum())
    # replica r belongs to the rank whose slice holds its first node
    owner = (starts * world) // max(total, 1)
    out = []
    last = 0
    for k in range(world):
        idx = np.nonzero(owner == k)[0]
        if idx.size:
            out.append((int(idx[0]), int(idx[-1]) + 1))
            last = int(idx[-1]) + 1
        else:
            out.append((last, last))  # empty range where the previous one ended
    return out


def local_workload(wl, rank: int, world: int):
    """The part of a Workload that rank `rank` steps, and its first replica index."""
    from dataclasses import replace
    b, e = partition(wl.L, world)[rank]
    off = np.concatenate([[0], np.cumsum(wl.L.astype(np.int64))])
    sl = slice(int(off[b]), int(off[e]))
    return replace(wl, L=wl.L[b:e].copy(), rho=wl.rho[sl], u=wl.u[sl]), b


def allreduce_sum_int64(values, group=None) -> np.ndarray:
    """Exact sum over ranks of int64 values (e.g. the totals of mclg_moments)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.asarray(values, dtype=np.int64)).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()
