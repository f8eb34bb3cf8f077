"""Host-side sharding over ranks (one GPU per rank).

Replica batches: replicas are independent lattices, so a batch splits over
ranks with no exchange during stepping: rank k steps a contiguous range of
replicas and passes the index of its first replica as ``first_replica``, which
keeps every replica on the random stream it has in the unsplit batch.  Only
results are combined afterwards: int64 sums of the totals, and the ensemble
statistics (exact int64 sums all-reduced, FP32 running moments merged with
Chan et al.'s pairwise update).

One large lattice: it splits into contiguous blocks (``blocks``), each a
handle created with ``node_offset`` = its first node; the evolution equation
(Sec. III) moves one population per link and step, so after every step each
block sends one value across each of its two cuts and receives one
(``exchange_halo``).  Random numbers are keyed by the global node index, so
the blocks reproduce the undecomposed lattice bit for bit.
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


def blocks(L: int, world: int, align: int = 8) -> list[tuple[int, int]]:
    """Contiguous node ranges [begin, end) of one periodic lattice of L nodes,
    one per rank, as equal as possible, every begin a multiple of `align` (the
    slice sampler draws the top bits of eight consecutive nodes' uniforms from
    one Philox block, so its blocks start on multiples of 8).  Needs
    L >= world * align."""
    if world < 1 or align < 1:
        raise ValueError("world and align must be >= 1")
    if L < world * align:
        raise ValueError("too few nodes for that many blocks")
    cuts = [0] + [((k * L) // world) // align * align for k in range(1, world)] + [L]
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def exchange_halo(out, group=None):
    """One step's edge exchange of a block (see mclg_halo_get / mclg_halo_put):
    out[0] (the v = -1 value leaving the first node) goes to the left neighbour,
    out[1] (the v = +1 value leaving the last node) to the right neighbour; the
    result is in = (the left neighbour's out[1], the right neighbour's out[0]).
    With one rank the block is the whole periodic lattice: in = (out[1], out[0]).

    `out` is a tensor of two 16-bit values (host memory for gloo, device memory
    for NCCL); point-to-point messages only, posted in the same order on every
    rank (leftward send, rightward send, then the receives that match them), so
    that two ranks, each the other's left and right neighbour, pair them up."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        return torch.stack([out[1], out[0]])
    rank = dist.get_rank(group)
    left, right = (rank - 1) % world, (rank + 1) % world
    to_left, to_right = out[0:1].clone(), out[1:2].clone()
    from_right, from_left = torch.empty_like(to_left), torch.empty_like(to_right)
    reqs = [dist.isend(to_left, left, group, tag=1), dist.isend(to_right, right, group, tag=2),
            dist.irecv(from_right, right, group, tag=1), dist.irecv(from_left, left, group, tag=2)]
    for r in reqs:
        r.wait()
    return torch.cat([from_left, from_right])


_PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def merge_stats(st: dict, group=None) -> dict:
    """Pool the per-position statistics (mclg_stats_read) of replica shards.

    The exact int64 sums s1, s2, snb and the sample counts add up over the ranks
    (all-reduce).  The FP32 (co)variances are merged in rank order with the
    pairwise update of Chan, Golub and LeVeque,
        n = n_a + n_b,  d = mean_b - mean_a,
        M2_ij = M2a_ij + M2b_ij + d_i d_j n_a n_b / n,
    in FP32 like the library's running moments (mean_k = s1_k / n_k,
    M2_k = cov32_k n_k); cov64 is recomputed in FP64 from the pooled exact sums
    (Eqs. poisson, corr).  Every rank returns the same result."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    s1 = np.asarray(st["s1"], dtype=np.int64)
    s2 = np.asarray(st["s2"], dtype=np.int64)
    snb = np.asarray(st["snb"], dtype=np.int64)
    cnt = int(st["count"])
    cov32 = np.asarray(st["cov32"], dtype=np.float32)
    Lc = s1.shape[0]
    mean32 = (s1.astype(np.float32) / np.float32(max(cnt, 1))).astype(np.float32)
    m2 = (cov32 * np.float32(cnt)).astype(np.float32)
    if world > 1:
        ints = torch.from_numpy(np.concatenate([s1.ravel(), s2.ravel(), snb.ravel(),
                                                np.array([cnt], dtype=np.int64)]))
        dist.all_reduce(ints, op=dist.ReduceOp.SUM, group=group)
        ints = ints.numpy()
        packed = torch.from_numpy(np.concatenate([mean32.ravel(), m2.ravel(),
                                                  np.array([cnt], dtype=np.float64)
                                                  .view(np.float32)]).astype(np.float32))
        parts = [torch.empty_like(packed) for _ in range(world)]
        dist.all_gather(parts, packed, group=group)
        parts = [p.numpy() for p in parts]
    else:
        ints = np.concatenate([s1.ravel(), s2.ravel(), snb.ravel(), np.array([cnt])])
        parts = [np.concatenate([mean32.ravel(), m2.ravel(),
                                 np.array([cnt], dtype=np.float64).view(np.float32)])]
    n3, n6, n9 = 3 * Lc, 6 * Lc, 9 * Lc
    out = {"s1": ints[:n3].reshape(Lc, 3), "s2": ints[n3:n3 + n6].reshape(Lc, 6),
           "snb": ints[n3 + n6:n3 + n6 + n9].reshape(Lc, 9), "count": int(ints[-1])}
    # Chan et al.'s merge in rank order, FP32
    na = 0
    mean = np.zeros((Lc, 3), dtype=np.float32)
    M2 = np.zeros((Lc, 6), dtype=np.float32)
    for p in parts:
        mb = p[:n3].reshape(Lc, 3)
        m2b = p[n3:n3 + n6].reshape(Lc, 6)
        nb = int(p[n3 + n6:].view(np.float64)[0])
        if nb == 0:
            continue
        n = na + nb
        d = (mb - mean).astype(np.float32)
        w = np.float32(na * nb / n)
        for k, (i, j) in enumerate(_PAIRS):
            M2[:, k] = M2[:, k] + m2b[:, k] + d[:, i] * d[:, j] * w
        mean = (mean + d * np.float32(nb / n)).astype(np.float32)
        na = n
    out["cov32"] = (M2 / np.float32(max(na, 1))).astype(np.float32)
    cov64 = np.zeros((Lc, 6), dtype=np.float64)
    if out["count"]:
        M = out["count"]
        for k, (i, j) in enumerate(_PAIRS):
            for x in range(Lc):
                num = M * int(out["s2"][x, k]) - int(out["s1"][x, i]) * int(out["s1"][x, j])
                cov64[x, k] = num / (M * M)
    out["cov64"] = cov64
    return out
