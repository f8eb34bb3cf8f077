"""Sharding a replica batch over ranks (host logic, CPU): balanced contiguous
ranges, and a world-size-2 gloo run of the oracle on the two shards that
reproduces the unsplit batch bit for bit and its exact int64 totals."""
import os
import socket

import numpy as np
import pytest

from paper_1706_01094_gb300 import sharding, workloads


def test_partition_covers_and_balances():
    g = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        for _ in range(20):
            L = g.integers(1, 5000, g.integers(1, 40))
            parts = sharding.partition(L, world)
            assert len(parts) == world
            assert parts[0][0] == 0 and parts[-1][1] == len(L)
            for (b0, e0), (b1, e1) in zip(parts, parts[1:]):
                assert e0 == b1 and b0 <= e0
            if len(L) >= world:
                loads = [int(L[b:e].sum()) for b, e in parts]
                assert max(loads) <= L.sum() / world + L.max()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, L, n0, steps, out_dir):
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        b, e = sharding.partition(L, world)[rank]
        off = np.concatenate([[0], np.cumsum(L)])
        local = n0[:, off[b]:off[e]]
        n, err = oracle.step(L[b:e], 9, local, 0, steps, first_replica=b)
        assert err == 0
        _, _, tot = oracle.moments(L[b:e], n)
        total = sharding.allreduce_sum_int64(tot)
        np.save(os.path.join(out_dir, f"state_{rank}.npy"), n)
        np.save(os.path.join(out_dir, f"tot_{rank}.npy"), total)
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_shards_reproduce_unsplit_batch(tmp_path):
    torch = pytest.importorskip("torch")
    import oracle
    import torch.multiprocessing as mp
    oracle.build()
    L = np.array([64, 9, 300, 17, 128, 1, 77], dtype=np.int64)
    n0 = workloads.random_state(L, 20.0, seed=4)
    steps = 15
    mp.start_processes(_rank_main, args=(2, _free_port(), L, n0, steps, str(tmp_path)),
                       nprocs=2, join=True, start_method="spawn")
    whole, err = oracle.step(L, 9, n0, 0, steps)
    assert err == 0
    got = np.concatenate([np.load(tmp_path / "state_0.npy"), np.load(tmp_path / "state_1.npy")],
                         axis=1)
    assert np.array_equal(got, whole)
    _, _, tot = oracle.moments(L, whole)
    for r in (0, 1):
        assert np.array_equal(np.load(tmp_path / f"tot_{r}.npy"), tot)


def test_blocks_cover_the_lattice_on_aligned_starts():
    for L, world in ((1000, 2), (1001, 3), (64, 8), (2**24, 8), (64, 1), (17, 8)):
        align = 8 if L >= 8 * world else 2
        parts = sharding.blocks(L, world, align=align)
        assert parts[0][0] == 0 and parts[-1][1] == L and len(parts) == world
        for (b0, e0), (b1, e1) in zip(parts, parts[1:]):
            assert e0 == b1 and b0 < e0 and b1 % align == 0
        assert max(e - b for b, e in parts) <= L // world + align
    with pytest.raises(ValueError):
        sharding.blocks(5, 3)
    with pytest.raises(ValueError):
        sharding.blocks(60, 8)      # fewer than 8 nodes per block


def _halo_rank_main(rank, world, port, L, n0, steps, sampler, out_dir):
    import torch
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        b, e = sharding.blocks(L, world)[rank]
        blk = oracle.Block(n0[:, b:e], b, 13, sampler=sampler, n_max=90)
        for t in range(7, 7 + steps):
            out, err = blk.collide(t)
            assert err == 0
            inc = sharding.exchange_halo(torch.from_numpy(out.view(np.int16)))
            blk.stream(inc.numpy().view(np.uint16))
        np.save(os.path.join(out_dir, f"block_{rank}.npy"), blk.n)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("sampler", ["sequential", "slice"])
def test_two_rank_gloo_blocks_of_one_lattice_reproduce_it(tmp_path, sampler):
    """One periodic lattice split into two blocks on two gloo ranks, one value
    exchanged across each cut per step (point-to-point), equals the undecomposed
    oracle bit for bit (the random numbers are keyed by the global node index)."""
    pytest.importorskip("torch")
    import oracle
    import torch.multiprocessing as mp
    oracle.build()
    L = 1234
    n0 = workloads.random_state([L], 30.0, seed=8)
    steps = 12
    mp.start_processes(_halo_rank_main, args=(2, _free_port(), L, n0, steps, sampler,
                                              str(tmp_path)),
                       nprocs=2, join=True, start_method="spawn")
    if sampler == "slice":
        whole, err = oracle.slice_step([L], 13, n0, 7, steps, n_max=90)
    else:
        whole, err = oracle.step([L], 13, n0, 7, steps)
    assert err == 0
    got = np.concatenate([np.load(tmp_path / "block_0.npy"), np.load(tmp_path / "block_1.npy")],
                         axis=1)
    assert np.array_equal(got, whole)


def test_single_rank_exchange_closes_the_ring():
    torch = pytest.importorskip("torch")
    import oracle
    oracle.build()
    L = 300
    n0 = workloads.random_state([L], 25.0, seed=2)
    blk = oracle.Block(n0, 0, 5)
    for t in range(9):
        out, _ = blk.collide(t)
        blk.stream(sharding.exchange_halo(torch.from_numpy(out.view(np.int16))).numpy()
                   .view(np.uint16))
    whole, _ = oracle.step([L], 5, n0, 0, 9)
    assert np.array_equal(blk.n, whole)


def _local_stats(L, n0, first, R_local, steps, seed):
    """Exact sums of a replica shard (the oracle) and FP32 (co)variances derived
    from them, as a rank's mclg_stats_read would give them."""
    import oracle
    Lc = int(L[0])
    ref = oracle.Stats(Lc, R_local)
    n = n0
    for t in range(steps):
        n, err = oracle.step(L, seed, n, t, 1, first_replica=first)
        assert err == 0
        ref.accumulate(n)
    cnt = ref.count
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    cov = np.zeros((Lc, 6), dtype=np.float32)
    for k, (i, j) in enumerate(pairs):
        num = cnt * ref.s2[:, k].astype(np.float64) - ref.s1[:, i].astype(np.float64) * ref.s1[:, j]
        cov[:, k] = (num / (float(cnt) ** 2)).astype(np.float32)
    return {"s1": ref.s1, "s2": ref.s2, "snb": ref.snb, "count": cnt, "cov32": cov}


def _stats_rank_main(rank, world, port, L, n0, steps, out_dir):
    import pickle
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        b, e = sharding.partition(L, world)[rank]
        Lc = int(L[0])
        local = _local_stats(L[b:e], n0[:, b * Lc:e * Lc], b, e - b, steps, 3)
        merged = sharding.merge_stats(local)
        with open(os.path.join(out_dir, f"stats_{rank}.pkl"), "wb") as f:
            pickle.dump(merged, f)
    finally:
        dist.destroy_process_group()


def test_two_rank_statistics_merge(tmp_path):
    """Replica shards on two gloo ranks: the pooled int64 sums equal one rank's
    sums over all replicas bit for bit, and the FP32 (co)variances merged with
    Chan et al.'s update agree with the FP64 values of the pooled exact sums to
    1e-6 (relative for variances, of sqrt(var_i var_j) for covariances)."""
    pytest.importorskip("torch")
    import pickle
    import oracle
    import torch.multiprocessing as mp
    oracle.build()
    R, Lc, steps = 24, 16, 30
    L = np.full(R, Lc, dtype=np.int64)
    n0 = workloads.random_state(L, 30.0, seed=6)
    mp.start_processes(_stats_rank_main, args=(2, _free_port(), L, n0, steps, str(tmp_path)),
                       nprocs=2, join=True, start_method="spawn")
    whole = _local_stats(L, n0, 0, R, steps, 3)
    for r in (0, 1):
        with open(tmp_path / f"stats_{r}.pkl", "rb") as f:
            m = pickle.load(f)
        assert m["count"] == whole["count"] == R * steps
        for k in ("s1", "s2", "snb"):
            assert np.array_equal(m[k], whole[k]), k
        var64 = m["cov64"][:, [0, 3, 5]]
        assert (np.abs(m["cov32"][:, [0, 3, 5]] - var64) / var64).max() <= 1e-6
        scale = np.sqrt(var64[:, [0, 0, 1]] * var64[:, [1, 2, 2]])
        assert (np.abs(m["cov32"][:, [1, 2, 4]] - m["cov64"][:, [1, 2, 4]]) / scale).max() <= 1e-6
