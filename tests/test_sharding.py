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
