"""GPU parity: the sm_103a library against the CPU oracle, bit for bit.

Every test calls the library through its C ABI (ctypes binding) and compares
integer fields element by element with the oracle on the same seeded inputs.
"""
import numpy as np
import pytest

import oracle
from paper_1706_01094_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_01094_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1706_01094_gb300 import mclg  # noqa: E402

MODES = [mclg.MODE_PLAIN, mclg.MODE_BATCHED, mclg.MODE_PERSISTENT, mclg.MODE_AUTO]


def run_gpu(L, seed, n0, t0, steps, **kw):
    with mclg.Lattice(L, seed=seed, **kw) as lat:
        lat.set_state(n0, t=t0)
        lat.step(steps)
        out, t = lat.get_state()
        assert t == t0 + steps
    return out


def test_philox_device_matches_oracle():
    g = np.random.default_rng(0)
    ctr = g.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:8] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
               [2**32 - 1] * 4, [5, 6, 7, 1 << 28], [9, 9, 9, 9]]
    for seed in (0, 1, 0x0123456789ABCDEF):
        d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
        out = mclg.philox(d_ctr, seed).cpu().numpy().view(np.uint32)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for i in range(0, 4096, 97):
            assert list(out[i]) == list(oracle.philox(ctr[i], key)), (seed, i)


@pytest.mark.parametrize("L", [[1], [2], [7], [8], [9], [64], [1000], [4099]])
def test_single_lattice_bit_exact(L):
    n0 = workloads.random_state(L, 25.0, seed=len(L) + L[0])
    want, err = oracle.step(L, 5, n0, 17, 12)
    assert err == 0
    got = run_gpu(L, 5, n0, 17, 12)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", MODES)
def test_ragged_batch_all_modes_bit_exact(mode):
    L = [64, 1, 37, 128, 9, 1024, 5, 16384, 16391, 3000, 33]
    n0 = workloads.random_state(L, 12.0, seed=7)
    want, err = oracle.step(L, 123, n0, 0, 20)
    assert err == 0
    got = run_gpu(L, 123, n0, 0, 20, mode=mode)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", [mclg.MODE_PLAIN, mclg.MODE_PERSISTENT])
@pytest.mark.parametrize("C,lam", [(1, (1, 1)), (3, (1, 2)), (10, (3, 7)), (23, (1, 1)),
                                   (10, (0, 1)), (0, (1, 1)), (17, (255, 256))])
def test_parameters_bit_exact(mode, C, lam):
    L = [50, 200, 13]
    n0 = workloads.random_state(L, 40.0, seed=C)
    want, err = oracle.step(L, 99, n0, 3, 9, C=C, lam=lam)
    assert err == 0
    got = run_gpu(L, 99, n0, 3, 9, C=C, lam=lam, mode=mode)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", [mclg.MODE_PLAIN, mclg.MODE_PERSISTENT])
def test_collide_only_bit_exact(mode):
    L = [300, 41]
    n0 = workloads.random_state(L, 30.0, seed=2)
    want, err = oracle.step(L, 8, n0, 0, 15, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    got = run_gpu(L, 8, n0, 0, 15, flags=mclg.NO_STREAM, mode=mode)
    assert np.array_equal(got, want)
    N0, J0, _ = oracle.moments(L, n0)
    N1, J1, _ = oracle.moments(L, got)
    assert (N0 == N1).all() and (J0 == J1).all()


def test_dense_nodes_and_refinement_paths():
    """Large N (64-bit thresholds) and thousands of node-steps: the 2^-11 refinement
    path is taken many times and must consume the same chunks as the oracle."""
    L = [2048, 777]
    g = np.random.default_rng(4)
    n0 = g.integers(0, 20000, size=(3, sum(L))).astype(np.uint16)
    want, err = oracle.step(L, 31, n0, 1000, 6)
    assert err == 0
    for mode in (mclg.MODE_PLAIN, mclg.MODE_PERSISTENT):
        got = run_gpu(L, 31, n0, 1000, 6, mode=mode)
        assert np.array_equal(got, want)


def test_device_pointers_and_moments():
    L = [100, 57]
    n0 = workloads.random_state(L, 15.0, seed=9)
    dn = torch.from_numpy(n0.view(np.int16)).cuda().contiguous()
    with mclg.Lattice(L, seed=2) as lat:
        lat.set_state(dn, t=0)
        lat.step(7)
        out = torch.empty_like(dn)
        lat.get_state(out)
        Nd = torch.empty(sum(L), dtype=torch.int32, device="cuda")
        Jd = torch.empty(sum(L), dtype=torch.int32, device="cuda")
        _, _, tot = lat.moments(Nd, Jd)
        Nh, Jh, toth = lat.moments()
    want, _ = oracle.step(L, 2, n0, 0, 7)
    assert np.array_equal(out.cpu().numpy().view(np.uint16), want)
    N, J, T = oracle.moments(L, want)
    assert np.array_equal(Nd.cpu().numpy(), N) and np.array_equal(Jd.cpu().numpy(), J)
    assert np.array_equal(Nh, N) and np.array_equal(Jh, J)
    assert np.array_equal(tot, T) and np.array_equal(toth, T)


def test_init_matches_oracle():
    wl = workloads.uneven(R=20, Lmax=3000, steps=1)
    want, err = oracle.init(wl.L, 77, wl.rho, wl.u)
    assert err == 0
    with mclg.Lattice(wl.L, seed=77) as lat:
        lat.init(wl.rho, wl.u)
        got, t = lat.get_state()
    assert t == 0
    assert np.array_equal(got, want)


def test_overflow_is_reported_and_cleared():
    L = [64]
    n0 = np.array([[30000] * 64, [65535] * 64, [30000] * 64], dtype=np.uint16)
    with mclg.Lattice(L, seed=1, flags=mclg.NO_STREAM) as lat:
        lat.set_state(n0)
        lat.step(1)
        assert lat.sync_status() == 4
        with pytest.raises(mclg.MCLGError):
            lat.step(1)
        lat.set_state(workloads.random_state(L, 3.0, seed=1))
        lat.step(2)
        lat.sync()


def test_invalid_arguments():
    with pytest.raises(mclg.MCLGError):
        mclg.Lattice([0])
    with pytest.raises(mclg.MCLGError):
        mclg.Lattice([8], lam=(2, 1))
    with pytest.raises(mclg.MCLGError):
        mclg.Lattice([8, 9], flags=mclg.STATS)
    with mclg.Lattice([8]) as lat:
        with pytest.raises(mclg.MCLGError):
            lat.step(1)                      # no state yet
        with pytest.raises(mclg.MCLGError):
            lat.init(np.full(8, -1.0), np.zeros(8))


def test_statistics_exact_sums_and_fp32_error():
    R, Lc = 64, 256
    L = np.full(R, Lc, dtype=np.uint32)
    wl = workloads.fluct(R=R, L=Lc, rho=50.0, u=0.2)
    n0, err = oracle.init(L, 1, wl.rho, wl.u)
    assert err == 0
    ref = oracle.Stats(Lc, R)
    n = n0
    steps = 60
    for k in range(steps):
        n, err = oracle.step(L, 1, n, k, 1)
        ref.accumulate(n)
    with mclg.Lattice(L, seed=1, flags=mclg.STATS) as lat:
        lat.set_state(n0, t=0)
        lat.stats_reset()
        lat.step(steps)
        st = lat.stats_read()
    assert st["count"] == ref.count == steps * R
    assert np.array_equal(st["s1"], ref.s1)
    assert np.array_equal(st["s2"], ref.s2)
    assert np.array_equal(st["snb"], ref.snb)
    # FP32 compensated path vs the exact int64 -> FP64 normalisation
    var32 = st["cov32"][:, [0, 3, 5]].astype(np.float64)
    var64 = st["cov64"][:, [0, 3, 5]]
    rel = np.abs(var32 - var64) / np.abs(var64)
    assert rel.max() <= 1e-6, rel.max()
    # off-diagonal: error relative to sqrt(var_i var_j)
    scale = np.sqrt(var64[:, [0, 0, 1]] * var64[:, [1, 2, 2]])
    off = np.abs(st["cov32"][:, [1, 2, 4]] - st["cov64"][:, [1, 2, 4]]) / scale
    assert off.max() <= 1e-6, off.max()
    for x in (0, 17, Lc - 1):
        for q, (i, j) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
            assert abs(st["cov64"][x, q] - ref.cov(x, i, j)) <= 1e-12 * max(1.0, abs(ref.cov(x, i, j)))


# ---------------------------------------------------------------- full sizes ---
def test_single_lattice_full_size_prefix():
    """The 2^24-node single lattice in the launch configuration the benchmark times:
    the first steps bit-exact against the oracle, then conservation over a longer run."""
    wl = workloads.single()
    n0, err = oracle.init(wl.L, wl.seed, wl.rho, wl.u)
    assert err == 0
    want, err = oracle.step(wl.L, wl.seed, n0, 0, 2)
    assert err == 0
    with mclg.Lattice(wl.L, seed=wl.seed) as lat:
        lat.init(wl.rho, wl.u)
        got0, _ = lat.get_state()
        assert np.array_equal(got0, n0)
        tot0 = lat.totals()
        lat.step(2)
        got, _ = lat.get_state()
        assert np.array_equal(got, want)
        lat.step(200)
        assert np.array_equal(lat.totals(), tot0)
        fin, _ = lat.get_state()
        assert np.array_equal(fin[1] % 2, n0[1] % 2)      # rest-particle parity, Sec. III.A


def test_batched_full_size_prefix():
    wl = workloads.batched()
    n0, err = oracle.init(wl.L, wl.seed, wl.rho, wl.u)
    assert err == 0
    want, err = oracle.step(wl.L, wl.seed, n0, 0, 2)
    assert err == 0
    for mode in (mclg.MODE_PERSISTENT, mclg.MODE_BATCHED):
        with mclg.Lattice(wl.L, seed=wl.seed, mode=mode) as lat:
            lat.set_state(n0)
            lat.step(2)
            got, _ = lat.get_state()
        assert np.array_equal(got, want)


def test_uneven_full_size_prefix():
    wl = workloads.uneven()
    n0, err = oracle.init(wl.L, wl.seed, wl.rho, wl.u)
    assert err == 0
    want, err = oracle.step(wl.L, wl.seed, n0, 0, 2)
    assert err == 0
    with mclg.Lattice(wl.L, seed=wl.seed, mode=mclg.MODE_PERSISTENT) as lat:
        lat.init(wl.rho, wl.u)
        lat.step(2)
        got, _ = lat.get_state()
    assert np.array_equal(got, want)


def test_split_batch_with_first_replica_is_bit_exact():
    """Two handles with first_replica = index of their first replica reproduce one
    handle over the whole batch (the rule that lets a batch shard over GPUs)."""
    L = [300, 17, 1024, 64, 5000, 9]
    n0 = workloads.random_state(L, 18.0, seed=12)
    whole = run_gpu(L, 3, n0, 5, 11, mode=mclg.MODE_PERSISTENT)
    cut = 3
    S0 = sum(L[:cut])
    a = run_gpu(L[:cut], 3, n0[:, :S0].copy(), 5, 11, mode=mclg.MODE_PLAIN)
    b = run_gpu(L[cut:], 3, n0[:, S0:].copy(), 5, 11, mode=mclg.MODE_BATCHED, first_replica=cut)
    assert np.array_equal(np.concatenate([a, b], axis=1), whole)
    want, err = oracle.step(L[cut:], 3, n0[:, S0:], 5, 11, first_replica=cut)
    assert err == 0 and np.array_equal(b, want)


@pytest.mark.parametrize("u", [0.0, 0.2])
def test_fluctuation_statistics_full_size(u):
    """512 replicas x 4096 nodes at rho = 50 (the fluctuation workload): the FP32
    compensated (co)variances agree with the exact int64 -> FP64 ones to 1e-6, and
    the occupations are Poisson around the entropic equilibrium (Eqs. poisson,
    Poisson2, corr, D1Q3equil): pooled mean and variance equal f^eq."""
    wl = workloads.fluct(u=u)
    f = oracle.feq(50.0, u)
    with mclg.Lattice(wl.L, seed=wl.seed, flags=mclg.STATS) as lat:
        lat.init(wl.rho, wl.u)
        tot0 = lat.totals()
        lat.step(200)
        lat.stats_reset()
        lat.step(400)
        st = lat.stats_read()
        assert np.array_equal(lat.totals(), tot0)
    cnt = st["count"]
    assert cnt == 400 * wl.replicas
    var32 = st["cov32"][:, [0, 3, 5]].astype(np.float64)
    var64 = st["cov64"][:, [0, 3, 5]]
    assert (np.abs(var32 - var64) / var64).max() <= 1e-6
    scale = np.sqrt(var64[:, [0, 0, 1]] * var64[:, [1, 2, 2]])
    assert (np.abs(st["cov32"][:, [1, 2, 4]] - st["cov64"][:, [1, 2, 4]]) / scale).max() <= 1e-6
    mean = st["s1"].sum(axis=0) / (cnt * 4096)
    assert np.allclose(mean, f, rtol=2e-3), (mean, f)
    assert np.allclose(var64.mean(axis=0), f, rtol=1e-2), (var64.mean(axis=0), f)
    # correlator of distinct velocities at one node is zero (Eq. corr)
    corr = st["cov64"][:, [1, 2, 4]].mean(axis=0) / np.sqrt(f[[0, 0, 1]] * f[[1, 2, 2]])
    assert np.abs(corr).max() < 0.01, corr


@pytest.mark.parametrize("mode,L", [(mclg.MODE_AUTO, [777]), (mclg.MODE_BATCHED, [64, 9, 300]),
                                    (mclg.MODE_PERSISTENT, [5000, 64, 9000, 33])])
def test_graph_replayed_steps_bit_exact(mode, L):
    """Per-step launches replayed from captured CUDA graphs (32 steps each), from
    both buffer parities, with a remainder launched directly."""
    n0 = workloads.random_state(L, 22.0, seed=sum(L))
    want, err = oracle.step(L, 17, n0, 40, 1 + 70 + 33)
    assert err == 0
    with mclg.Lattice(L, seed=17, mode=mode) as lat:
        lat.set_state(n0, t=40)
        lat.step(1)      # odd parity for the next call
        lat.step(70)     # 2 graph replays + 6 direct steps
        lat.step(33)     # 1 replay from the other parity + 1 direct step
        got, t = lat.get_state()
    assert t == 40 + 104
    assert np.array_equal(got, want)


def test_near_maximum_occupations_agree_with_oracle():
    """Occupations near the uint16 limit take the fully checked path: the error flag
    and, where no transition overflows, the state agree with the oracle."""
    g = np.random.default_rng(8)
    for trial in range(6):
        S = 256
        n0 = g.integers(60000, 65536, size=(3, S)).astype(np.uint16)
        n0[:, ::3] = g.integers(0, 30, size=(3, (S + 2) // 3)).astype(np.uint16)
        want, err = oracle.step([S], 40 + trial, n0, 0, 1, C=1 + trial, flags=oracle.FLAG_NO_STREAM)
        with mclg.Lattice([S], seed=40 + trial, C=1 + trial, flags=mclg.NO_STREAM) as lat:
            lat.set_state(n0)
            lat.step(1)
            status = lat.sync_status()
            assert (status == 4) == bool(err & oracle.ERR_OVERFLOW), (trial, status, err)
            if status == 0:
                got, _ = lat.get_state()
                assert np.array_equal(got, want)


def test_largest_masses_without_overflow():
    # (a, b, c) = (65535, 1, 65535): only {-1,+1} -> {0,0} can happen and b stays small
    S = 64
    n0 = np.tile(np.array([[65535], [1], [65535]], dtype=np.uint16), (1, S))
    want, err = oracle.step([S], 9, n0, 0, 1, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    got = run_gpu([S], 9, n0, 0, 1, flags=mclg.NO_STREAM)
    assert np.array_equal(got, want)


def test_time_limit_and_equal_rationals():
    L = [100, 7]
    n0 = workloads.random_state(L, 30.0, seed=2)
    t0 = 2**32 - 5
    want, err = oracle.step(L, 4, n0, t0, 5)
    assert err == 0
    with mclg.Lattice(L, seed=4) as lat:
        lat.set_state(n0, t=t0)
        with pytest.raises(mclg.MCLGError):
            lat.step(6)                      # would pass t = 2^32
        lat.step(5)
        got, t = lat.get_state()
        assert t == 2**32 and np.array_equal(got, want)
    a = run_gpu(L, 4, n0, 3, 20, lam=(1, 1))
    b = run_gpu(L, 4, n0, 3, 20, lam=(256, 256), mode=mclg.MODE_PERSISTENT)
    assert np.array_equal(a, b)


def test_degenerate_and_empty_nodes():
    L = [8, 1, 2]
    n0 = np.zeros((3, 11), dtype=np.uint16)
    n0[:, 1] = [0, 1, 0]
    n0[:, 8] = [1, 0, 0]                     # the single-node replica
    n0[:, 9:] = [[2, 0], [0, 3], [0, 0]]
    for mode in (mclg.MODE_PLAIN, mclg.MODE_PERSISTENT, mclg.MODE_BATCHED):
        want, err = oracle.step(L, 6, n0, 0, 7)
        assert err == 0
        assert np.array_equal(run_gpu(L, 6, n0, 0, 7, mode=mode), want)


@pytest.mark.parametrize("Lc,R", [(100, 16), (33, 5), (1, 3)])
def test_statistics_ragged_lengths_exact(Lc, R):
    """Statistics for lengths that leave part of a 32-position tile empty."""
    L = np.full(R, Lc, dtype=np.uint32)
    n0 = workloads.random_state(L, 9.0, seed=Lc)
    ref = oracle.Stats(Lc, R)
    n = n0
    for k in range(40):
        n, err = oracle.step(L, 2, n, k, 1)
        ref.accumulate(n)
    with mclg.Lattice(L, seed=2, flags=mclg.STATS) as lat:
        lat.set_state(n0, t=0)
        lat.stats_reset()
        lat.step(40)
        st = lat.stats_read()
    assert st["count"] == ref.count
    assert np.array_equal(st["s1"], ref.s1)
    assert np.array_equal(st["s2"], ref.s2)
    assert np.array_equal(st["snb"], ref.snb)


@pytest.mark.parametrize("variant", range(6))
def test_every_plain_launch_variant_bit_exact(variant):
    """Each launch shape of the plain kernel (1 or 2 nodes per thread, register
    bounds) gives the oracle's bits, per replica and batched, including replicas
    whose padding fills whole vectors."""
    L = [8, 3, 100, 1, 517, 64, 6]
    n0 = workloads.random_state(L, 40.0, seed=variant)
    want, err = oracle.step(L, 5, n0, 2, 4)
    assert err == 0
    for mode in (mclg.MODE_BATCHED, mclg.MODE_PLAIN):
        assert np.array_equal(run_gpu(L, 5, n0, 2, 4, mode=mode, kernel_variant=variant), want)
    with pytest.raises(mclg.MCLGError):
        mclg.Lattice(L, kernel_variant=6)  # six variants: 0 .. 5


@pytest.mark.parametrize("mode", [mclg.MODE_PLAIN, mclg.MODE_BATCHED, mclg.MODE_PERSISTENT])
def test_galilean_rate_bit_exact(mode):
    """The Galilean-invariant collision rate (end of Sec. IV.A), node by node as the
    oracle computes it, in every mode of the sequential sampler."""
    L = [64, 37, 300, 9]
    g = np.random.default_rng(13)
    S = sum(L)
    n0 = np.stack([g.poisson(3, S), g.poisson(12, S), g.poisson(9, S)]).astype(np.uint16)
    want, err = oracle.step(L, 21, n0, 3, 12, lam=(3, 4), flags=oracle.FLAG_GALILEAN)
    assert err == 0
    got = run_gpu(L, 21, n0, 3, 12, lam=(3, 4), flags=mclg.GALILEAN, mode=mode)
    assert np.array_equal(got, want)


def test_statistics_merged_at_the_end_of_every_call():
    """The FP32 running moments take the exact sums in batches (one per 32-step
    graph and one per call); after calls of 7, 40 and 1 steps, each read gives the
    oracle's exact sums and FP32 (co)variances within 1e-6 of the exact ones."""
    R, Lc = 40, 96
    L = np.full(R, Lc, dtype=np.uint32)
    wl = workloads.fluct(R=R, L=Lc, rho=30.0, u=0.1)
    n0, err = oracle.init(L, 3, wl.rho, wl.u)
    assert err == 0
    ref = oracle.Stats(Lc, R)
    n, t = n0, 0
    with mclg.Lattice(L, seed=3, flags=mclg.STATS, sampler=mclg.SAMPLER_SLICE) as lat:
        lat.set_state(n0, t=0)
        lat.stats_reset()
        for steps in (7, 40, 1):
            lat.step(steps)
            for _ in range(steps):
                n, err = oracle.slice_step(L, 3, n, t, 1)
                assert err == 0
                ref.accumulate(n)
                t += 1
            st = lat.stats_read()
            assert st["count"] == ref.count == t * R
            assert np.array_equal(st["s1"], ref.s1) and np.array_equal(st["s2"], ref.s2)
            assert np.array_equal(st["snb"], ref.snb)
            var32 = st["cov32"][:, [0, 3, 5]].astype(np.float64)
            var64 = st["cov64"][:, [0, 3, 5]]
            assert (np.abs(var32 - var64) / np.abs(var64)).max() <= 1e-6


@pytest.mark.parametrize("flags", [0, mclg.NO_STREAM])
def test_state_transfer_through_pinned_host_buffers(flags):
    """mclg_set_state / mclg_get_state with pinned host buffers (the e2e path of
    the benchmark) give the fields of pageable buffers, on ragged replicas, with
    and without streaming, and agree with the oracle."""
    L = [1000, 37, 4099, 8]
    S = sum(L)
    n0 = workloads.random_state(L, 30.0, seed=9)
    with mclg.Lattice(L, seed=3, flags=flags) as lat:
        pin_in = torch.from_numpy(n0.view(np.int16)).pin_memory()
        lat.set_state(pin_in, t=5)
        got, t = lat.get_state()                  # pageable, staged
        assert t == 5 and np.array_equal(got, n0)
        lat.step(3)
        want, _ = lat.get_state()
        pin_out = torch.zeros((3, S), dtype=torch.int16).pin_memory()
        lat.get_state(pin_out)                     # pinned
        assert np.array_equal(pin_out.numpy().view(np.uint16), want)
        lat.set_state(pin_out, t=8)                # and back
        again, _ = lat.get_state()
        assert np.array_equal(again, want)
    ref, err = oracle.step(L, 3, n0, 5, 3, flags=oracle.FLAG_NO_STREAM if flags else 0)
    assert err == 0 and np.array_equal(want, ref)
