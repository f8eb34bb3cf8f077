"""Whole-field parity at the benchmarked sizes: every node of the 2^24-node
single lattice after 100 steps (both samplers, in the launch configuration
bench.py times), the 4096-replica batch and the 1000-replica uneven batch
after 50 steps in the persistent mode, all bit for bit against the oracle
(which runs its node loops on every host core)."""
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

oracle.set_threads(0)


def _diff(got, want):
    bad = np.nonzero((got != want).any(axis=0))[0]
    return f"{bad.size} nodes differ, first {bad[:5].tolist()}"


@pytest.mark.parametrize("sampler", [mclg.SAMPLER_SLICE, mclg.SAMPLER_SEQUENTIAL])
def test_single_lattice_whole_field_100_steps(sampler):
    """The single-lattice workload (L = 2^24, rho = 100 with a 1 % density wave,
    u = 0, Poisson(f^eq) start): the initial field, the field after the first 20
    steps (launched one by one, as a short benchmark run issues them) and after
    80 more (32-step graph replays plus a remainder) equal the oracle's on every
    node."""
    wl = workloads.single()
    ostep = oracle.slice_step if sampler == mclg.SAMPLER_SLICE else oracle.step
    n0, err = oracle.init(wl.L, wl.seed, wl.rho, wl.u)
    assert err == 0
    stream = torch.cuda.Stream()
    with mclg.Lattice(wl.L, seed=wl.seed, C=wl.C, lam=wl.lam, sampler=sampler,
                      stream=stream) as lat:
        lat.init(wl.rho, wl.u)
        got, _ = lat.get_state()
        assert np.array_equal(got, n0), _diff(got, n0)
        want, t = n0, 0
        for chunk in (20, 80):
            lat.step(chunk)
            got, tg = lat.get_state()
            want, err = ostep(wl.L, wl.seed, want, t, chunk, C=wl.C, lam=wl.lam)
            t += chunk
            assert err == 0 and tg == t
            assert np.array_equal(got, want), _diff(got, want)
        assert lat.sync_status() == mclg.MCLG_OK


@pytest.mark.parametrize("name,steps", [("batched", 50), ("uneven", 50)])
def test_batches_whole_field_persistent(name, steps):
    """The 4096 x 1024 batch (rho, u per replica) and the uneven batch (1000
    replicas of 32 .. 65536 nodes, long ones stepped beside the persistent
    kernel) after 50 steps in the persistent mode, every node."""
    wl = workloads.BY_NAME[name]()
    n0, err = oracle.init(wl.L, wl.seed, wl.rho, wl.u)
    assert err == 0
    want, err = oracle.step(wl.L, wl.seed, n0, 0, steps, C=wl.C, lam=wl.lam)
    assert err == 0
    with mclg.Lattice(wl.L, seed=wl.seed, mode=mclg.MODE_PERSISTENT) as lat:
        lat.init(wl.rho, wl.u)
        lat.step(steps)
        got, _ = lat.get_state()
    assert np.array_equal(got, want), _diff(got, want)


def _stats_errors(st):
    var32 = st["cov32"][:, [0, 3, 5]].astype(np.float64)
    var64 = st["cov64"][:, [0, 3, 5]]
    scale = np.sqrt(var64[:, [0, 0, 1]] * var64[:, [1, 2, 2]])
    return ((np.abs(var32 - var64) / var64).max(),
            (np.abs(st["cov32"][:, [1, 2, 4]] - st["cov64"][:, [1, 2, 4]]) / scale).max())


@pytest.mark.parametrize("u", [0.0, 0.2])
def test_statistics_workload_fp32_bound_over_2000_steps(u):
    """The fluctuation workload (512 x 4096, rho = 50) with the slice sampler, as
    bench.py runs it: after 200 burn-in steps, 2000 steps of statistics (63 merges
    of 32-step batches into the FP32 running moments) keep every FP32 variance
    within 1e-6 relative, and every covariance within 1e-6 of sqrt(var_i var_j),
    of the FP64 value normalised from the exact int64 sums."""
    wl = workloads.fluct(u=u)
    with mclg.Lattice(wl.L, seed=wl.seed, flags=mclg.STATS, sampler=mclg.SAMPLER_SLICE) as lat:
        lat.init(wl.rho, wl.u)
        lat.step(200)
        lat.stats_reset()
        lat.step(2000)
        st = lat.stats_read()
    assert st["count"] == 2000 * wl.replicas
    ev, ec = _stats_errors(st)
    assert ev <= 1e-6 and ec <= 1e-6, (ev, ec)


def test_statistics_exact_sums_against_oracle_slice_sampler():
    """The int64 sums of the fluctuation workload's first 40 steps with the slice
    sampler equal the oracle's (sums of n_i, n_i n_j and neighbour products)."""
    wl = workloads.fluct(u=0.2)
    Lc, R = int(wl.L[0]), wl.replicas
    n, err = oracle.init(wl.L, wl.seed, wl.rho, wl.u)
    assert err == 0
    ref = oracle.Stats(Lc, R)
    for t in range(40):
        n, err = oracle.slice_step(wl.L, wl.seed, n, t, 1)
        assert err == 0
        ref.accumulate(n)
    with mclg.Lattice(wl.L, seed=wl.seed, flags=mclg.STATS, sampler=mclg.SAMPLER_SLICE) as lat:
        lat.init(wl.rho, wl.u)
        lat.step(40)
        st = lat.stats_read()
    assert st["count"] == ref.count
    assert np.array_equal(st["s1"], ref.s1)
    assert np.array_equal(st["s2"], ref.s2)
    assert np.array_equal(st["snb"], ref.snb)


def test_statistics_fp32_bound_beyond_2_to_24_samples():
    """Past 2^24 samples per position the merge's sample counts are no longer
    exact in FP32; the running moments must still meet the 1e-6 bound
    (512 replicas x 64 nodes, 33000 steps = 1.7e7 samples per position)."""
    R, Lc, steps = 512, 64, 33000
    L = np.full(R, Lc, dtype=np.uint32)
    rho = np.full(R * Lc, 50.0)
    u = np.full(R * Lc, 0.1)
    with mclg.Lattice(L, seed=3, flags=mclg.STATS, sampler=mclg.SAMPLER_SLICE) as lat:
        lat.init(rho, u)
        lat.step(100)
        lat.stats_reset()
        lat.step(steps)
        st = lat.stats_read()
    assert st["count"] == steps * R > 2**24
    ev, ec = _stats_errors(st)
    assert ev <= 1e-6 and ec <= 1e-6, (ev, ec)


def test_batch_whole_field_slice_sampler():
    """The 4096 x 1024 batch's first 512 replicas (densities across the batch's
    whole range) with the slice sampler and tables to mass 512, the configuration
    bench.py times: every node after 20 steps in the persistent kernel (the
    per-step kernel over a batch is checked bit for bit in test_gpu_slice)."""
    full = workloads.batched()
    R = 512
    L = full.L[:R]
    rho, u = full.rho[: R * int(L[0])], full.u[: R * int(L[0])]
    n0, err = oracle.init(L, full.seed, rho, u)
    assert err == 0
    want, err = oracle.slice_step(L, full.seed, n0, 0, 20, C=full.C, lam=full.lam, n_max=512)
    assert err == 0
    with mclg.Lattice(L, seed=full.seed, mode=mclg.MODE_PERSISTENT, sampler=mclg.SAMPLER_SLICE,
                      slice_n_max=512) as lat:
        lat.init(rho, u)
        lat.step(20)
        got, _ = lat.get_state()
    assert np.array_equal(got, want), _diff(got, want)
