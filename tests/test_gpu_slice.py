"""GPU parity of the slice sampler (the C sub-collisions of a node drawn at once
from exact tables) against the oracle, bit for bit."""
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

SLICE = mclg.SAMPLER_SLICE


def run_slice(L, seed, n0, t0, steps, **kw):
    with mclg.Lattice(L, seed=seed, sampler=SLICE, **kw) as lat:
        lat.set_state(n0, t=t0)
        lat.step(steps)
        out, t = lat.get_state()
        assert t == t0 + steps
    return out


@pytest.mark.parametrize("mode", [mclg.MODE_AUTO, mclg.MODE_PLAIN, mclg.MODE_BATCHED])
def test_slice_ragged_batch_bit_exact(mode):
    L = [64, 1, 37, 128, 9, 1024, 5, 3, 300]
    n0 = workloads.random_state(L, 15.0, seed=3)
    want, err = oracle.slice_step(L, 12, n0, 6, 9)
    assert err == 0
    assert np.array_equal(run_slice(L, 12, n0, 6, 9, mode=mode), want)


@pytest.mark.parametrize("C,lam", [(10, (1, 1)), (3, (1, 2)), (1, (3, 7)), (0, (1, 1)),
                                   (10, (255, 256)), (7, (0, 1))])
def test_slice_parameters_bit_exact(C, lam):
    L = [50, 200, 13]
    n0 = workloads.random_state(L, 30.0, seed=C + 1)
    want, err = oracle.slice_step(L, 99, n0, 3, 5, C=C, lam=lam)
    assert err == 0
    assert np.array_equal(run_slice(L, 99, n0, 3, 5, C=C, lam=lam), want)


def test_slice_collide_only_and_graph_replay():
    L = [300, 41]
    n0 = workloads.random_state(L, 25.0, seed=2)
    want, err = oracle.slice_step(L, 8, n0, 0, 70, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    got = run_slice(L, 8, n0, 0, 70, flags=mclg.NO_STREAM)   # 2 graph replays + 6 direct
    assert np.array_equal(got, want)
    n1 = workloads.random_state([777], 25.0, seed=5)
    want, err = oracle.slice_step([777], 8, n1, 11, 65)
    assert err == 0 and np.array_equal(run_slice([777], 8, n1, 11, 65), want)


@pytest.mark.parametrize("variant", [0, 2, 5])
def test_nodes_beyond_n_max_take_sequential_draws(variant):
    """Masses above the tables' range collide with the sequential sampler's draws,
    node by node as the oracle does; with n_max = 1 the whole step equals the
    sequential sampler's."""
    L = [16, 333, 40]
    n0 = workloads.random_state(L, 10.0, seed=1)
    n0[:, 3] = [100, 200, 100]                 # mass 400 at one node
    for n_max in (20, 300, 450):
        want, err = oracle.slice_step(L, 1, n0, 0, 6, n_max=n_max)
        assert err == 0
        got = run_slice(L, 1, n0, 0, 6, slice_n_max=n_max, kernel_variant=variant)
        assert np.array_equal(got, want), n_max
    seq, err = oracle.step(L, 1, n0, 0, 6)
    assert err == 0
    assert np.array_equal(run_slice(L, 1, n0, 0, 6, slice_n_max=1, kernel_variant=variant), seq)
    with pytest.raises(mclg.MCLGError):
        mclg.Lattice(L, sampler=SLICE, C=11)
    with pytest.raises(mclg.MCLGError):
        mclg.Lattice(L, sampler=SLICE, slice_n_max=1025)


def test_slice_full_size_sampled_nodes():
    """The 2^24-node single lattice: every sampled node's post-collision state is
    recomputed by the oracle from the pre-step field and its own random bits."""
    wl = workloads.single()
    with mclg.Lattice(wl.L, seed=wl.seed, sampler=SLICE) as lat:
        lat.init(wl.rho, wl.u)
        lat.step(3)
        before, t = lat.get_state()
        lat.step(1)
        after, _ = lat.get_state()
    L = int(wl.L[0])
    g = np.random.default_rng(0)
    ys = np.concatenate([[0, 1, L - 2, L - 1], g.integers(0, L, 3000)])
    for y in ys:
        y = int(y)
        a, b, c = (int(v) for v in before[:, y])
        N, J = a + b + c, c - a
        assert N <= oracle.SLICE_N_MAX                # every node on the tables here
        nb = oracle.slice_draw(N, J, b, oracle.slice_q(y, 0, t, wl.seed)) if N >= 2 else b
        assert nb >= 0
        na, nc = (N - J - nb) // 2, (N + J - nb) // 2
        assert after[1, y] == nb
        assert after[0, (y - 1) % L] == na      # v = -1 moved left
        assert after[2, (y + 1) % L] == nc      # v = +1 moved right


@pytest.mark.parametrize("variant", range(20))
def test_slice_every_launch_variant_bit_exact(variant):
    """Each launch shape of the slice kernel (2, 4 or 8 nodes per thread, register
    bounds; for single-replica launches the warp-specialised form with bulk-copy
    stages, the grid-stride form and the temporally blocked form) gives the
    oracle's bits, on ragged replicas whose ends fall inside a thread's vector, on
    one long lattice, and without streaming."""
    L = [8, 3, 100, 1, 517, 64, 6]
    n0 = workloads.random_state(L, 40.0, seed=variant)
    want, err = oracle.slice_step(L, 5, n0, 2, 4)
    assert err == 0
    for mode in (mclg.MODE_BATCHED, mclg.MODE_PLAIN):
        got = run_slice(L, 5, n0, 2, 4, mode=mode, kernel_variant=variant)
        assert np.array_equal(got, want), mode
    n1 = workloads.random_state([4099], 90.0, seed=7)
    want, err = oracle.slice_step([4099], 6, n1, 1, 3)
    assert err == 0
    assert np.array_equal(run_slice([4099], 6, n1, 1, 3, kernel_variant=variant), want)
    with pytest.raises(mclg.MCLGError):
        mclg.Lattice(L, sampler=SLICE, kernel_variant=20)  # twenty variants: 0 .. 19
    for Ls in ([1], [7], [8], [1031], [3 * 4096 + 13]):     # tails inside a tile and a vector
        n2 = workloads.random_state(Ls, 45.0, seed=Ls[0])
        want, err = oracle.slice_step(Ls, 6, n2, 9, 5)
        assert err == 0
        assert np.array_equal(run_slice(Ls, 6, n2, 9, 5, kernel_variant=variant), want), Ls
    want, err = oracle.slice_step(L, 5, n0, 2, 4, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    got = run_slice(L, 5, n0, 2, 4, flags=mclg.NO_STREAM, kernel_variant=variant)
    assert np.array_equal(got, want)


def test_slice_galilean_rate_bit_exact():
    """Slice tables built with each slice's Galilean-invariant rate, heavy nodes
    with the sequential draws at their own rate."""
    L = [64, 37, 300, 9]
    g = np.random.default_rng(13)
    S = sum(L)
    n0 = np.stack([g.poisson(3, S), g.poisson(12, S), g.poisson(9, S)]).astype(np.uint16)
    for n_max in (256, 20):
        want, err = oracle.slice_step(L, 21, n0, 3, 12, lam=(3, 4), flags=oracle.FLAG_GALILEAN,
                                      n_max=n_max)
        assert err == 0
        got = run_slice(L, 21, n0, 3, 12, lam=(3, 4), flags=mclg.GALILEAN, slice_n_max=n_max)
        assert np.array_equal(got, want), n_max


@pytest.mark.parametrize("variant", range(6, 20))
def test_single_replica_forms_walk_many_tiles(variant):
    """A lattice long enough that every CTA of the warp-specialised kernel cycles
    through its ring of shared-memory stages several times, and every warp of the
    grid-stride kernel walks many tiles (2^24 + 12345 nodes, a tail inside the
    last tile and inside a vector), two steps, every node."""
    L = [(1 << 24) + 12345]
    n0 = workloads.random_state(L, 33.0, seed=variant)
    want, err = oracle.slice_step(L, 17, n0, 40, 2)
    assert err == 0
    got = run_slice(L, 17, n0, 40, 2, kernel_variant=variant)
    bad = np.nonzero((got != want).any(axis=0))[0]
    assert bad.size == 0, f"{bad.size} nodes differ, first {bad[:5].tolist()}"


@pytest.mark.parametrize("config", [None, 0, 3])
@pytest.mark.parametrize("Lc,R,flags,dense", [(100, 37, 0, False), (33, 5, 0, False),
                                              (1, 3, 0, False), (70, 9, mclg.NO_STREAM, False),
                                              (64, 33, 0, False), (40, 11, 0, True)])
def test_slice_statistics_form_exact_sums(Lc, R, flags, dense, config):
    """The slice step's statistics form (the step kernel adds the field it reads),
    autotuned and pinned to two of its configurations (kernel_variant):
    every field after a reset counted once over calls of 5, 33 and 1 steps (graph
    replays among them) and across a reset; tiles with empty positions, ragged
    replica counts, collide-only runs, and values of 2^14 or more (64-bit path)."""
    L = np.full(R, Lc, dtype=np.uint32)
    n0 = workloads.random_state(L, 12.0, seed=Lc + R)
    if dense:
        n0[:, 3] = [20000, 17000, 19000]
        n0[:, Lc + 7] = [16384, 300, 16500]
    oflags = oracle.FLAG_NO_STREAM if flags & mclg.NO_STREAM else 0
    ref = oracle.Stats(Lc, R)
    n, t = n0, 0
    with mclg.Lattice(L, seed=6, flags=mclg.STATS | flags, sampler=SLICE,
                      kernel_variant=config) as lat:
        if config is not None:
            assert lat.tuning()["stats_config"] == config
        lat.set_state(n0, t=0)
        lat.stats_reset()
        for steps in (5, 33, 1, "reset", 4):
            if steps == "reset":
                lat.stats_reset()
                ref = oracle.Stats(Lc, R)
                continue
            lat.step(steps)
            for _ in range(steps):
                n, err = oracle.slice_step(L, 6, n, t, 1, flags=oflags)
                assert err == 0
                ref.accumulate(n)
                t += 1
            st = lat.stats_read()
            assert st["count"] == ref.count
            assert np.array_equal(st["s1"], ref.s1)
            assert np.array_equal(st["s2"], ref.s2)
            assert np.array_equal(st["snb"], ref.snb)
        got, _ = lat.get_state()
    assert np.array_equal(got, n)


@pytest.mark.parametrize("flags", [0, mclg.NO_STREAM, mclg.GALILEAN])
def test_slice_persistent_kernel_bit_exact(flags):
    """The persistent kernel with the slice sampler (table draws on chip for
    masses up to n_max, the sequential draws above), on a ragged batch with
    replicas beyond a work unit (stepped beside it) and heavy nodes."""
    L = [64, 1, 37, 128, 9, 1024, 5, 4099, 300, 16391, 33]
    n0 = workloads.random_state(L, 18.0, seed=flags + 1)
    n0[:, 70] = [150, 100, 120]                  # a mass beyond the tables at node 70
    oflags = (oracle.FLAG_NO_STREAM if flags & mclg.NO_STREAM else 0) | \
        (oracle.FLAG_GALILEAN if flags & mclg.GALILEAN else 0)
    for n_max in (256, 60):
        want, err = oracle.slice_step(L, 23, n0, 9, 70, flags=oflags, n_max=n_max)
        assert err == 0
        got = run_slice(L, 23, n0, 9, 70, mode=mclg.MODE_PERSISTENT, flags=flags,
                        slice_n_max=n_max)
        assert np.array_equal(got, want), n_max


def test_slice_persistent_full_size_batch_prefix():
    """The 4096 x 1024 batch (rho per replica up to 500: many masses beyond the
    tables) with the slice sampler in the persistent kernel, 10 steps, every node."""
    wl = workloads.batched()
    n0, err = oracle.init(wl.L, wl.seed, wl.rho, wl.u)
    assert err == 0
    want, err = oracle.slice_step(wl.L, wl.seed, n0, 0, 10)
    assert err == 0
    with mclg.Lattice(wl.L, seed=wl.seed, sampler=SLICE, mode=mclg.MODE_PERSISTENT) as lat:
        lat.set_state(n0)
        lat.step(10)
        got, _ = lat.get_state()
    bad = np.nonzero((got != want).any(axis=0))[0]
    assert bad.size == 0, f"{bad.size} nodes differ, first {bad[:5].tolist()}"


# tiles of the temporally blocked configurations (window E = threads of the CTA,
# or of the warp, x nodes per thread; halo K on each side)
_TB_TILES = {14: 992, 15: 496, 16: 120, 17: 112, 18: 480, 19: 992}


@pytest.mark.parametrize("variant", range(14, 20))
def test_blocked_form_many_steps_bit_exact(variant):
    """The temporally blocked form over many steps per launch: lattices shorter
    than one window (it then wraps several times), of odd length (the random
    numbers' node pairs straddle the wrap), one and two tiles with tails, and a
    tile plus one node; step counts below, at and above the steps of one launch,
    and past a 32-step graph replay."""
    T = _TB_TILES[variant]
    for L, steps in (([1], 3), ([2], 17), ([5], 9), ([33], 40), ([1000], 16), ([T], 5),
                     ([T + 1], 17), ([2 * T + 37], 70), ([3 * T - 6], 33)):
        n0 = workloads.random_state(L, 37.0, seed=L[0])
        want, err = oracle.slice_step(L, 8, n0, 11, steps)
        assert err == 0
        got = run_slice(L, 8, n0, 11, steps, kernel_variant=variant)
        bad = np.nonzero((got != want).any(axis=0))[0]
        assert bad.size == 0, f"L={L} steps={steps}: {bad.size} nodes differ, first {bad[:5].tolist()}"


@pytest.mark.parametrize("variant", [14, 16, 19])
def test_blocked_form_heavy_nodes_rates_and_no_stream(variant):
    """Nodes beyond the tables collided in place by the sequential draws, the
    Galilean rate, other C and lambda, and collide-only steps, over 40 steps."""
    L = [3 * _TB_TILES[variant] + 11]
    n0 = workloads.random_state(L, 40.0, seed=3)
    want, err = oracle.slice_step(L, 4, n0, 0, 40, n_max=48)
    assert err == 0
    assert np.array_equal(run_slice(L, 4, n0, 0, 40, slice_n_max=48, kernel_variant=variant), want)
    want, err = oracle.slice_step(L, 4, n0, 5, 40, C=3, lam=(3, 4), flags=oracle.FLAG_GALILEAN)
    assert err == 0
    got = run_slice(L, 4, n0, 5, 40, C=3, lam=(3, 4), flags=mclg.GALILEAN, kernel_variant=variant)
    assert np.array_equal(got, want)
    want, err = oracle.slice_step(L, 4, n0, 5, 40, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    got = run_slice(L, 4, n0, 5, 40, flags=mclg.NO_STREAM, kernel_variant=variant)
    assert np.array_equal(got, want)
