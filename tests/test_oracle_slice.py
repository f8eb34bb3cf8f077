"""Pins of the oracle's slice sampler (the C sub-collisions of a node drawn at once).

The C-step law of a node on its (N, J) slice is the C-th power of the exact
one-sub-collision matrix of the paper's particle picks (Sec. III, Sec. III.A).
The oracle computes it with big-integer dynamic programming; these tests
compare it with an independent rational matrix power (Python fractions) and
check the inversion rule and the invariants.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact

stats = pytest.importorskip("scipy.stats")


@pytest.mark.parametrize("C,lam", [(1, Fraction(1)), (3, Fraction(1, 2)), (10, Fraction(1)),
                                   (10, Fraction(3, 7))])
def test_cdf_equals_rational_matrix_power(C, lam):
    for N in range(0, 11):
        for J in range(-N, N + 1):
            states, P = exact.transition_matrix(N, J, lam)
            if not states:
                continue
            PC = exact.matpow(P, C)
            for i, (a, b, c) in enumerate(states):
                F, dmin, dmax = oracle.slice_cdf(N, J, b, C, (lam.numerator, lam.denominator))
                # the law over b' = b + 2d, cumulated in increasing d
                cum = Fraction(0)
                for d in range(-C, C + 1):
                    bp = b + 2 * d
                    for k, s in enumerate(states):
                        if s[1] == bp:
                            cum += PC[i][k]
                    want = min((cum * 2**64).numerator // (cum * 2**64).denominator, 2**64 - 1)
                    assert int(F[d + C]) == want, (N, J, b, d)
                reach = [s[1] for k, s in enumerate(states) if PC[i][k] > 0] or [b]
                assert dmin <= (min(reach) - b) // 2 and dmax >= (max(reach) - b) // 2


def test_cdf_matches_large_N_recursion_in_fractions():
    """N = 150 (the single-lattice density): the big-integer recursion against
    exact fractions propagated over the same band of states."""
    N, J, b, C = 150, 7, 99, 10
    lam = Fraction(1)
    F, dmin, dmax = oracle.slice_cdf(N, J, b, C)
    def probs(bb):
        if bb < 0 or bb > N - abs(J) or (N - abs(J) - bb) % 2:
            return Fraction(0), Fraction(0)
        a, c = (N - J - bb) // 2, (N + J - bb) // 2
        return Fraction(2 * a * c, N * N) * lam, Fraction(bb * (bb - 1), 8 * N * N) * lam
    dist = {b: Fraction(1)}
    for _ in range(C):
        new = {}
        for bb, p in dist.items():
            dn, up = probs(bb)
            new[bb] = new.get(bb, 0) + p * (1 - dn - up)
            if dn:
                new[bb + 2] = new.get(bb + 2, 0) + p * dn
            if up:
                new[bb - 2] = new.get(bb - 2, 0) + p * up
        dist = new
    cum = Fraction(0)
    for d in range(-C, C + 1):
        cum += dist.get(b + 2 * d, Fraction(0))
        want = min(int(cum * 2**64), 2**64 - 1)
        assert int(F[d + C]) == want, d
    assert (dmin, dmax) == (-10, 10)


@pytest.mark.parametrize("state,C,lam", [((3, 4, 5), 10, (1, 1)), ((0, 9, 1), 4, (1, 2)),
                                          ((6, 0, 6), 10, (3, 7))])
def test_slice_step_law_equals_matrix_power(state, C, lam):
    N, J = sum(state), state[2] - state[0]
    states, P = exact.transition_matrix(N, J, Fraction(*lam))
    row = exact.matpow(P, C)[states.index(tuple(state))]
    probs = np.array([float(p) for p in row])
    L = np.full(40, 2500, dtype=np.uint32)
    S = int(L.sum())
    n = np.tile(np.array(state, dtype=np.uint16)[:, None], (1, S))
    out, err = oracle.slice_step(L, 77, n, 2, 1, C=C, lam=lam, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    counts = np.zeros(len(states))
    for s, cnt in zip(*np.unique(out.T, axis=0, return_counts=True)):
        counts[states.index(tuple(int(v) for v in s))] += cnt
    exp = probs * S
    keep = exp >= 5
    chi2 = (((counts[keep] - exp[keep]) ** 2) / exp[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4


def test_slice_step_invariants():
    g = np.random.default_rng(1)
    L = np.array([37, 64, 5], dtype=np.uint32)
    n = g.poisson(40, size=(3, int(L.sum()))).astype(np.uint16)
    N0, J0, tot0 = oracle.moments(L, n)
    out, err = oracle.slice_step(L, 3, n, 0, 1, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    N1, J1, _ = oracle.moments(L, out)
    assert (N0 == N1).all() and (J0 == J1).all() and (out != n).any()
    out2, err = oracle.slice_step(L, 3, n, 0, 25)
    assert err == 0
    assert np.array_equal(oracle.moments(L, out2)[2], tot0)
    assert ((out2[1] % 2) == (n[1] % 2)).all()
    # the single-particle and empty nodes stay as they are
    tiny = np.array([[0, 1], [1, 0], [0, 0]], dtype=np.uint16)
    same, err = oracle.slice_step([2], 3, tiny, 0, 4, flags=oracle.FLAG_NO_STREAM)
    assert err == 0 and np.array_equal(same, tiny)
    with pytest.raises(ValueError):
        oracle.slice_cdf(10, 0, 6, C=11)


def test_nodes_beyond_n_max_take_the_sequential_draws():
    """The range rule: with n_max below every mass the slice step is the
    sequential step bit for bit; with n_max in the middle of the masses, the heavy
    nodes of a collide-only step agree with the sequential step and the light
    ones with the table draw."""
    g = np.random.default_rng(4)
    L = np.array([40, 17, 64], dtype=np.uint32)
    n = g.poisson(12, size=(3, int(L.sum()))).astype(np.uint16)
    seq, err = oracle.step(L, 21, n, 5, 6)
    assert err == 0
    sl, err = oracle.slice_step(L, 21, n, 5, 6, n_max=1)
    assert err == 0 and np.array_equal(sl, seq)
    N = n.astype(np.int64).sum(axis=0)
    cut = int(np.median(N))
    mixed, err = oracle.slice_step(L, 21, n, 5, 1, flags=oracle.FLAG_NO_STREAM, n_max=cut)
    assert err == 0
    seq1, _ = oracle.step(L, 21, n, 5, 1, flags=oracle.FLAG_NO_STREAM)
    tab1, _ = oracle.slice_step(L, 21, n, 5, 1, flags=oracle.FLAG_NO_STREAM, n_max=4096)
    heavy = N > cut
    assert heavy.any() and (~heavy).any()
    assert np.array_equal(mixed[:, heavy], seq1[:, heavy])
    assert np.array_equal(mixed[:, ~heavy], tab1[:, ~heavy])
    assert not np.array_equal(seq1[:, ~heavy & (N >= 2)], tab1[:, ~heavy & (N >= 2)])


def test_slice_uniform_bits_are_uniform_and_independent():
    """Q (its top 16 bits from a Philox block shared by eight nodes, the rest
    from a block shared by two) behaves as uniform bits: each byte of Q is
    uniform over 256 values, neighbouring nodes' top bytes are uncorrelated, and
    no two nodes share a prefix."""
    qs = np.array([oracle.slice_q(x, 3, 7, 12345) for x in range(16384)], dtype=np.uint64)
    for shift in (56, 48, 40, 0):
        counts = np.bincount(((qs >> np.uint64(shift)) & np.uint64(0xFF)).astype(np.int64),
                             minlength=256)
        chi2 = ((counts - 64.0) ** 2 / 64.0).sum()
        assert stats.chi2.sf(chi2, 255) > 1e-4, shift
    top = (qs >> np.uint64(56)).astype(np.float64)
    assert abs(np.corrcoef(top[:-1], top[1:])[0, 1]) < 0.04
    assert len(set(int(q) for q in qs)) == len(qs)


def test_slice_uniform_layout_over_philox_blocks():
    """Q's bits come from the oracle's Philox4x32-10 (pinned to cuRAND's host
    generator) as the contract lays them out: the top 16 bits of nodes
    8k .. 8k+7 read in order are the four words of block (k, r, t, 6 << 28),
    low half first, and the next 48 bits of node x are the low 16 bits of word
    1 (even x) or 3 (odd x) and word 0 or 2 of block (x // 2, r, t, 4 << 28)."""
    seed, r, t = 987654321987, 5, 11
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for k in (0, 1, 77, 2**29 - 1):
        top = [oracle.slice_q(8 * k + j, r, t, seed) >> 48 for j in range(8)]
        w = oracle.philox([k, r, t, 6 << 28], key)
        assert [int(v) for v in w] == [top[2 * i] | top[2 * i + 1] << 16 for i in range(4)]
        for x in (8 * k, 8 * k + 3):
            w = oracle.philox([x // 2, r, t, 4 << 28], key)
            lo, mid = (w[0], w[1]) if x % 2 == 0 else (w[2], w[3])
            assert oracle.slice_q(x, r, t, seed) & (2**48 - 1) == (int(mid) & 0xFFFF) << 32 | int(lo)


def test_results_do_not_depend_on_thread_count_or_remembered_laws():
    """The node loops run on several host threads and the exact laws are
    remembered between calls: neither may change a single bit.  One thread with
    laws computed afresh (distinct lambda keys, so nothing is remembered yet)
    against all threads with laws remembered from the first pass."""
    from paper_1706_01094_gb300 import workloads
    L = np.array([3000, 17, 65536 + 9, 64], dtype=np.uint32)
    n0 = workloads.random_state(L, 60.0, seed=44)
    results = []
    for threads in (1, 0, 3):
        oracle.set_threads(threads)
        a, ea = oracle.step(L, 5, n0, 2, 3, lam=(5, 7))
        b, eb = oracle.slice_step(L, 5, n0, 2, 3, lam=(5, 7), n_max=80)
        rho = np.full(int(L.sum()), 37.5)
        u = np.linspace(-0.3, 0.3, int(L.sum()))
        c, ec = oracle.init(L, 9, rho, u)
        results.append((a, b, c, ea, eb, ec))
    oracle.set_threads(0)
    for other in results[1:]:
        for x, y in zip(results[0], other):
            assert np.array_equal(x, y)
    # a remembered law equals the same law computed with C changed and back
    F1 = oracle.slice_cdf(77, -5, 30, 10, (5, 7))
    oracle.slice_cdf(77, -5, 30, 9, (5, 7))
    F2 = oracle.slice_cdf(77, -5, 30, 10, (5, 7))
    assert np.array_equal(F1[0], F2[0]) and F1[1:] == F2[1:]
