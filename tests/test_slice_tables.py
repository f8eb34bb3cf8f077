"""The library's slice-sampler tables (exact big-integer C-step laws built on
the host) against the oracle's independent computation, on CPU."""
import random

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def lib():
    from paper_1706_01094_gb300 import build
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    build.build()
    from paper_1706_01094_gb300 import mclg
    return mclg


def test_rows_equal_oracle(lib):
    rnd = random.Random(7)
    for _ in range(400):
        N = rnd.randint(2, 400)
        J = rnd.randint(-N, N)
        b = rnd.randrange((N - abs(J)) & 1, N - abs(J) + 1, 2)
        C = rnd.choice([0, 1, 2, 5, 10])
        lam = rnd.choice([(1, 1), (1, 2), (3, 7), (255, 256), (0, 1)])
        F, dmin, dmax = lib.slice_row(N, J, b, C, lam)
        Fo, omin, omax = oracle.slice_cdf(N, J, b, C, lam)
        assert (dmin, dmax) == (omin, omax)
        assert [int(v) for v in F] == [int(Fo[dmin + k + C]) for k in range(dmax - dmin)]


def test_rows_are_cumulative_and_symmetric(lib):
    F, dmin, dmax = lib.slice_row(120, 9, 71)
    assert (np.diff(F.astype(np.float64)) >= 0).all()
    G, gmin, gmax = lib.slice_row(120, -9, 71)
    assert (gmin, gmax) == (dmin, dmax) and np.array_equal(F, G)  # J -> -J symmetry
    with pytest.raises(lib.MCLGError):
        lib.slice_row(10, 0, 5)        # parity of b does not match the slice
    with pytest.raises(lib.MCLGError):
        lib.slice_row(10, 0, 4, C=11)  # the slice sampler draws at most 10 at once


def test_records_decide_draws_like_the_oracle(lib):
    """Record lane j of a state holds the top 15 bits of the oracle's F[c0 - 4 + j]
    (c0 = -dmin; 0 below the row, 0x7FFF past its end).  Wherever the record
    decides (q = Q >> 49 equals no lane, lies above lane 0 and below lane 7),
    every Q with those top bits draws d = #{lanes below q} - 4: checked with the
    oracle's draw at the first and last Q of such prefixes, among them the
    prefixes next to every lane."""
    rnd = random.Random(11)
    decided = 0
    for _ in range(150):
        N = rnd.randint(2, 300)
        J = rnd.randint(-N, N)
        b = rnd.randrange((N - abs(J)) & 1, N - abs(J) + 1, 2)
        C = rnd.choice([1, 3, 10])
        lam = rnd.choice([(1, 1), (2, 5), (0, 1)])
        F, dmin, dmax, R = lib.slice_row(N, J, b, C, lam, record=True)
        Fo, omin, omax = oracle.slice_cdf(N, J, b, C, lam)
        Fo = [int(Fo[d + C]) for d in range(omin, omax)]
        c0, n = -omin, omax - omin
        lanes = [0 if k < 0 else 0x7FFF if k >= n else Fo[k] >> 49
                 for k in (c0 - 4 + j for j in range(8))]
        assert [int(v) for v in R] == lanes, (N, J, b, C, lam)
        qs = {0, 1, 0x7FFE, 0x7FFF} | {rnd.randrange(0x8000) for _ in range(6)}
        qs |= {t + e for t in lanes for e in (-1, 1) if 0 <= t + e <= 0x7FFF}
        for q in sorted(qs):
            g = sum(q >= t for t in lanes)
            if q in lanes or not 1 <= g <= 7:
                continue
            decided += 1
            for Q in (q << 49, ((q + 1) << 49) - 1):
                assert oracle.slice_draw(N, J, b, Q, C, lam) == b + 2 * (g - 4), (N, J, b, Q)
    assert decided > 500


def test_rows_at_the_largest_accepted_denominators_equal_oracle(lib):
    """The exact law's numerators over D^C must fit the builder's integers: every
    (N, lambda_den) the ABI accepts gives the oracle's F (640-bit integers), and
    D = 8 N^2 lambda_den >= 2^44 is refused instead of returning a wrong row."""
    cases = [(2**20 - 1, 1), (2**20, 1), (92681, 256), (65535, 256), (46340, 1000 % 257)]
    for N, ld in cases:
        assert 8 * N * N * ld < 2**44
        for J, b in ((0, N - 2 * (N // 3)), (N // 5, (N - N // 5) % 2), (1, N - 1), (N - 2, 2)):
            for C in (10, 3):
                lam = (max(1, ld // 2), ld)
                F, dmin, dmax = lib.slice_row(N, J, b, C, lam)
                Fo, omin, omax = oracle.slice_cdf(N, J, b, C, lam)
                assert (dmin, dmax) == (omin, omax)
                assert [int(v) for v in F] == [int(Fo[dmin + k + C]) for k in range(dmax - dmin)]
    for N, ld in ((2**20 - 1, 256), (92682, 256), (2**21, 1), (3 * 2**19, 2)):
        assert 8 * N * N * ld >= 2**44
        with pytest.raises(lib.MCLGError):
            lib.slice_row(N, 0, N % 2, 10, (1, ld))


def test_d2q9_outcome_table_equals_oracle(lib):
    """The library's D2Q9 outcome table (built on the host from its own class
    list) against the oracle's, for every ordered pick and three rate sets,
    and a rate set whose probabilities exceed 1 is refused."""
    import oracle
    for lam in (oracle.D2Q9_PAPER_LAMBDA, ((128, 64, 32, 16, 8, 4, 2, 1, 96), 128),
                ((1, 2, 3, 4, 5, 6, 7, 8, 9), 37)):
        for s1 in range(9):
            for s2 in range(9):
                assert lib.pair_outcomes2d(s1, s2, lam) == oracle.d2q9_outcomes(s1, s2, lam), \
                    (s1, s2, lam)
    with pytest.raises(lib.MCLGError):   # from {5,7}: lambda_3 + 2 lambda_4 + lambda_6 > 1
        lib.pair_outcomes2d(5, 7, ((1, 1, 64, 64, 1, 64, 1, 1, 1), 128))
