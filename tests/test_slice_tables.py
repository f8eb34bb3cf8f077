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
