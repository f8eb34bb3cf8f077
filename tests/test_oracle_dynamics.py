"""Statistical pins of the oracle's dynamics (fixed seeds, so deterministic).

* The law of one collide-only time step (C sub-collisions) from a fixed state
  equals the C-th power of the exact one-sub-collision matrix of the paper's
  particle picks (Sec. III), for both the bit-exact contract sampler and the
  literal particle-pick form.
* With streaming, the ensemble means relax to the entropic equilibrium of
  Eq. D1Q3equil (Sec. IV.A, Fig. D1Q3equil), not to the polynomial LB
  equilibrium of Eq. LBequil.
* Started from product-Poisson(f^eq), occupations stay Poisson: mean and
  variance equal f^eq and distinct velocities are uncorrelated (Eqs. poisson,
  Poisson2, corr).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact

stats = pytest.importorskip("scipy.stats")


def _chi2_pvalue(counts, probs, min_expected=5.0):
    total = counts.sum()
    exp = probs * total
    keep = exp >= min_expected
    obs_k, exp_k = counts[keep], exp[keep]
    # lump the sparse bins together
    if (~keep).any():
        obs_k = np.append(obs_k, counts[~keep].sum())
        exp_k = np.append(exp_k, exp[~keep].sum())
    chi2 = float(((obs_k - exp_k) ** 2 / np.maximum(exp_k, 1e-300)).sum())
    return float(stats.chi2.sf(chi2, len(obs_k) - 1))


@pytest.mark.parametrize("mode", ["contract", "literal"])
@pytest.mark.parametrize("state,C,lam", [((3, 4, 5), 10, (1, 1)), ((0, 9, 1), 4, (1, 2)),
                                          ((6, 0, 6), 10, (3, 7))])
def test_one_step_law_equals_matrix_power(mode, state, C, lam):
    N = sum(state)
    J = state[2] - state[0]
    states, P = exact.transition_matrix(N, J, Fraction(*lam))
    row = exact.matpow(P, C)[states.index(tuple(state))]
    probs = np.array([float(p) for p in row])
    L = np.full(50, 2000, dtype=np.uint32)
    S = int(L.sum())
    n = np.tile(np.array(state, dtype=np.uint16)[:, None], (1, S))
    fn = oracle.step if mode == "contract" else oracle.literal_step
    out, err = fn(L, 20240601, n, 3, 1, C=C, lam=lam, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    idx = {s: k for k, s in enumerate(states)}
    counts = np.zeros(len(states))
    for s, cnt in zip(*np.unique(out.T, axis=0, return_counts=True)):
        counts[idx[tuple(int(v) for v in s)]] += cnt
    assert counts.sum() == S
    assert _chi2_pvalue(counts, probs) > 1e-4


def test_collide_only_reaches_local_equilibrium():
    """Many collide-only steps give the stationary law prod w^n / n! on the slice."""
    state = (1, 2, 5)
    N, J = 8, 4
    pi = exact.stationary(N, J)
    states = sorted(pi)
    L = np.full(20, 1000, dtype=np.uint32)
    S = int(L.sum())
    n = np.tile(np.array(state, dtype=np.uint16)[:, None], (1, S))
    out, err = oracle.step(L, 99, n, 0, 40, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    counts = np.zeros(len(states))
    for s, cnt in zip(*np.unique(out.T, axis=0, return_counts=True)):
        counts[states.index(tuple(int(v) for v in s))] += cnt
    # 400 sub-collisions mix this 5-state slice to within 1e-9 of stationarity
    _, Pm = exact.transition_matrix(N, J)
    row = exact.matpow(Pm, 400)[exact.slice_states(N, J).index(state)]
    sl = exact.slice_states(N, J)
    for s in states:
        assert abs(float(row[sl.index(s)]) - float(pi[s])) < 1e-9
    probs = np.array([float(pi[s]) for s in states])
    assert _chi2_pvalue(counts, probs) > 1e-4


def test_means_relax_to_entropic_equilibrium():
    """Fig. D1Q3equil: from a uniform non-equilibrium start with u = 0.4 the
    measured <n_i> approach f^eq (Eq. D1Q3equil), clearly apart from LB's f^0."""
    R, Lr, rho, u = 16, 64, 50.0, 0.4
    L = np.full(R, Lr, dtype=np.uint32)
    S = R * Lr
    n = np.tile(np.array([10, 10, 30], dtype=np.uint16)[:, None], (1, S))  # N = 50, J = 20
    n, err = oracle.step(L, 5, n, 0, 200)
    assert err == 0
    acc = np.zeros(3)
    steps = 200
    for k in range(steps):
        n, err = oracle.step(L, 5, n, 200 + k, 1)
        assert err == 0
        acc += n.astype(np.float64).mean(axis=1)
    mean = acc / steps
    feq = oracle.feq(rho, u)
    w = np.array([1 / 6, 2 / 3, 1 / 6])
    v = np.array([-1.0, 0.0, 1.0])
    f0 = rho * w * (1 + 3 * v * u + 4.5 * (v * u) ** 2 - 1.5 * u * u)   # Eq. LBequil, theta = 1/3
    # statistical error ~0.03 (time-correlated samples) plus an O(1/S) shift from
    # the exactly fixed totals of this finite system
    assert np.abs(mean - feq).max() < 0.12, (mean, feq)
    assert np.abs(feq - f0).max() > 0.5


def test_poisson_statistics_preserved():
    """Eqs. poisson and corr: Poisson(f^eq) stays Poisson under the dynamics."""
    R, Lr, rho, u = 32, 64, 20.0, 0.1
    L = np.full(R, Lr, dtype=np.uint32)
    S = R * Lr
    n, err = oracle.init(L, 1, np.full(S, rho), np.full(S, u))
    assert err == 0
    st = oracle.Stats(Lr, R)
    for k in range(150):
        n, err = oracle.step(L, 1, n, k, 1)
        assert err == 0
        if k >= 20:
            st.accumulate(n)
    f = oracle.feq(rho, u)
    M = st.count * Lr
    mean = st.s1.sum(axis=0) / M
    assert np.abs(mean - f).max() < 0.1, (mean, f)
    # pooled (co)variances over positions: every position has the same law
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    s2 = st.s2.sum(axis=0) / M
    for p, (i, j) in enumerate(pairs):
        cov = s2[p] - mean[i] * mean[j]
        corr = cov / np.sqrt(f[i] * f[j])
        target = 1.0 if i == j else 0.0
        assert abs(corr - target) < 0.06, (i, j, corr)


def test_galilean_rate_is_lambda_over_sqrt_1_plus_3u2_rounded_down():
    """q / 256 <= lt / sqrt(1 + 3 u^2) < (q + 1) / 256 with u = J / N (end of
    Sec. IV.A), checked in 50-digit decimal arithmetic, including exact ties."""
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    g = np.random.default_rng(9)
    cases = [(100, 0, (1, 1)), (5, 5, (1, 1)), (100, 30, (1, 1)), (7, -3, (3, 7)), (60000, 17, (255, 256))]
    cases += [(int(N), int(g.integers(-N, N + 1)), (int(a), int(b)))
              for N, (a, b) in zip(g.integers(2, 200000, 400),
                                   [(g.integers(0, 9), 8)] * 200 + [(1, 1)] * 200)]
    for N, J, (ln, ld) in cases:
        q = oracle.galilean_q(N, J, (ln, ld))
        lam = Decimal(ln) / Decimal(ld) / (1 + 3 * (Decimal(J) / Decimal(N)) ** 2).sqrt()
        assert Decimal(q) / 256 <= lam < Decimal(q + 1) / 256, (N, J, ln, ld, q)


@pytest.mark.parametrize("stepper", ["step", "slice_step"])
def test_galilean_rate_at_rest_nodes_is_the_constant_rate(stepper):
    """With J = 0 at every node (kept by collisions without streaming) the
    Galilean-invariant rate is lambda~ itself, so the step equals the plain step
    at lambda = lambda~ bit for bit (the exact decisions compare with the same
    rational thresholds)."""
    fn = getattr(oracle, stepper)
    L = np.array([64, 33], dtype=np.uint32)
    g = np.random.default_rng(2)
    side = g.poisson(6, int(L.sum())).astype(np.uint16)
    n = np.stack([side, g.poisson(20, int(L.sum())).astype(np.uint16), side])
    flags = oracle.FLAG_NO_STREAM
    want, err = fn(L, 4, n, 0, 5, lam=(1, 2), flags=flags)
    assert err == 0
    got, err = fn(L, 4, n, 0, 5, lam=(1, 2), flags=flags | oracle.FLAG_GALILEAN)
    assert err == 0 and np.array_equal(got, want)
    moving = n.copy()
    moving[2] += 3                               # J = 3 at every node: a slower rate
    a, _ = fn(L, 4, moving, 0, 5, lam=(1, 2), flags=flags)
    b, _ = fn(L, 4, moving, 0, 5, lam=(1, 2), flags=flags | oracle.FLAG_GALILEAN)
    assert not np.array_equal(a, b)
