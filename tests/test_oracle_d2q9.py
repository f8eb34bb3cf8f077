"""Pins of the D2Q9 oracle (Sec. II.B, III.B, IV.B) against what the paper and
the mathematics fix: the collision classes (every momentum-conserving binary
collision, up to the symmetries of the square), the linearised relaxation of
Eq. D2Q9MOmega as the paper prints it, detailed balance of the product Poisson
law, the exact one-collision law of the particle picks, conservation, and the
entropic equilibrium of Eq. D2Q9eqdist."""
import itertools
import json
import os
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "d2q9_relaxation.json")))
VX, VY = oracle.D2Q9_VX, oracle.D2Q9_VY
W = [Fraction(x) for x in GOLD["weights"]["w"]]
LAM = GOLD["simulation_rates"]
LAM_PAPER = (LAM["num"], LAM["den"])


def test_collision_table_is_every_momentum_conserving_pair_change():
    """Brute force over all unordered velocity pairs: the pairs of pairs with equal
    total momentum are exactly the oracle's 30 collisions; under the 8 symmetries
    of the square they fall into 9 classes, whose momenta are those the paper
    lists (5 of zero momentum, two of (1,0), one of (1,1), one of (2,0))."""
    pairs = sorted({tuple(sorted(p)) for p in itertools.product(range(9), repeat=2)})
    mom = lambda p: (VX[p[0]] + VX[p[1]], VY[p[0]] + VY[p[1]])
    brute = {tuple(sorted([a, b])) for a, b in itertools.combinations(pairs, 2) if mom(a) == mom(b)}
    table = oracle.d2q9_collisions()
    assert {tuple(sorted([a, b])) for a, b, _ in table} == brute and len(brute) == 30
    # classes: orbits under the symmetry group
    def img(v, sw, sx, sy):
        x, y = VX[v], VY[v]
        nx, ny = sx * (y if sw else x), sy * (x if sw else y)
        return [i for i in range(9) if VX[i] == nx and VY[i] == ny][0]
    def orbit(c):
        out = set()
        for sw, sx, sy in itertools.product((0, 1), (-1, 1), (-1, 1)):
            a = tuple(sorted(img(v, sw, sx, sy) for v in c[0]))
            b = tuple(sorted(img(v, sw, sx, sy) for v in c[1]))
            out.add(tuple(sorted([a, b])))
        return frozenset(out)
    orbits = {orbit(c) for c in brute}
    assert len(orbits) == 9
    by_class = {}
    for a, b, k in table:
        by_class.setdefault(k, set()).add(tuple(sorted([a, b])))
    assert {frozenset(v) for v in by_class.values()} == orbits
    momenta = Counter(tuple(sorted(map(abs, mom(next(iter(v))[0])))) for v in by_class.values())
    assert momenta == {(0, 0): 5, (0, 1): 2, (1, 1): 1, (0, 2): 1}


def _one_collision_law(state, lam=LAM_PAPER):
    """Exact law of one sub-collision from `state` (Sec. III: two independent uniform
    picks of particle indices; the same particle twice collides nothing; then the
    outcome table): {new state: probability}."""
    N = sum(state)
    D = 128 * lam[1]
    law = Counter()
    vel = [s for s in range(9) for _ in range(state[s])]
    for p1 in range(N):
        for p2 in range(N):
            if p1 == p2:
                law[tuple(state)] += Fraction(1, N * N)
                continue
            s1, s2 = vel[p1], vel[p2]
            outs = oracle.d2q9_outcomes(s1, s2, lam)
            rest = Fraction(1)
            for (b0, b1), num in outs:
                p = Fraction(num, D)
                nxt = list(state)
                nxt[s1] -= 1; nxt[s2] -= 1; nxt[b0] += 1; nxt[b1] += 1
                law[tuple(nxt)] += p / (N * N)
                rest -= p
            assert rest >= 0
            law[tuple(state)] += rest / (N * N)
    return law


def _moment_matrix():
    import sympy as sp
    s3, s32, s6 = sp.sqrt(3), sp.sqrt(sp.Rational(3, 2)), sp.sqrt(6)
    h = sp.Rational(1, 2)
    return sp.Matrix([
        [1] * 9,
        [0, s3, 0, -s3, 0, s3, -s3, -s3, s3],
        [0, 0, s3, 0, -s3, s3, s3, -s3, -s3],
        [0, 3 * h, -3 * h, 3 * h, -3 * h, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 3, -3, 3, -3],
        [-1, h, h, h, h, 2, 2, 2, 2],
        [0, -s32, 0, s32, 0, s6, -s6, -s6, s6],
        [0, 0, -s32, 0, s32, s6, s6, -s6, -s6],
        [h, -1, -1, -1, -1, 2, 2, 2, 2]])


def test_linearised_relaxation_equals_the_papers_printed_operator():
    """The mean-field change per sub-collision built from the oracle's outcome
    table (ordered picks of velocities (i, j) with probability f_i f_j / rho^2),
    linearised at f = rho w and written in the moments of Eq. MomD2Q9, equals
    Eq. D2Q9MOmega term by term: one class rate at a time, every row (sigma_-,
    sigma_xy, the sigma_+ / t block, q_x, q_y).  This fixes the class numbering,
    the outcome probabilities and the velocity numbering against the paper."""
    sp = pytest.importorskip("sympy")
    M = _moment_matrix()
    w = [sp.Rational(x.numerator, x.denominator) for x in W]
    Minv = sp.diag(*w) * M.T
    assert sp.simplify(M * Minv) == sp.eye(9)
    rho = sp.Symbol("rho", positive=True)
    f = sp.symbols("f0:9")
    index = {"sigma_minus": 3, "sigma_xy": 4, "sigma_plus": 5, "q_x": 6, "q_y": 7, "t": 8}
    for c in range(1, 10):
        lam = ([128 if k == c - 1 else 0 for k in range(9)], 128)   # lambda_c = 1 alone
        Om = [0] * 9
        for s1, s2 in itertools.product(range(9), repeat=2):
            for (b0, b1), num in oracle.d2q9_outcomes(s1, s2, lam):
                rate = f[s1] * f[s2] / rho**2 * sp.Rational(num, 128 * 128)
                for v, d in ((s1, -1), (s2, -1), (b0, 1), (b1, 1)):
                    Om[v] += d * rate
        J = sp.Matrix(Om).jacobian(sp.Matrix(f)).subs({f[i]: rho * w[i] for i in range(9)})
        L = (M * J * Minv).applyfunc(lambda e: sp.nsimplify(sp.simplify(e * rho / 2)))
        for name, row in GOLD["rows"].items():
            a = index[name]
            pre = sp.Rational(row["prefactor"])
            want = {index[m]: 0 for m in index}
            for k, m in enumerate(row["moments"]):
                coeff = row["terms"].get(str(c), ["0"] * len(row["moments"]))[k]
                want[index[m]] = pre * sp.Rational(coeff)
            got = {b: L[a, b] for b in index.values()}
            assert got == want, (c, name, got, want)


def test_paper_rates_decouple_the_modes_and_make_the_stress_isotropic():
    """The simulation rates satisfy Eq. decouple and Eq. rotational exactly in the
    numbering of Eq. D2Q9MOmega."""
    lam = [Fraction(n, LAM["den"]) for n in LAM["num"]]
    dec = sum(Fraction(v) * lam[int(k) - 1] for k, v in GOLD["decouple"]["coefficients"].items())
    assert dec == 0
    rows = GOLD["rows"]
    def rate(row):
        return sum(Fraction(v[0]) * lam[int(k) - 1] for k, v in rows[row]["terms"].items()
                   if k != "7")  # Eq. rotational leaves out the lambda_7 term common to both
    assert rate("sigma_minus") == rate("sigma_xy")


@pytest.mark.parametrize("lam", [LAM_PAPER, ((128, 64, 32, 16, 8, 4, 2, 1, 96), 128)])
def test_product_poisson_law_is_in_detailed_balance(lam):
    """Exactly, for every state with N <= 5: pi(n) P(n -> n') = pi(n') P(n' -> n)
    for pi(n) = prod_i w_i^{n_i} / n_i! (the product Poisson law at u = 0, Eq.
    poisson), so it is stationary."""
    def pi(n):
        out = Fraction(1)
        for i, k in enumerate(n):
            out *= W[i] ** k / np.prod(range(1, k + 1), dtype=object) if k else 1
        return out
    for N in range(2, 6):
        states = [s for s in itertools.product(range(N + 1), repeat=9) if sum(s) == N]
        laws = {s: _one_collision_law(s, lam) for s in states}
        for s, law in laws.items():
            for s2, p in law.items():
                if s2 == s:
                    continue
                assert pi(s) * p == pi(s2) * laws[s2][s], (s, s2)


@pytest.mark.parametrize("state", [(1, 1, 0, 1, 0, 1, 0, 1, 0), (2, 1, 1, 0, 0, 0, 0, 0, 1),
                                   (0, 0, 0, 0, 0, 2, 1, 1, 1)])
def test_one_step_law_of_the_sampler_equals_the_particle_picks(state):
    """Collide-only, C = 1, many replicas of one node in the same state: the
    frequencies of the new states match the exact law of the particle picks
    (chi-square at a fixed seed)."""
    from scipy import stats
    R = 60000
    n0 = np.repeat(np.asarray(state, dtype=np.uint16)[:, None], R, axis=1)
    n1, err = oracle.d2q9_step(1, 1, R, 77, n0, 5, 1, C=1, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    law = _one_collision_law(state)
    got = Counter(map(tuple, n1.T.tolist()))
    assert set(got) <= set(law)
    keys = sorted(law)
    exp = np.array([float(law[k]) * R for k in keys])
    obs = np.array([got.get(k, 0) for k in keys])
    keep = exp >= 5
    chi2 = (((obs - exp) ** 2)[keep] / exp[keep]).sum() + ((obs[~keep].sum() - exp[~keep].sum()) ** 2 / max(exp[~keep].sum(), 1e-9) if (~keep).any() else 0)
    dof = keep.sum() - (0 if (~keep).any() else 1)
    assert stats.chi2.sf(chi2, max(dof, 1)) > 1e-4, (chi2, dof)


def test_conservation_and_streaming():
    g = np.random.default_rng(4)
    Lx, Ly, R = 7, 5, 3
    n0 = g.poisson(6, size=(9, Lx * Ly * R)).astype(np.uint16)
    rho0, jx0, jy0, tot0 = oracle.d2q9_moments(n0)
    n1, err = oracle.d2q9_step(Lx, Ly, R, 9, n0, 0, 6, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    rho1, jx1, jy1, _ = oracle.d2q9_moments(n1)
    assert np.array_equal(rho0, rho1) and np.array_equal(jx0, jx1) and np.array_equal(jy0, jy1)
    n2, err = oracle.d2q9_step(Lx, Ly, R, 9, n0, 0, 6)
    assert err == 0 and np.array_equal(oracle.d2q9_moments(n2)[3], tot0)
    # no collisions (all rates 0): pure streaming n_i(x + v_i) = n_i(x), periodic
    n3, _ = oracle.d2q9_step(Lx, Ly, R, 9, n0, 0, 1, lam=([0] * 9, 1))
    a = n0.reshape(9, R, Ly, Lx)
    for i in range(9):
        want = np.roll(np.roll(a[i], VY[i], axis=1), VX[i], axis=2)
        assert np.array_equal(n3.reshape(9, R, Ly, Lx)[i], want)


@pytest.mark.parametrize("ux,uy", [(0.0, 0.0), (0.1, 0.25), (-0.3, 0.05)])
def test_equilibrium_is_the_entropic_product_and_minimises_H(ux, uy):
    """Eq. D2Q9eqdist: at u = 0 the weights times rho; it carries density rho and
    momentum rho u; it minimises H = sum f ln(f / w) (Eq. Hfunc) at fixed density
    and momentum."""
    from scipy.optimize import minimize
    rho = 36.0
    f = oracle.d2q9_feq(rho, ux, uy)
    assert np.isclose(f.sum(), rho)
    assert np.isclose((f * VX).sum(), rho * ux) and np.isclose((f * VY).sum(), rho * uy)
    w = np.array([float(x) for x in W])
    if ux == 0 and uy == 0:
        assert np.allclose(f, rho * w)
    H = lambda g: float((g * np.log(g / w)).sum())
    cons = [{"type": "eq", "fun": lambda g: g.sum() - rho},
            {"type": "eq", "fun": lambda g: (g * VX).sum() - rho * ux},
            {"type": "eq", "fun": lambda g: (g * VY).sum() - rho * uy}]
    res = minimize(H, rho * w, constraints=cons, bounds=[(1e-9, None)] * 9, method="SLSQP",
                   options={"ftol": 1e-14, "maxiter": 500})
    assert np.allclose(res.x, f, rtol=1e-5, atol=1e-6)


def test_init_is_poisson_around_the_equilibrium():
    Lx, Ly, R = 64, 32, 4
    S = Lx * Ly * R
    n, err = oracle.d2q9_init(Lx, Ly, R, 3, np.full(S, 40.0), np.full(S, 0.1), np.full(S, -0.2))
    assert err == 0
    f = oracle.d2q9_feq(40.0, 0.1, -0.2)
    m, v = n.mean(axis=1), n.var(axis=1)
    assert np.allclose(m, f, rtol=0.03, atol=0.05) and np.allclose(v, f, rtol=0.1, atol=0.1)
