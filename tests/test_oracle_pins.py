"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (cuRAND's host Philox, scipy), exact rational enumeration of the
paper's particle picks, closed forms printed in the paper, or invariants the
method must keep exactly.
"""
import ctypes
import ctypes.util
import json
import os
from fractions import Fraction
from math import sqrt

import numpy as np
import pytest

import oracle
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if path and os.path.exists(path):
            try:
                return ctypes.CDLL(path)
            except OSError:
                pass
    return None


# ---------------------------------------------------------------- Philox ---
def test_philox_matches_curand_host_generator():
    """cuRAND's host PHILOX4_32_10 generator emits, from offset 4*(65536*c0 + c2),
    the block of counter (c0, 0, c2, 0) under key (seed lo, seed hi)."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    for seed in (0, 1, 0x0F1E2D3C4B5A6978, 2**64 - 1):
        gen = ctypes.c_void_p()
        assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
        try:
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            for c0, c2 in ((0, 0), (0, 7), (3, 65535), (12345, 4321), (2**31 + 5, 17)):
                off = 4 * (65536 * c0 + c2)
                assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(off)) == 0
                out = np.zeros(4, dtype=np.uint32)
                assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                          ctypes.c_size_t(4)) == 0
                mine = oracle.philox((c0, 0, c2, 0), (seed & 0xFFFFFFFF, seed >> 32))
                assert list(mine) == list(out), (seed, c0, c2)
        finally:
            lib.curandDestroyGenerator(gen)


# ------------------------------------------------ transition probabilities ---
def _contract_probs(state, lam):
    a, b, c = state
    N = a + b + c
    ln, ld = lam.numerator, lam.denominator
    if N < 2:
        return Fraction(0), Fraction(0)
    D = 8 * N * N * ld
    T1 = 16 * a * c * ln
    T2 = T1 + b * (b - 1) * ln
    return Fraction(T1, D), Fraction(T2 - T1, D)


@pytest.mark.parametrize("lam", [Fraction(1), Fraction(1, 2), Fraction(3, 7)])
def test_thresholds_equal_enumerated_particle_picks(lam):
    """T1/D and (T2-T1)/D equal the exact law of one sub-collision of the paper's
    algorithm (Eqs. select and omega, D1Q3 table), enumerated over all N^2 draws."""
    for N in range(0, 13):
        for a in range(N + 1):
            for b in range(N + 1 - a):
                c = N - a - b
                law = exact.literal_transition((a, b, c), lam)
                pd, pu = _contract_probs((a, b, c), lam)
                assert law.get((a - 1, b + 2, c - 1), Fraction(0)) == pd
                assert law.get((a + 1, b - 2, c + 1), Fraction(0)) == pu
                assert law.get((a, b, c), Fraction(0)) == 1 - pd - pu


def test_transition_table_matches_paper_golden():
    g = json.load(open(GOLDEN))["d1q3_transitions"]
    lam = Fraction(2, 5)
    env = {"lam": lam}
    val = {k: eval(v.replace("lambda", "lam"), {}, env) for k, v in g.items() if k.startswith("P_")}
    # state with exactly one -1 particle, one +1 particle and N = 2: the only pair
    # is (-1, +1) in one of two orders; the pick law is 2*(1*1)/4 = 1/2 for a pair
    law = exact.literal_transition((1, 0, 1), lam)
    assert law[(0, 2, 0)] == Fraction(1, 2) * val["P_m1p1_to_00"]
    law = exact.literal_transition((0, 2, 0), lam)
    assert law[(1, 0, 1)] == Fraction(1, 2) * (val["P_00_to_m1p1"] + val["P_00_to_p1m1"])
    assert val["P_00_to_00"] + val["P_00_to_m1p1"] + val["P_00_to_p1m1"] == 1


# ---------------------------------------------------------- exact sampler ---
def _region_mass(T1, T2, D, q_bits=12):
    """Exact probability of each region under uniform chunks, by enumerating
    the primary chunk and the first refinement chunk; returns (mass[3], open)."""
    mass = [Fraction(0)] * 3
    open_mass = Fraction(0)
    for q0 in range(1 << q_bits):
        reg, used = oracle.decide(T1, T2, D, q0)
        if reg >= 0:
            mass[reg] += Fraction(1, 1 << q_bits)
            continue
        assert reg == -1
        for q1 in range(1 << 16):
            reg2, used2 = oracle.decide(T1, T2, D, q0, [q1])
            if reg2 >= 0:
                assert used2 == 1
                mass[reg2] += Fraction(1, 1 << (q_bits + 16))
            else:
                open_mass += Fraction(1, 1 << (q_bits + 16))
    return mass, open_mass


@pytest.mark.parametrize("T1,T2,D", [
    (16 * 3 * 5 * 1, 16 * 3 * 5 + 7 * 6, 8 * 15 * 15),      # N = 15 state (3, 7, 5), lambda 1
    (16 * 2 * 1, 16 * 2 + 0, 8 * 9),                        # (2, 1, 1)
    (0, 12 * 11, 8 * 12 * 12),                              # (0, 12, 0): no down move
    (16 * 40 * 60 * 3, 16 * 40 * 60 * 3 + 9 * 8 * 3, 8 * 109 ** 2 * 7),  # lambda 3/7
    (0, 0, 8 * 4),                                          # nothing possible
])
def test_decide_is_exact(T1, T2, D):
    """The lazily refined uniform hits each region with probability T/D exactly:
    the mass decided after 28 bits brackets the target, the rest is < 2^-27."""
    mass, open_mass = _region_mass(T1, T2, D)
    target = [Fraction(T1, D), Fraction(T2 - T1, D), Fraction(D - T2, D)]
    for k in range(3):
        assert mass[k] <= target[k] <= mass[k] + open_mass
    assert open_mass <= Fraction(2, 1 << 28)


def test_decide_reads_minimal_chunks():
    # T/D = 1/3: q0 = 1365 = floor(4096/3) is the only open primary chunk
    T1, T2, D = 1, 2, 3
    assert oracle.decide(T1, T2, D, 1364) == (0, 0)
    assert oracle.decide(T1, T2, D, 1365) == (-1, 0)
    assert oracle.decide(T1, T2, D, 1366)[0] == 1
    assert oracle.decide(T1, T2, D, 4095)[0] == 2
    # 4096/3 = 1365.333..: next 16 bits of U decide; 0x5555 = 21845.33 boundary
    assert oracle.decide(T1, T2, D, 1365, [21844]) == (0, 1)
    assert oracle.decide(T1, T2, D, 1365, [21846]) == (1, 1)
    # the cap: a fraction with no finite binary expansion, keep feeding the open chunk
    reg, used = oracle.decide(1, 2, 3, 1365, [21845] * 5)
    assert (reg, used) == (-2, 4)


# ------------------------------------------------------------- invariants ---
def _rand_case(seed, R=3, Lmax=40, mean=30):
    g = np.random.default_rng(seed)
    L = g.integers(1, Lmax, R).astype(np.uint32)
    n = g.poisson(mean, size=(3, int(L.sum()))).astype(np.uint16)
    return L, n


def test_pure_streaming_when_no_collisions():
    """C = 0: the step is the evolution equation with Xi = 0, n_i(x + v_i, t+1) = n_i(x, t)."""
    L, n = _rand_case(1, R=4)
    out, err = oracle.step(L, 7, n, 0, 1, C=0)
    assert err == 0
    off = 0
    for Lr in L:
        sl = slice(off, off + int(Lr))
        assert (out[0, sl] == np.roll(n[0, sl], -1)).all()   # v = -1 moves left
        assert (out[1, sl] == n[1, sl]).all()
        assert (out[2, sl] == np.roll(n[2, sl], 1)).all()    # v = +1 moves right
        off += int(Lr)
    out0, err = oracle.step(L, 7, n, 0, 1, C=10, lam=(0, 1))  # lambda = 0: no collision
    assert err == 0 and (out0 == out).all()


def test_conservation_and_rest_parity():
    L, n = _rand_case(2, R=3, mean=25)
    N0, J0, tot0 = oracle.moments(L, n)
    out, err = oracle.step(L, 11, n, 5, 1, flags=oracle.FLAG_NO_STREAM)
    assert err == 0
    N1, J1, tot1 = oracle.moments(L, out)
    assert (N0 == N1).all() and (J0 == J1).all()            # per node, collide only
    assert (out != n).any()
    out2, err = oracle.step(L, 11, n, 5, 20)
    assert err == 0
    _, _, tot2 = oracle.moments(L, out2)
    assert (tot2 == tot0).all()                              # globally, with streaming
    assert ((out2[1] % 2) == (n[1] % 2)).all()               # rest-particle parity, Sec. III.A
    assert out2.min() >= 0


def test_overflow_is_flagged_not_saturated():
    L = np.array([1], dtype=np.uint32)
    n = np.array([[30000], [65534], [30000]], dtype=np.uint16)
    _, err = oracle.step(L, 3, n, 0, 1, flags=oracle.FLAG_NO_STREAM)
    assert err & oracle.ERR_OVERFLOW


def test_moments_small_case():
    L = [2, 1]
    n = np.array([[1, 2, 3], [4, 5, 6], [7, 8, 10]], dtype=np.uint16)
    N, J, tot = oracle.moments(L, n)
    assert list(N) == [12, 15, 19] and list(J) == [6, 6, 7]
    assert list(tot) == [46, 19]


# ---------------------------------------------------- equilibrium closed form ---
def test_feq_zero_velocity_is_weights():
    g = json.load(open(GOLDEN))["feq_u0"]["over_rho"]
    for rho in (1.0, 12.0, 36.0):
        f = oracle.feq(rho, 0.0)
        assert np.allclose(f / rho, [float(Fraction(x)) for x in g], rtol=0, atol=1e-15)


@pytest.mark.parametrize("u", [-0.6, -0.2, 0.0, 0.1, 0.35, 0.9])
def test_feq_minimises_H_and_zeroes_collision_operator(u):
    """Eq. D1Q3equil is the minimiser of H = sum f ln(f / w) at fixed mass and
    momentum (entropic LB, Sec. IV.B) and makes Omega^(1) of Eq. collmatD1Q3 vanish."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    rho = 7.0
    f = oracle.feq(rho, u)
    assert abs(f.sum() - rho) < 1e-12 and abs(f[2] - f[0] - rho * u) < 1e-12
    assert abs(f[1] ** 2 / 8 - 2 * f[0] * f[2]) < 1e-12 * rho ** 2
    w = np.array([1 / 6, 2 / 3, 1 / 6])
    # parametrise the slice by f_0, minimise H numerically
    def H(f0):
        fm = (rho - f0 - rho * u) / 2
        fp = (rho - f0 + rho * u) / 2
        v = np.array([fm, f0, fp])
        return float((v * np.log(v / w)).sum())
    hi = rho - abs(rho * u)
    res = scipy_opt.minimize_scalar(H, bounds=(1e-9, hi - 1e-9), method="bounded",
                                    options={"xatol": 1e-12})
    assert abs(res.x - f[1]) < 1e-6
    gpi = json.load(open(GOLDEN))["pi_eq"]
    pi = sqrt(2) * (f[0] - f[1] / 2 + f[2])
    assert abs(pi - sqrt(2) * rho * (-1 + sqrt(1 + 3 * u * u))) < 1e-12 * rho
    assert gpi["expr"]


def test_local_equilibrium_small_N():
    """Stationary law of the collide-only chain on a slice: N = 1 gives M f =
    (1, 0, -sqrt(1/2)) as printed; N = 2, J = 0 gives 8/9 and 1/9 (the paper
    prints 16/17, 1/17; see the golden file)."""
    st = exact.stationary(1, 0)
    assert st == {(0, 1, 0): 1}
    M3 = (sqrt(2), -sqrt(0.5), sqrt(2))
    assert abs(sum(M3[i] * (0, 1, 0)[i] for i in range(3)) + sqrt(0.5)) < 1e-15
    st2 = exact.stationary(2, 0)
    assert st2 == {(1, 0, 1): Fraction(1, 9), (0, 2, 0): Fraction(8, 9)}
    # and it is stationary for the paper's sub-collision: detailed balance
    for N in range(2, 11):
        for J in range(-N, N + 1):
            pi = exact.stationary(N, J)
            for s, p in pi.items():
                for s2, q in exact.literal_transition(s).items():
                    if s2 != s:
                        back = exact.literal_transition(s2)[s]
                        assert p * q == pi[s2] * back


# ------------------------------------------------------------ Poisson init ---
def test_poisson_inversion_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    g = np.random.default_rng(5)
    for mu in (0.3, 2.5, 11.0, 31.9, 32.0):
        for U in g.uniform(0, 1, 300):
            k = oracle.poisson_inv(mu, U)
            ref = int(stats.poisson.ppf(U, mu))
            # scipy's ppf is the smallest k with cdf(k) >= U; ours needs U < F(k)
            if abs(stats.poisson.cdf(ref, mu) - U) > 1e-12:
                assert k == ref, (mu, U)
    assert oracle.poisson_inv(0.0, 0.999) == 0


def test_init_mean_and_variance_follow_feq():
    L = np.full(64, 1024, dtype=np.uint32)
    S = int(L.sum())
    rho, u = 20.0, 0.1
    n, err = oracle.init(L, 1, np.full(S, rho), np.full(S, u))
    assert err == 0
    f = oracle.feq(rho, u)
    m = n.astype(np.float64).mean(axis=1)
    v = n.astype(np.float64).var(axis=1)
    se = np.sqrt(f / S)
    assert (np.abs(m - f) < 5 * se).all(), (m, f)
    assert (np.abs(v - f) < 5 * f * np.sqrt(2.0 / S) + 5 * se).all(), (v, f)
    # large means go through the split into parts of at most 32
    n2, err = oracle.init([4096], 2, np.full(4096, 900.0), np.zeros(4096))
    f2 = oracle.feq(900.0, 0.0)
    assert err == 0
    assert (np.abs(n2.mean(axis=1) - f2) < 5 * np.sqrt(f2 / 4096)).all()


def test_init_rejects_bad_profiles():
    _, err = oracle.init([2], 1, [1.0, -1.0], [0.0, 0.0])
    assert err == 8
    _, err = oracle.init([2], 1, [1.0, 1.0], [0.0, 1.5])
    assert err == 8


# -------------------------------------------------------------- statistics ---
def test_stats_sums_small_case():
    Lc, R = 3, 2
    n = np.array([[1, 2, 3, 4, 5, 6], [0, 1, 0, 1, 0, 1], [2, 2, 2, 3, 3, 3]], dtype=np.uint16)
    st = oracle.Stats(Lc, R)
    st.accumulate(n)
    st.accumulate(n)
    assert st.count == 4
    v = n.reshape(3, R, Lc).astype(np.int64)
    assert (st.s1 == 2 * v.sum(axis=1).T).all()
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for p, (i, j) in enumerate(pairs):
        assert (st.s2[:, p] == 2 * (v[i] * v[j]).sum(axis=0)).all()
    for i in range(3):
        for j in range(3):
            assert (st.snb[:, 3 * i + j] == 2 * (v[i] * np.roll(v[j], -1, axis=1)).sum(axis=0)).all()
    cov = st.cov(1, 0, 2)
    samples0 = np.concatenate([v[0, :, 1], v[0, :, 1]])
    samples2 = np.concatenate([v[2, :, 1], v[2, :, 1]])
    assert abs(cov - np.cov(samples0, samples2, bias=True)[0, 1]) < 1e-12


def test_equal_rationals_give_identical_trajectories():
    """lambda = 256/256 and 1/1 define the same thresholds T/D, so the exact sampler
    makes the same decisions from the same bits (Sec. III.A with lambda = 1)."""
    L, n = _rand_case(6, R=3, mean=40)
    a, err1 = oracle.step(L, 21, n, 0, 12, lam=(1, 1))
    b, err2 = oracle.step(L, 21, n, 0, 12, lam=(256, 256))
    c, err3 = oracle.step(L, 21, n, 0, 12, lam=(3, 7))
    assert err1 == err2 == err3 == 0
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_degenerate_nodes_are_left_alone():
    """N < 2: no pair can collide (and no random bits are drawn)."""
    L = [6]
    n = np.array([[0, 1, 0, 0, 0, 1], [0, 0, 1, 0, 0, 0], [0, 0, 0, 1, 0, 0]], dtype=np.uint16)
    out, err = oracle.step(L, 1, n, 0, 3, flags=oracle.FLAG_NO_STREAM)
    assert err == 0 and np.array_equal(out, n)
