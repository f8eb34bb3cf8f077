"""Exact rational tools for pinning the oracle (test infrastructure only).

Pure Python with ``fractions.Fraction``; meant for small particle numbers.

* ``literal_transition``: the distribution of one sub-collision of the paper's
  algorithm (Sec. III, Eqs. select and omega; D1Q3 table of Sec. III.A),
  obtained by enumerating all N^2 ordered draws (r1, r2) of particle indices
  and the tabulated outcome probabilities.  Drawing the same particle twice
  collides nothing.
* ``slice_states`` / ``stationary``: the states with fixed mass N and momentum
  J, and the law proportional to prod_i w_i^{n_i} / n_i! on them (Eq. poisson
  restricted to one (N, J) slice).
* ``transition_matrix`` / ``matpow``: the one-sub-collision Markov matrix on a
  slice and its C-th power (one time step without streaming).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

# D1Q3 weights, Eq. D1Q3wi; index order (v = -1, 0, +1)
W = (Fraction(1, 6), Fraction(2, 3), Fraction(1, 6))


def literal_transition(state, lam: Fraction = Fraction(1)) -> dict:
    """Exact distribution of the state after one sub-collision of the paper's algorithm."""
    a, b, c = state
    N = a + b + c
    out: dict = {}

    def add(s, p):
        if p:
            out[s] = out.get(s, Fraction(0)) + p

    if N == 0:
        return {tuple(state): Fraction(1)}
    counts = (a, b, c)
    cum = (a, a + b, a + b + c)

    def kind(r):  # Eq. select with r in [1, N], velocity order (-1, 0, +1)
        for s in range(3):
            if r <= cum[s]:
                return s
        raise AssertionError

    pick = Fraction(1, N * N)
    for r1 in range(1, N + 1):
        for r2 in range(1, N + 1):
            s1, s2 = kind(r1), kind(r2)
            if r1 == r2:
                add(tuple(state), pick)
                continue
            if {s1, s2} == {0, 2}:
                # P_{-1 1 -> 0 0} = lambda, P_{-1 1 -> -1 1} = 1 - lambda
                add((a - 1, b + 2, c - 1), pick * lam)
                add(tuple(state), pick * (1 - lam))
            elif s1 == 1 and s2 == 1:
                # P_{00 -> -1 1} = P_{00 -> 1 -1} = lambda/16, P_{00 -> 00} = 1 - lambda/8
                add((a + 1, b - 2, c + 1), pick * lam / 8)
                add(tuple(state), pick * (1 - lam / 8))
            else:
                add(tuple(state), pick)
    assert sum(out.values()) == 1 and all(min(s) >= 0 for s in out)
    _ = counts
    return out


def slice_states(N: int, J: int) -> list:
    """All (a, b, c) >= 0 with a + b + c = N and c - a = J, ordered by b."""
    out = []
    for b in range(N + 1):
        rest = N - b
        if (rest + J) % 2 or abs(J) > rest:
            continue
        c = (rest + J) // 2
        a = rest - c
        out.append((a, b, c))
    return out


def stationary(N: int, J: int) -> dict:
    """Law proportional to prod_i w_i^{n_i} / n_i! on the (N, J) slice."""
    states = slice_states(N, J)
    wts = {}
    for s in states:
        v = Fraction(1)
        for i in range(3):
            v *= W[i] ** s[i] / factorial(s[i])
        wts[s] = v
    Z = sum(wts.values())
    return {s: v / Z for s, v in wts.items()}


def transition_matrix(N: int, J: int, lam: Fraction = Fraction(1)):
    states = slice_states(N, J)
    idx = {s: k for k, s in enumerate(states)}
    P = [[Fraction(0)] * len(states) for _ in states]
    for s in states:
        for s2, p in literal_transition(s, lam).items():
            P[idx[s]][idx[s2]] += p
    return states, P


def matpow(P, k: int):
    n = len(P)
    R = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    B = [row[:] for row in P]
    while k:
        if k & 1:
            R = [[sum(R[i][m] * B[m][j] for m in range(n)) for j in range(n)] for i in range(n)]
        B = [[sum(B[i][m] * B[m][j] for m in range(n)) for j in range(n)] for i in range(n)]
        k >>= 1
    return R
