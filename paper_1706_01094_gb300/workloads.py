"""Seeded synthetic workloads shaped like the paper's D1Q3 runs.

This module only generates inputs: replica lengths L_r and the density and
velocity profiles rho(x), u(x) handed to ``mclg_init``.  It holds none of the
method's arithmetic, so both the CUDA path and the CPU oracle can be fed from
it.  Parameters are drawn with numpy's PCG64 generator from the stated seed.

Workloads (the paper's D1Q3 runs are L_x = 100..1000, C = 10, lambda = 1,
rho = 12..300, Sec. III.A and Sec. IV.A; these scale them up):

* ``small``      16 replicas x L = 64, rho = 20, u = 0.1, 1000 steps.
* ``single``     one lattice, L = 2^24, rho(x) = 100 (1 + 0.01 sin(2 pi 4 x / L)),
                 u = 0, 10^4 steps.
* ``batched``    4096 replicas x L = 1024, rho_r ~ U[5, 500], u_r ~ U[-0.3, 0.3],
                 2000 steps.
* ``uneven``     1000 replicas, L_r log-uniform in [32, 65536] (rounded),
                 rho_r log-uniform in [2, 1000], u(x) = 0.2 sin(2 pi x / L_r),
                 5000 steps.
* ``fluct``      512 replicas x L = 4096, rho = 50, u in {0, 0.2}, 1000 burn-in
                 then 10^4 measured steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    L: np.ndarray          # uint32 [R] replica lengths
    rho: np.ndarray        # float64 [sum L] density per node
    u: np.ndarray          # float64 [sum L] velocity per node
    steps: int             # time steps of the full run
    seed: int = 1          # Philox key of the run
    C: int = 10            # sub-collisions per node and step
    lam: tuple = (1, 1)    # lambda = lam[0] / lam[1]
    burn_in: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def replicas(self) -> int:
        return int(self.L.size)

    @property
    def nodes(self) -> int:
        return int(self.L.sum())

    def node_steps(self, steps: int | None = None) -> int:
        return self.nodes * (self.steps if steps is None else steps)


def _uniform_profiles(L, rho_r, u_r):
    rho = np.repeat(np.asarray(rho_r, dtype=np.float64), L)
    u = np.repeat(np.asarray(u_r, dtype=np.float64), L)
    return rho, u


def small(R: int = 16, L: int = 64, rho: float = 20.0, u: float = 0.1, steps: int = 1000,
          seed: int = 1) -> Workload:
    Ls = np.full(R, L, dtype=np.uint32)
    r, v = _uniform_profiles(Ls, np.full(R, rho), np.full(R, u))
    return Workload("small", Ls, r, v, steps, seed)


def single(L: int = 1 << 24, rho0: float = 100.0, amp: float = 0.01, k: int = 4,
           steps: int = 10_000, seed: int = 1) -> Workload:
    x = np.arange(L, dtype=np.float64)
    rho = rho0 * (1.0 + amp * np.sin(2.0 * np.pi * k * x / L))
    u = np.zeros(L, dtype=np.float64)
    return Workload("single", np.array([L], dtype=np.uint32), rho, u, steps, seed,
                    meta={"rho0": rho0, "amp": amp, "k": k})


def batched(R: int = 4096, L: int = 1024, steps: int = 2000, seed: int = 1,
            param_seed: int = 1) -> Workload:
    g = np.random.default_rng(param_seed)
    rho_r = g.uniform(5.0, 500.0, R)
    u_r = g.uniform(-0.3, 0.3, R)
    Ls = np.full(R, L, dtype=np.uint32)
    r, v = _uniform_profiles(Ls, rho_r, u_r)
    return Workload("batched", Ls, r, v, steps, seed, meta={"rho_r": rho_r, "u_r": u_r})


def uneven(R: int = 1000, Lmin: int = 32, Lmax: int = 65536, rmin: float = 2.0,
           rmax: float = 1000.0, amp: float = 0.2, steps: int = 5000, seed: int = 1,
           param_seed: int = 1) -> Workload:
    g = np.random.default_rng(param_seed)
    Ls = np.exp(g.uniform(np.log(Lmin), np.log(Lmax), R))
    Ls = np.clip(np.rint(Ls), Lmin, Lmax).astype(np.uint32)
    rho_r = np.exp(g.uniform(np.log(rmin), np.log(rmax), R))
    rho = np.repeat(rho_r, Ls)
    u = np.concatenate([amp * np.sin(2.0 * np.pi * np.arange(l) / l) for l in Ls])
    return Workload("uneven", Ls, rho, u, steps, seed, meta={"rho_r": rho_r})


def fluct(R: int = 512, L: int = 4096, rho: float = 50.0, u: float = 0.0, steps: int = 10_000,
          burn_in: int = 1000, seed: int = 1) -> Workload:
    Ls = np.full(R, L, dtype=np.uint32)
    r, v = _uniform_profiles(Ls, np.full(R, rho), np.full(R, u))
    return Workload("fluct", Ls, r, v, steps, seed, burn_in=burn_in, meta={"rho": rho, "u": u})


def random_state(L, mean: float, seed: int, dtype=np.uint16) -> np.ndarray:
    """A seeded occupation field n[3, sum L] with independent Poisson(mean) entries.

    Used for parity tests that start from a given state instead of mclg_init."""
    S = int(np.asarray(L).sum())
    g = np.random.default_rng(seed)
    return g.poisson(mean, size=(3, S)).astype(dtype)


BY_NAME = {"small": small, "single": single, "batched": batched, "uneven": uneven,
           "fluct": fluct}
