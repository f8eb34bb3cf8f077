"""Plain CPU oracle for the D1Q3 Monte Carlo Lattice Gas (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_1706_01094_gb300`` never imports it, and this package never imports
the library: the two share nothing but the seeded workload generators.

``mclg_oracle.c`` holds the slow, plain reference (Philox4x32-10, the exact
sub-collision sampler, streaming, Poisson initialisation, moments, exact
statistics); this module builds it with gcc (OpenMP over the nodes of a step,
which does not change any result) and wraps it with ctypes.
``exact.py`` holds rational-arithmetic tools (enumeration of the paper's
particle picks, stationary laws) used to pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mclg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERR_OVERFLOW = 1
ERR_SAMPLER = 2
FLAG_NO_STREAM = 1
FLAG_GALILEAN = 4


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
            lib.orc_philox.argtypes = [P, P, P]
            lib.orc_feq.argtypes = [ctypes.c_double, ctypes.c_double, P]
            lib.orc_poisson_inv.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.orc_poisson_inv.restype = u32
            lib.orc_init.argtypes = [P, u32, u64, P, P, P, u32]
            lib.orc_init.restype = i32
            lib.orc_decide.argtypes = [u64, u64, u64, u32, P, i32, P]
            lib.orc_decide.restype = i32
            for name in ("orc_step", "orc_literal_step"):
                fn = getattr(lib, name)
                fn.argtypes = [P, u32, u64, u32, u32, u32, u32, P, u64, u64, u32]
                fn.restype = i32
            lib.orc_slice_step.argtypes = [P, u32, u64, u32, u32, u32, u32, P, u64, u64, u32, u32]
            lib.orc_slice_step.restype = i32
            lib.orc_slice_cdf.argtypes = [u32, ctypes.c_int32, u32, u32, u32, u32, P, P, P]
            lib.orc_slice_cdf.restype = i32
            lib.orc_slice_draw.argtypes = [u32, ctypes.c_int32, u32, u64, u32, u32, u32]
            lib.orc_slice_draw.restype = ctypes.c_int64
            lib.orc_slice_q.argtypes = [u32, u32, u32, P]
            lib.orc_galilean_q.argtypes = [u32, ctypes.c_int32, u32, u32]
            lib.orc_galilean_q.restype = u32
            lib.orc_slice_q.restype = u64
            lib.orc_moments.argtypes = [P, u32, P, P, P, P]
            lib.orc_stats_accumulate.argtypes = [u32, u32, P, P, P, P, P]
            lib.orc_exact_cov.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, u64]
            lib.orc_exact_cov.restype = ctypes.c_double
            lib.orc_block_collide.argtypes = [u32, u32, u32, u64, u32, u32, u32, u32, u32, u32,
                                              P, P, u32, P]
            lib.orc_block_collide.restype = i32
            lib.orc_block_stream.argtypes = [u32, P, P, P]
            lib.orc_block_stream.restype = None
            lib.orc2_collision_count.restype = i32
            lib.orc2_collision.argtypes = [i32, P]
            lib.orc2_outcomes.argtypes = [i32, i32, P, u32, P, P]
            lib.orc2_outcomes.restype = i32
            lib.orc2_feq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, P]
            lib.orc2_init.argtypes = [u32, u32, u32, u64, P, P, P, P, u32]
            lib.orc2_init.restype = i32
            lib.orc2_step.argtypes = [u32, u32, u32, u64, u32, P, u32, u32, P, u64, u64, u32]
            lib.orc2_step.restype = i32
            lib.orc2_moments.argtypes = [u64, P, P, P, P, P]
            lib.orc_set_threads.argtypes = [i32]
            lib.orc_set_threads.restype = i32
            lib.orc_threads.argtypes = []
            lib.orc_threads.restype = i32
            _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's node loops (0: every core); returns the count in use.
    Results do not depend on it: every node writes only its own entries."""
    return int(_load().orc_set_threads(int(n)))


def threads() -> int:
    return int(_load().orc_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _lengths(L) -> np.ndarray:
    L = np.ascontiguousarray(np.asarray(L, dtype=np.uint32).reshape(-1))
    if L.size == 0 or (L == 0).any():
        raise ValueError("every replica needs at least one node")
    return L


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def feq(rho: float, u: float) -> np.ndarray:
    """Entropic D1Q3 equilibrium (f_-1, f_0, f_+1), Eq. D1Q3equil."""
    f = np.zeros(3, dtype=np.float64)
    _load().orc_feq(float(rho), float(u), _ptr(f))
    return f


def poisson_inv(mu: float, U: float) -> int:
    return int(_load().orc_poisson_inv(float(mu), float(U)))


def init(L, seed: int, rho, u, first_replica: int = 0) -> tuple[np.ndarray, int]:
    """n_i(x, 0) ~ Poisson(f_i^eq(rho(x), u(x))); returns (n[3, S] uint16, error bits)."""
    L = _lengths(L)
    S = int(L.sum())
    rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(-1))
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
    if rho.size != S or u.size != S:
        raise ValueError("rho and u need one value per node")
    n = np.zeros((3, S), dtype=np.uint16)
    err = _load().orc_init(_ptr(L), L.size, seed & (2**64 - 1), _ptr(rho), _ptr(u), _ptr(n),
                           first_replica)
    return n, int(err)


def decide(T1: int, T2: int, D: int, q0: int, refine=()) -> tuple[int, int]:
    """Region (0 down, 1 up, 2 nothing, -1 needs more chunks, -2 cap) and chunks used."""
    ref = np.ascontiguousarray(np.asarray(list(refine), dtype=np.uint16))
    if ref.size == 0:
        ref = np.zeros(1, dtype=np.uint16)
        nref = 0
    else:
        nref = ref.size
    used = ctypes.c_int(0)
    region = _load().orc_decide(T1, T2, D, q0, _ptr(ref), nref, ctypes.byref(used))
    return int(region), int(used.value)


def _run(fn_name, L, seed, n, t0, n_steps, C=10, lam=(1, 1), flags=0, first_replica=0,
         extra=()):
    L = _lengths(L)
    S = int(L.sum())
    n = np.array(n, dtype=np.uint16, copy=True).reshape(3, S)
    n = np.ascontiguousarray(n)
    fn = getattr(_load(), fn_name)
    err = fn(_ptr(L), L.size, seed & (2**64 - 1), C, lam[0], lam[1], flags, _ptr(n), t0, n_steps,
             first_replica, *extra)
    return n, int(err)


def step(L, seed, n, t0, n_steps, C=10, lam=(1, 1), flags=0, first_replica=0):
    """Contract-mode time steps (bit-exact reference).  Returns (n, error bits)."""
    return _run("orc_step", L, seed, n, t0, n_steps, C, lam, flags, first_replica)


def literal_step(L, seed, n, t0, n_steps, C=10, lam=(1, 1), flags=0, first_replica=0):
    """The paper's particle-pick algorithm with its own random stream (distribution reference)."""
    return _run("orc_literal_step", L, seed, n, t0, n_steps, C, lam, flags, first_replica)


SLICE_N_MAX = 256  # the slice sampler's default table range


def slice_step(L, seed, n, t0, n_steps, C=10, lam=(1, 1), flags=0, first_replica=0,
               n_max=SLICE_N_MAX):
    """Time steps with the slice sampler (the C sub-collisions of a node drawn at
    once from their exact joint law) for nodes of mass N <= n_max; heavier nodes
    take the sequential draws of ``step``.  Returns (n, error bits)."""
    return _run("orc_slice_step", L, seed, n, t0, n_steps, C, lam, flags, first_replica,
                extra=(n_max,))


def slice_cdf(N: int, J: int, b: int, C: int = 10, lam=(1, 1)):
    """(F, dmin, dmax): F[d + C] = floor(CDF[d] 2^64) (capped at 2^64 - 1) of the
    C-step law of the rest count from b on the (N, J) slice."""
    F = np.zeros(2 * C + 1, dtype=np.uint64)
    dmin, dmax = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = _load().orc_slice_cdf(N, J, b, C, lam[0], lam[1], _ptr(F), ctypes.byref(dmin),
                               ctypes.byref(dmax))
    if rc != 0:
        raise ValueError("C too large for the slice sampler")
    return F, int(dmin.value), int(dmax.value)


def galilean_q(N: int, J: int, lam=(1, 1)) -> int:
    """Numerator q of the node's Galilean-invariant collision rate q / 256."""
    return int(_load().orc_galilean_q(N, J, lam[0], lam[1]))


def slice_q(x: int, r: int, t: int, seed: int) -> int:
    """The slice sampler's 64-bit uniform prefix Q of node x of replica r at time t."""
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    return int(_load().orc_slice_q(x, r, t, _ptr(key)))


def slice_draw(N: int, J: int, b: int, Q: int, C: int = 10, lam=(1, 1)) -> int:
    """New rest count of one node from the 64-bit prefix Q of its uniform (-1: undecided)."""
    return int(_load().orc_slice_draw(N, J, b, Q, C, lam[0], lam[1]))


def moments(L, n):
    """Per-node N, J (int32) and exact int64 totals (sum N, sum J)."""
    L = _lengths(L)
    S = int(L.sum())
    n = np.ascontiguousarray(np.asarray(n, dtype=np.uint16).reshape(3, S))
    N = np.zeros(S, dtype=np.int32)
    J = np.zeros(S, dtype=np.int32)
    tot = np.zeros(2, dtype=np.int64)
    _load().orc_moments(_ptr(L), L.size, _ptr(n), _ptr(N), _ptr(J), _ptr(tot))
    return N, J, tot


class Stats:
    """Exact int64 ensemble sums per node position, pooled over equal-length replicas."""

    def __init__(self, Lc: int, R: int):
        self.Lc, self.R = int(Lc), int(R)
        self.s1 = np.zeros((self.Lc, 3), dtype=np.int64)
        self.s2 = np.zeros((self.Lc, 6), dtype=np.int64)
        self.snb = np.zeros((self.Lc, 9), dtype=np.int64)
        self._count = np.zeros(1, dtype=np.uint64)

    @property
    def count(self) -> int:
        return int(self._count[0])

    def accumulate(self, n):
        n = np.ascontiguousarray(np.asarray(n, dtype=np.uint16).reshape(3, self.Lc * self.R))
        _load().orc_stats_accumulate(self.Lc, self.R, _ptr(n), _ptr(self.s1), _ptr(self.s2),
                                     _ptr(self.snb), _ptr(self._count))

    def cov(self, x: int, i: int, j: int) -> float:
        """Exact covariance of n_i(x), n_j(x) from the int64 sums (FP64 only at the end)."""
        pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        p = pairs.index((min(i, j), max(i, j)))
        return float(_load().orc_exact_cov(int(self.s2[x, p]), int(self.s1[x, i]),
                                           int(self.s1[x, j]), self.count))


class Block:
    """One block of a periodic lattice, global nodes [x0, x0 + len(n)), for a
    decomposition over ranks: collide() returns the two values that leave the
    block, stream(in) takes the two that arrive (see orc_block_collide)."""

    def __init__(self, n, x0: int, seed: int, C: int = 10, lam=(1, 1), flags: int = 0,
                 replica: int = 0, sampler: str = "sequential", n_max: int = SLICE_N_MAX):
        self.n = np.ascontiguousarray(np.asarray(n, dtype=np.uint16).reshape(3, -1)).copy()
        self.Lb = int(self.n.shape[1])
        self.x0, self.seed, self.C, self.lam, self.flags = int(x0), int(seed), int(C), lam, flags
        self.replica = int(replica)
        self.sampler = 1 if sampler == "slice" else 0
        self.n_max = int(n_max)
        self.post = np.zeros_like(self.n)

    def collide(self, t: int) -> tuple[np.ndarray, int]:
        out = np.zeros(2, dtype=np.uint16)
        err = _load().orc_block_collide(self.Lb, self.x0, self.replica, self.seed & (2**64 - 1),
                                        self.C, self.lam[0], self.lam[1], self.flags, self.sampler,
                                        self.n_max, _ptr(self.n), _ptr(self.post), t, _ptr(out))
        return out, int(err)

    def stream(self, incoming) -> None:
        inc = np.ascontiguousarray(np.asarray(incoming, dtype=np.uint16).reshape(2))
        _load().orc_block_stream(self.Lb, _ptr(self.post), _ptr(inc), _ptr(self.n))


# ---------------------------------------------------------------------- D2Q9 ---
# Velocities 0 = (0,0), 1 = (1,0), 2 = (0,1), 3 = (-1,0), 4 = (0,-1), 5 = (1,1),
# 6 = (-1,1), 7 = (-1,-1), 8 = (1,-1); rates lambda_1 .. lambda_9 numbered as in
# Eq. D2Q9MOmega.  The paper's simulation rates (Sec. IV.B): 15/128, 1/4 (x6),
# 1/8, 18/144.
D2Q9_VX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
D2Q9_VY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
D2Q9_PAPER_LAMBDA = ((15, 32, 32, 32, 32, 32, 32, 16, 16), 128)


def _lam2(lam):
    num = np.ascontiguousarray(np.asarray(lam[0], dtype=np.uint32).reshape(9))
    return num, int(lam[1])


def d2q9_collisions():
    """The 30 binary collisions [(pair A, pair B, class)] of the oracle's table."""
    lib = _load()
    out = []
    buf = np.zeros(5, dtype=np.int32)
    for k in range(lib.orc2_collision_count()):
        lib.orc2_collision(k, _ptr(buf))
        out.append(((int(buf[0]), int(buf[1])), (int(buf[2]), int(buf[3])), int(buf[4])))
    return out


def d2q9_outcomes(s1: int, s2: int, lam=D2Q9_PAPER_LAMBDA):
    """[(target pair, numerator)] of a pick of velocities (s1, s2); numerators over
    128 * lambda_den."""
    num, den = _lam2(lam)
    targets = np.zeros(8, dtype=np.int32)
    nums = np.zeros(4, dtype=np.uint64)
    n = _load().orc2_outcomes(s1, s2, _ptr(num), den, _ptr(targets), _ptr(nums))
    return [((int(targets[2 * k]), int(targets[2 * k + 1])), int(nums[k])) for k in range(n)]


def d2q9_feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Entropic D2Q9 equilibrium of Eq. D2Q9eqdist."""
    f = np.zeros(9, dtype=np.float64)
    _load().orc2_feq(float(rho), float(ux), float(uy), _ptr(f))
    return f


def d2q9_init(Lx: int, Ly: int, R: int, seed: int, rho, ux, uy, first_replica: int = 0):
    S = Lx * Ly * R
    args = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1)) for a in (rho, ux, uy)]
    if any(a.size != S for a in args):
        raise ValueError("rho, ux, uy need one value per node")
    n = np.zeros((9, S), dtype=np.uint16)
    err = _load().orc2_init(Lx, Ly, R, seed & (2**64 - 1), *[_ptr(a) for a in args], _ptr(n),
                            first_replica)
    return n, int(err)


def d2q9_step(Lx: int, Ly: int, R: int, seed: int, n, t0: int, n_steps: int, C: int = 10,
              lam=D2Q9_PAPER_LAMBDA, flags: int = 0, first_replica: int = 0):
    """D2Q9 time steps (the paper's particle-pick algorithm with exact integer
    draws); n is [9, R Lx Ly].  Returns (n, error bits)."""
    S = Lx * Ly * R
    n = np.ascontiguousarray(np.array(n, dtype=np.uint16, copy=True).reshape(9, S))
    num, den = _lam2(lam)
    err = _load().orc2_step(Lx, Ly, R, seed & (2**64 - 1), C, _ptr(num), den, flags, _ptr(n), t0,
                            n_steps, first_replica)
    return n, int(err)


def d2q9_moments(n):
    n = np.ascontiguousarray(np.asarray(n, dtype=np.uint16))
    S = n.shape[1]
    rho, jx, jy = (np.zeros(S, dtype=np.int32) for _ in range(3))
    tot = np.zeros(3, dtype=np.int64)
    _load().orc2_moments(S, _ptr(n), _ptr(rho), _ptr(jx), _ptr(jy), _ptr(tot))
    return rho, jx, jy, tot
