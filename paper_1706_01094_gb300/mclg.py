"""Python binding of the C ABI in ``include/mclg.h`` (argument marshalling only).

Every step of the lattice-gas path runs in the sm_103a library
``_build/libmclg.so``; this module loads it with ctypes and converts numpy
arrays or torch tensors to pointers.  If the library has not been built, every
call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MCLG_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA runtime error",
          4: "occupation overflow", 5: "device wait timed out", 6: "no state set",
          7: "sampler could not decide"}
NO_STREAM = 1
STATS = 2
GALILEAN = 4
HALO = 8
MODE_AUTO, MODE_PLAIN, MODE_PERSISTENT, MODE_BATCHED = 0, 1, 2, 3
SAMPLER_SEQUENTIAL, SAMPLER_SLICE = 0, 1

EXPORTS = ["mclg_default_params", "mclg_create", "mclg_init", "mclg_set_state",
           "mclg_get_state", "mclg_step", "mclg_moments", "mclg_stats_reset", "mclg_stats_read",
           "mclg_sync", "mclg_time", "mclg_destroy", "mclg_status_str", "mclg_philox",
           "mclg_moments_noalloc", "mclg_tuning", "mclg_slice_row", "mclg_halo_get",
           "mclg_halo_put", "mclg2d_default_params", "mclg2d_create", "mclg2d_init",
           "mclg2d_set_state", "mclg2d_get_state", "mclg2d_step", "mclg2d_moments",
           "mclg2d_sync", "mclg2d_time", "mclg2d_destroy", "mclg2d_pair_outcomes"]


class MCLGError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, 'unknown')} (status {status})")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("C", ctypes.c_uint32), ("lambda_num", ctypes.c_uint32),
                ("lambda_den", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("mode", ctypes.c_uint32), ("first_replica", ctypes.c_uint32),
                ("sampler", ctypes.c_uint32), ("slice_n_max", ctypes.c_uint32),
                ("kernel_variant", ctypes.c_uint32), ("node_offset", ctypes.c_uint32)]


class Params2D(ctypes.Structure):
    _fields_ = [("C", ctypes.c_uint32), ("lambda_num", ctypes.c_uint32 * 9),
                ("lambda_den", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("first_replica", ctypes.c_uint32)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load the built library; raises if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libmclg.so is not built ({path}); run "
                               "paper_1706_01094_gb300.build.build() first")
        lib = ctypes.CDLL(path)
        P, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        st = ctypes.c_int
        lib.mclg_default_params.argtypes = [ctypes.POINTER(Params)]
        lib.mclg_create.argtypes = [P, u32, u64, ctypes.POINTER(Params), P, ctypes.POINTER(P)]
        lib.mclg_create.restype = st
        lib.mclg_init.argtypes = [P, P, P]
        lib.mclg_init.restype = st
        lib.mclg_set_state.argtypes = [P, P, u64]
        lib.mclg_set_state.restype = st
        lib.mclg_get_state.argtypes = [P, P, ctypes.POINTER(u64)]
        lib.mclg_get_state.restype = st
        lib.mclg_step.argtypes = [P, u64]
        lib.mclg_step.restype = st
        lib.mclg_moments.argtypes = [P, P, P, P]
        lib.mclg_moments.restype = st
        lib.mclg_stats_reset.argtypes = [P]
        lib.mclg_stats_reset.restype = st
        lib.mclg_stats_read.argtypes = [P, P, P, P, P, P, P]
        lib.mclg_stats_read.restype = st
        lib.mclg_sync.argtypes = [P]
        lib.mclg_sync.restype = st
        lib.mclg_time.argtypes = [P]
        lib.mclg_time.restype = u64
        lib.mclg_destroy.argtypes = [P]
        lib.mclg_destroy.restype = None
        lib.mclg_status_str.argtypes = [st]
        lib.mclg_status_str.restype = ctypes.c_char_p
        lib.mclg_philox.argtypes = [P, u64, u64, P, P]
        lib.mclg_philox.restype = st
        lib.mclg_slice_row.argtypes = [u32, ctypes.c_int32, u32, u32, u32, u32, P, P, P, P]
        lib.mclg_slice_row.restype = st
        lib.mclg_tuning.argtypes = [P, P]
        lib.mclg_tuning.restype = st
        lib.mclg_moments_noalloc.argtypes = [P, u64, P, P, P, P]
        lib.mclg_moments_noalloc.restype = st
        lib.mclg_halo_get.argtypes = [P, P]
        lib.mclg_halo_get.restype = st
        lib.mclg_halo_put.argtypes = [P, P]
        lib.mclg_halo_put.restype = st
        lib.mclg2d_default_params.argtypes = [ctypes.POINTER(Params2D)]
        lib.mclg2d_create.argtypes = [u32, u32, u32, u64, ctypes.POINTER(Params2D), P,
                                      ctypes.POINTER(P)]
        lib.mclg2d_create.restype = st
        lib.mclg2d_init.argtypes = [P, P, P, P]
        lib.mclg2d_init.restype = st
        lib.mclg2d_set_state.argtypes = [P, P, u64]
        lib.mclg2d_set_state.restype = st
        lib.mclg2d_get_state.argtypes = [P, P, ctypes.POINTER(u64)]
        lib.mclg2d_get_state.restype = st
        lib.mclg2d_step.argtypes = [P, u64]
        lib.mclg2d_step.restype = st
        lib.mclg2d_moments.argtypes = [P, P, P, P, P]
        lib.mclg2d_moments.restype = st
        lib.mclg2d_sync.argtypes = [P]
        lib.mclg2d_sync.restype = st
        lib.mclg2d_time.argtypes = [P]
        lib.mclg2d_time.restype = u64
        lib.mclg2d_destroy.argtypes = [P]
        lib.mclg2d_destroy.restype = None
        lib.mclg2d_pair_outcomes.argtypes = [u32, u32, ctypes.POINTER(Params2D), P, P, P]
        lib.mclg2d_pair_outcomes.restype = st
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != MCLG_OK:
        raise MCLGError(status, where)


def _ptr(a):
    """Pointer of a contiguous numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Lattice:
    """A handle: `replicas` independent periodic D1Q3 lattices of lengths L, or
    (``node_offset`` given) one block of a larger periodic lattice whose edges
    exchange values with the neighbouring blocks (halo_get / halo_put)."""

    def __init__(self, L, seed: int = 1, C: int = 10, lam=(1, 1), flags: int = 0,
                 mode: int = MODE_AUTO, stream=None, first_replica: int = 0,
                 sampler: int = SAMPLER_SEQUENTIAL, slice_n_max: int = 0,
                 kernel_variant=None, node_offset=None):
        self._lib = load()
        self.L = np.ascontiguousarray(np.asarray(L, dtype=np.uint32).reshape(-1))
        self.S = int(self.L.sum())
        self.seed = int(seed)
        kv = 0 if kernel_variant is None else int(kernel_variant) + 1  # None: autotune
        if node_offset is not None:
            flags |= HALO
        p = Params(C, lam[0], lam[1], flags, mode, first_replica, sampler, slice_n_max, kv,
                   0 if node_offset is None else int(node_offset))
        h = ctypes.c_void_p()
        _check(self._lib.mclg_create(_ptr(self.L), self.L.size, self.seed & (2**64 - 1),
                                     ctypes.byref(p), _stream_ptr(stream), ctypes.byref(h)),
               "mclg_create")
        self._h = h
        self.flags = flags

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.mclg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state ---------------------------------------------------------------
    def init(self, rho, u):
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(-1))
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
        if rho.size != self.S or u.size != self.S:
            raise ValueError("rho and u need one value per node")
        _check(self._lib.mclg_init(self._h, _ptr(rho), _ptr(u)), "mclg_init")

    def set_state(self, n, t: int = 0):
        if isinstance(n, np.ndarray):
            n = np.ascontiguousarray(n, dtype=np.uint16)
        if tuple(n.shape) not in ((3, self.S), (3 * self.S,)):
            raise ValueError("state must be [3, S]")
        _check(self._lib.mclg_set_state(self._h, _ptr(n), t), "mclg_set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((3, self.S), dtype=np.uint16)
        t = ctypes.c_uint64(0)
        _check(self._lib.mclg_get_state(self._h, _ptr(out), ctypes.byref(t)), "mclg_get_state")
        return out, int(t.value)

    def step(self, n_steps: int = 1):
        _check(self._lib.mclg_step(self._h, n_steps), "mclg_step")

    def sync(self):
        _check(self._lib.mclg_sync(self._h), "mclg_sync")

    # -- a block of a larger lattice -------------------------------------------
    def halo_get(self, out=None):
        """The two post-collision values leaving the block after the last step:
        (v = -1 of the first node, v = +1 of the last node)."""
        if out is None:
            out = np.zeros(2, dtype=np.uint16)
        _check(self._lib.mclg_halo_get(self._h, _ptr(out)), "mclg_halo_get")
        return out

    def halo_put(self, values):
        """The two values arriving for the next step: (v = +1 into the first node,
        from the left neighbour; v = -1 into the last node, from the right one)."""
        if isinstance(values, np.ndarray) or not hasattr(values, "data_ptr"):
            values = np.ascontiguousarray(np.asarray(values, dtype=np.uint16).reshape(2))
        _check(self._lib.mclg_halo_put(self._h, _ptr(values)), "mclg_halo_put")

    def sync_status(self) -> int:
        return int(self._lib.mclg_sync(self._h))

    def tuning(self) -> dict:
        cfg = np.zeros(6, dtype=np.uint32)
        _check(self._lib.mclg_tuning(self._h, _ptr(cfg)), "mclg_tuning")
        return {"plain_nodes_per_thread": int(cfg[0]) // 100, "plain_variant": int(cfg[0]) % 100,
                "persistent_threads": int(cfg[1]), "persistent_unit_nodes": int(cfg[2]),
                "persistent_units": int(cfg[3]), "persistent_variant": int(cfg[4]),
                "stats_config": int(cfg[5])}

    @property
    def t(self) -> int:
        return int(self._lib.mclg_time(self._h))

    def moments(self, N=None, J=None):
        if N is None:
            N = np.zeros(self.S, dtype=np.int32)
        if J is None:
            J = np.zeros(self.S, dtype=np.int32)
        tot = np.zeros(2, dtype=np.int64)
        _check(self._lib.mclg_moments(self._h, _ptr(N), _ptr(J), _ptr(tot)), "mclg_moments")
        return N, J, tot

    def totals(self):
        tot = np.zeros(2, dtype=np.int64)
        _check(self._lib.mclg_moments(self._h, None, None, _ptr(tot)), "mclg_moments")
        return tot

    # -- statistics ------------------------------------------------------------
    def stats_reset(self):
        _check(self._lib.mclg_stats_reset(self._h), "mclg_stats_reset")

    def stats_read(self):
        Lc = int(self.L[0])
        s1 = np.zeros((Lc, 3), dtype=np.int64)
        s2 = np.zeros((Lc, 6), dtype=np.int64)
        snb = np.zeros((Lc, 9), dtype=np.int64)
        cov32 = np.zeros((Lc, 6), dtype=np.float32)
        cov64 = np.zeros((Lc, 6), dtype=np.float64)
        cnt = np.zeros(1, dtype=np.uint64)
        _check(self._lib.mclg_stats_read(self._h, _ptr(s1), _ptr(s2), _ptr(snb), _ptr(cov32),
                                         _ptr(cov64), _ptr(cnt)), "mclg_stats_read")
        return {"s1": s1, "s2": s2, "snb": snb, "cov32": cov32, "cov64": cov64,
                "count": int(cnt[0])}


def _numel(a) -> int:
    return int(a.numel()) if hasattr(a, "numel") else int(np.asarray(a).size)


def _dtype_name(a) -> str:
    return str(a.dtype).replace("torch.", "")


def moments_noalloc(n, N=None, J=None, totals=None, stream=None) -> int:
    """mclg_moments_noalloc on a device field n[3, S] (caller-owned buffers).

    For callers that cannot allocate device memory; returns the raw status.
    Shapes and dtypes are checked here (ValueError) so that the library never
    reads or writes past a buffer: n is [3, S] or [3 S] of a 16-bit integer
    type, N and J int32 with at least S entries, totals int64 with at least 2."""
    shape = tuple(n.shape)
    if len(shape) == 2 and shape[0] == 3:
        S = int(shape[1])
    elif len(shape) == 1 and shape[0] % 3 == 0:
        S = int(shape[0]) // 3
    else:
        raise ValueError(f"n must be [3, S] or [3 S], got shape {shape}")
    if _dtype_name(n) not in ("uint16", "int16"):
        raise ValueError(f"n must hold 16-bit occupations, got {n.dtype}")
    for name, a in (("N", N), ("J", J)):
        if a is None:
            continue
        if _dtype_name(a) != "int32" or _numel(a) < S:
            raise ValueError(f"{name} must be int32 with at least {S} entries")
    if totals is not None and (_dtype_name(totals) != "int64" or _numel(totals) < 2):
        raise ValueError("totals must be int64 with at least 2 entries")
    lib = load()
    return int(lib.mclg_moments_noalloc(_ptr(n), S, _ptr(N), _ptr(J), _ptr(totals),
                                        _stream_ptr(stream)))


def slice_row(N: int, J: int, b: int, C: int = 10, lam=(1, 1), record: bool = False):
    """The library's slice-sampler table row (host computation): (F, dmin, dmax),
    and the state's 8-lane record (uint16) as a fourth item when ``record``."""
    lib = load()
    F = np.zeros(2 * max(C, 1), dtype=np.uint64)
    R = np.zeros(8, dtype=np.uint16)
    dmin, dmax = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib.mclg_slice_row(N, J, b, C, lam[0], lam[1], _ptr(F), ctypes.byref(dmin),
                              ctypes.byref(dmax), _ptr(R) if record else None), "mclg_slice_row")
    out = (F[: dmax.value - dmin.value], int(dmin.value), int(dmax.value))
    return out + (R,) if record else out


def philox(ctr, seed: int, out=None, stream=None):
    """The library's device Philox4x32-10 on device uint32 counters ctr[n, 4]."""
    lib = load()
    n = int(ctr.shape[0])
    if out is None:
        import torch
        out = torch.empty_like(ctr)
    _check(lib.mclg_philox(_ptr(ctr), n, seed & (2**64 - 1), _ptr(out), _stream_ptr(stream)),
           "mclg_philox")
    return out


# ---------------------------------------------------------------------- D2Q9 ---
D2Q9_PAPER_LAMBDA = ((15, 32, 32, 32, 32, 32, 32, 16, 16), 128)  # Sec. IV.B's rates


def params2d(C: int = 10, lam=D2Q9_PAPER_LAMBDA, flags: int = 0, first_replica: int = 0):
    p = Params2D()
    p.C = C
    for k in range(9):
        p.lambda_num[k] = int(lam[0][k])
    p.lambda_den = int(lam[1])
    p.flags = flags
    p.first_replica = first_replica
    return p


def pair_outcomes2d(s1: int, s2: int, lam=D2Q9_PAPER_LAMBDA):
    """The library's outcome list of a pick of velocities (s1, s2): [(target pair,
    numerator over 128 lambda_den)] (host computation)."""
    lib = load()
    p = params2d(lam=lam)
    cnt = ctypes.c_uint32(0)
    tg = np.zeros(8, dtype=np.uint32)
    nums = np.zeros(4, dtype=np.uint64)
    _check(lib.mclg2d_pair_outcomes(s1, s2, ctypes.byref(p), ctypes.byref(cnt), _ptr(tg), _ptr(nums)),
           "mclg2d_pair_outcomes")
    return [((int(tg[2 * k]), int(tg[2 * k + 1])), int(nums[k])) for k in range(cnt.value)]


class Lattice2D:
    """A D2Q9 handle: `replicas` periodic Lx x Ly lattices (state n[9, R Lx Ly])."""

    def __init__(self, Lx: int, Ly: int, replicas: int = 1, seed: int = 1, C: int = 10,
                 lam=D2Q9_PAPER_LAMBDA, flags: int = 0, stream=None, first_replica: int = 0):
        self._lib = load()
        self.Lx, self.Ly, self.R = int(Lx), int(Ly), int(replicas)
        self.S = self.Lx * self.Ly * self.R
        p = params2d(C, lam, flags, first_replica)
        h = ctypes.c_void_p()
        _check(self._lib.mclg2d_create(self.Lx, self.Ly, self.R, int(seed) & (2**64 - 1),
                                       ctypes.byref(p), _stream_ptr(stream), ctypes.byref(h)),
               "mclg2d_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mclg2d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, rho, ux, uy):
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1)) for a in (rho, ux, uy)]
        if any(a.size != self.S for a in arrs):
            raise ValueError("rho, ux, uy need one value per node")
        _check(self._lib.mclg2d_init(self._h, *[_ptr(a) for a in arrs]), "mclg2d_init")

    def set_state(self, n, t: int = 0):
        if isinstance(n, np.ndarray):
            n = np.ascontiguousarray(n, dtype=np.uint16)
        if tuple(n.shape) not in ((9, self.S), (9 * self.S,)):
            raise ValueError("state must be [9, S]")
        _check(self._lib.mclg2d_set_state(self._h, _ptr(n), t), "mclg2d_set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((9, self.S), dtype=np.uint16)
        t = ctypes.c_uint64(0)
        _check(self._lib.mclg2d_get_state(self._h, _ptr(out), ctypes.byref(t)), "mclg2d_get_state")
        return out, int(t.value)

    def step(self, n_steps: int = 1):
        _check(self._lib.mclg2d_step(self._h, n_steps), "mclg2d_step")

    def sync(self):
        _check(self._lib.mclg2d_sync(self._h), "mclg2d_sync")

    @property
    def t(self) -> int:
        return int(self._lib.mclg2d_time(self._h))

    def moments(self, rho=None, jx=None, jy=None):
        """Per-node density and momentum into device int32 tensors (or None) and the
        exact totals (host)."""
        tot = np.zeros(3, dtype=np.int64)
        _check(self._lib.mclg2d_moments(self._h, _ptr(rho), _ptr(jx), _ptr(jy), _ptr(tot)),
               "mclg2d_moments")
        return tot
