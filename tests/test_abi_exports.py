"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/mclg.h declares; the binding fails loudly without it."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mclg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mclg(?:2d)?_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1706_01094_gb300 import build
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mclg_create", "mclg_init", "mclg_step", "mclg_moments", "mclg_destroy",
                     "mclg_set_state", "mclg_get_state", "mclg_stats_read", "mclg_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True)
    if out.returncode == 0:
        exported = set(re.findall(r"\bT (mclg(?:2d)?_[a-z0-9_]+)", out.stdout))
        assert set(declared_functions()) <= exported


def test_binding_names_match_header():
    from paper_1706_01094_gb300 import mclg
    assert sorted(mclg.EXPORTS) == declared_functions()


def test_status_strings_and_defaults_without_gpu(libpath):
    from paper_1706_01094_gb300 import mclg
    lib = mclg.load()
    assert lib.mclg_status_str(0) == b"ok"
    assert lib.mclg_status_str(4).startswith(b"occupation overflow")
    p = mclg.Params()
    lib.mclg_default_params(ctypes.byref(p))
    assert (p.C, p.lambda_num, p.lambda_den, p.flags, p.mode) == (10, 1, 1, 0, 0)
    h = ctypes.c_void_p()
    # argument validation happens before any CUDA call
    assert lib.mclg_create(None, 0, 1, None, None, ctypes.byref(h)) == 1
    L = (ctypes.c_uint32 * 1)(0)
    assert lib.mclg_create(L, 1, 1, None, None, ctypes.byref(h)) == 1
    lib.mclg_destroy(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1706_01094_gb300 import mclg
    monkeypatch.setattr(mclg, "_lib", None)
    monkeypatch.setattr(mclg, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        mclg.Lattice([8])


def test_noalloc_binding_refuses_bad_buffers_before_the_library():
    """Shapes and dtypes that would let mclg_moments_noalloc run past a buffer are
    refused on the host (no device buffers, no launch)."""
    import numpy as np
    from paper_1706_01094_gb300 import mclg
    n = np.zeros((3, 10), dtype=np.uint16)
    good_N = np.zeros(10, dtype=np.int32)
    tot = np.zeros(2, dtype=np.int64)
    bad = [
        dict(n=np.zeros((4, 10), dtype=np.uint16)),           # not three planes
        dict(n=np.zeros(31, dtype=np.uint16)),                # length not a multiple of 3
        dict(n=np.zeros((3, 10), dtype=np.int32)),            # not 16-bit
        dict(n=n, N=np.zeros(9, dtype=np.int32)),             # N shorter than S
        dict(n=n, J=np.zeros(10, dtype=np.int64)),            # J not int32
        dict(n=n, N=good_N, totals=np.zeros(1, dtype=np.int64)),   # one total slot
        dict(n=n, totals=np.zeros(2, dtype=np.int32)),        # totals not int64
    ]
    for kw in bad:
        with pytest.raises(ValueError):
            mclg.moments_noalloc(**kw)


def test_noalloc_size_limit_is_checked_first(libpath):
    """Sizes beyond the fixed scratch are rejected before any CUDA call."""
    from paper_1706_01094_gb300 import mclg
    lib = mclg.load()
    buf = ctypes.create_string_buffer(64)
    assert lib.mclg_moments_noalloc(buf, (1 << 26) + 1, None, None, None, None) == 1
    assert lib.mclg_moments_noalloc(buf, 0, None, None, None, None) == 1
    assert lib.mclg_moments_noalloc(None, 8, None, None, None, None) == 1
