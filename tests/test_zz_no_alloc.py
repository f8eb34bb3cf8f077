"""The allocation-free moments entry point against mclg_moments.

mclg_moments_noalloc serves callers that cannot allocate device memory (their
GPU memory is owned by another pool, or they cannot accept the device-wide
synchronisation of cudaMalloc/cudaFree): they pass their own buffers and the
library uses only a fixed scratch array.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1706_01094_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_01094_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1706_01094_gb300 import mclg  # noqa: E402


def _existing(lat):
    """The existing entry point's results, with device N, J."""
    N = torch.empty(lat.S, dtype=torch.int32, device="cuda")
    J = torch.empty(lat.S, dtype=torch.int32, device="cuda")
    _, _, tot = lat.moments(N, J)
    return N.cpu().numpy(), J.cpu().numpy(), tot


def _noalloc(n_dev, S):
    N = torch.full((S,), -7, dtype=torch.int32, device="cuda")
    J = torch.full((S,), -7, dtype=torch.int32, device="cuda")
    tot = np.zeros(2, dtype=np.int64)
    status = mclg.moments_noalloc(n_dev, N, J, tot)
    assert status == mclg.MCLG_OK, mclg.STATUS.get(status)
    return N.cpu().numpy(), J.cpu().numpy(), tot


def test_noalloc_moments_match_existing_entry_point_twice():
    # several thousand blocks of partial sums, a ragged last block, two
    # different states so that stale scratch contents would show
    L = [70000, 13, 4099]
    S = sum(L)
    with mclg.Lattice(L, seed=21) as lat:
        lat.set_state(workloads.random_state(L, 40.0, seed=5), t=0)
        for call in range(2):
            lat.step(3 + call)
            n_dev = torch.empty((3, S), dtype=torch.int16, device="cuda")
            lat.get_state(n_dev)
            want = _existing(lat)
            got = _noalloc(n_dev, S)
            for w, g in zip(want, got):
                assert np.array_equal(w, g), f"call {call}"
        # a smaller field after a larger one: the final sums must not see old partials
        small = n_dev[:, :1000].contiguous()
        N, J, tot = _noalloc(small, 1000)
        host = small.cpu().numpy().view(np.uint16).astype(np.int64)
        assert tot[0] == host.sum() and tot[1] == (host[2] - host[0]).sum()
        assert np.array_equal(N, host.sum(axis=0)) and np.array_equal(J, host[2] - host[0])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = mclg.load()
    n_dev = torch.zeros((3, 8), dtype=torch.int16, device="cuda")
    tot = np.zeros(2, dtype=np.int64)
    status = lib.mclg_moments_noalloc(ctypes.c_void_p(n_dev.data_ptr()), (1 << 26) + 1, None,
                                      None, tot.ctypes.data_as(ctypes.c_void_p), None)
    assert status == 1  # MCLG_ERR_ARG, before any device work
    host = np.zeros((3, 8), dtype=np.uint16)
    assert mclg.moments_noalloc(host, None, None, tot) == 1  # host input is rejected
