"""One lattice split into blocks (MCLG_HALO handles with node_offset), one
value exchanged across each cut per step through mclg_halo_get / mclg_halo_put:
the blocks together reproduce the undecomposed lattice and the oracle bit for
bit, for both samplers and every launch variant, with host or device buffers."""
import numpy as np
import pytest

import oracle
from paper_1706_01094_gb300 import sharding, workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_01094_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1706_01094_gb300 import mclg  # noqa: E402

SEQ, SLICE = mclg.SAMPLER_SEQUENTIAL, mclg.SAMPLER_SLICE


def reference(L, seed, n0, t0, steps, sampler, n_max=oracle.SLICE_N_MAX):
    if sampler == SLICE:
        want, err = oracle.slice_step([L], seed, n0, t0, steps, n_max=n_max)
    else:
        want, err = oracle.step([L], seed, n0, t0, steps)
    assert err == 0
    return want


def run_blocks(L, cuts, seed, n0, t0, steps, sampler, device=False, **kw):
    """Step the blocks [cuts[k], cuts[k+1]) with a crossed exchange after every step."""
    lats = [mclg.Lattice([e - b], seed=seed, sampler=sampler, node_offset=b, **kw)
            for b, e in zip(cuts[:-1], cuts[1:])]
    try:
        for lat, b, e in zip(lats, cuts[:-1], cuts[1:]):
            lat.set_state(np.ascontiguousarray(n0[:, b:e]), t=t0)
        k = len(lats)
        for _ in range(steps):
            for lat in lats:
                lat.step(1)
            if device:
                outs = [lat.halo_get(torch.empty(2, dtype=torch.int16, device="cuda"))
                        for lat in lats]
                torch.cuda.synchronize()
                for i, lat in enumerate(lats):
                    lat.halo_put(torch.stack([outs[(i - 1) % k][1], outs[(i + 1) % k][0]]))
                    torch.cuda.synchronize()
            else:
                outs = [lat.halo_get() for lat in lats]
                for i, lat in enumerate(lats):
                    lat.halo_put([outs[(i - 1) % k][1], outs[(i + 1) % k][0]])
        got = np.concatenate([lat.get_state()[0] for lat in lats], axis=1)
        assert all(lat.t == t0 + steps for lat in lats)
        return got
    finally:
        for lat in lats:
            lat.close()


@pytest.mark.parametrize("sampler", [SEQ, SLICE])
def test_one_block_with_crossed_exchange_is_the_periodic_lattice(sampler):
    L = 1000
    n0 = workloads.random_state([L], 30.0, seed=1)
    want = reference(L, 4, n0, 3, 9, sampler)
    assert np.array_equal(run_blocks(L, [0, L], 4, n0, 3, 9, sampler), want)


@pytest.mark.parametrize("sampler,variant", [(SEQ, None), (SEQ, 1), (SEQ, 3), (SLICE, None),
                                             (SLICE, 0), (SLICE, 2), (SLICE, 5), (SLICE, 6),
                                             (SLICE, 9), (SLICE, 10), (SLICE, 13), (SLICE, 15)])
def test_blocks_reproduce_the_lattice(sampler, variant):
    """Four uneven blocks (one of 8 nodes, the last of 3, lengths not all
    multiples of 8), every launch shape of the per-step kernels."""
    L = 5003
    cuts = [0, 1200, 1208, 5000, L]
    n0 = workloads.random_state([L], 33.0, seed=7)
    want = reference(L, 11, n0, 20, 13, sampler)
    got = run_blocks(L, cuts, 11, n0, 20, 13, sampler, kernel_variant=variant)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("sampler", [SEQ, SLICE])
def test_device_buffers_and_a_long_lattice(sampler):
    """Halo values exchanged in device memory, blocks of a lattice of 2^20 + 6
    nodes (many tiles per block, heavier nodes past the tables' range), against
    the same lattice stepped as one periodic handle."""
    L = (1 << 20) + 6
    cuts = list(sharding.blocks(L, 3)[k][0] for k in range(3)) + [L]
    n0 = workloads.random_state([L], 40.0, seed=9)
    with mclg.Lattice([L], seed=2, sampler=sampler, slice_n_max=120) as lat:
        lat.set_state(n0, t=0)
        lat.step(6)
        whole, _ = lat.get_state()
    got = run_blocks(L, cuts, 2, n0, 0, 6, sampler, device=True, slice_n_max=120)
    assert np.array_equal(got, whole)
    assert np.array_equal(got, reference(L, 2, n0, 0, 6, sampler, n_max=120))


def test_init_of_blocks_equals_the_lattice_init():
    """mclg_init draws with the global node index: blocks initialised from their
    slices of the density and velocity profiles hold the lattice's initial field,
    and their moments include the arriving edge values."""
    wl = workloads.single(L=1 << 16)
    L = int(wl.L[0])
    n0, err = oracle.init(wl.L, wl.seed, wl.rho, wl.u)
    assert err == 0
    parts = []
    for b, e in sharding.blocks(L, 3):
        with mclg.Lattice([e - b], seed=wl.seed, node_offset=b) as lat:
            lat.init(wl.rho[b:e], wl.u[b:e])
            st, _ = lat.get_state()
            N, J, tot = lat.moments()
            assert np.array_equal(N, st.astype(np.int64).sum(axis=0))
            assert np.array_equal(J, st[2].astype(np.int64) - st[0])
            parts.append(st)
    assert np.array_equal(np.concatenate(parts, axis=1), n0)


def test_halo_arguments_and_order_of_calls():
    L = [100]
    with pytest.raises(mclg.MCLGError):          # one replica only
        mclg.Lattice([50, 50], node_offset=0)
    with pytest.raises(mclg.MCLGError):          # no statistics on a block
        mclg.Lattice(L, node_offset=0, flags=mclg.STATS)
    with pytest.raises(mclg.MCLGError):          # not the persistent mode
        mclg.Lattice(L, node_offset=0, mode=mclg.MODE_PERSISTENT)
    with pytest.raises(mclg.MCLGError):          # slice sampler: blocks start on multiples of 8
        mclg.Lattice(L, node_offset=12, sampler=SLICE)
    with pytest.raises(mclg.MCLGError):          # global indices below 2^32
        mclg.Lattice(L, node_offset=2**32 - 50)
    lib = mclg.load()
    p = mclg.Params(10, 1, 1, 0, 0, 0, 0, 0, 0, 5)   # an offset without MCLG_HALO
    import ctypes
    h = ctypes.c_void_p()
    Lc = np.array(L, dtype=np.uint32)
    assert lib.mclg_create(Lc.ctypes.data_as(ctypes.c_void_p), 1, 1, ctypes.byref(p), None,
                           ctypes.byref(h)) == 1
    n0 = workloads.random_state(L, 10.0, seed=1)
    with mclg.Lattice(L, node_offset=7) as lat:
        lat.set_state(n0, t=0)
        with pytest.raises(mclg.MCLGError):      # nothing has left the block yet
            lat.halo_get()
        with pytest.raises(mclg.MCLGError):      # one step per call
            lat.step(2)
        lat.step(1)
        with pytest.raises(mclg.MCLGError):      # the arriving values are missing
            lat.step(1)
        with pytest.raises(mclg.MCLGError):
            lat.get_state()
        out = lat.halo_get()
        lat.halo_put([out[1], out[0]])
        lat.step(1)
        out = lat.halo_get()
        lat.halo_put([out[1], out[0]])
        got, t = lat.get_state()
    assert t == 2
    # the same 100 nodes as a block at nodes 7 .. 106 of a lattice, ring closed on itself
    blk = oracle.Block(n0, 7, 1)
    for tt in range(2):
        o, _ = blk.collide(tt)
        blk.stream([o[1], o[0]])
    assert np.array_equal(got, blk.n)
    with mclg.Lattice(L) as lat:                 # a periodic handle has no halo
        lat.set_state(n0)
        lat.step(1)
        with pytest.raises(mclg.MCLGError):
            lat.halo_get()
