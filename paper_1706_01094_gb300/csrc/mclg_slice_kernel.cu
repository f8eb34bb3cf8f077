// Slice-sampler time step (Sec. III with the C sub-collisions of a node drawn
// at once from their exact joint law, Sec. III.A).
//
// A node's C sub-collisions move it along its (N, J) slice: each one changes
// the rest count b by -2, 0 or +2 and keeps N and J.  The new rest count is
// b + 2 d with d drawn from the C-step law of the slice's birth-death chain,
// whose cumulative values F[k] = floor(CDF[dmin + k] 2^64) the host tables
// hold per state (N, |J|, b).  With the node's 64-bit uniform Q,
//     d = dmin + #{k : Q > F[k]}          (Q == F[k]: sampler error).
//
// One thread takes V consecutive nodes of a replica (V = 2, 4, 8: one 4-, 8-
// or 16-byte vector per plane; replicas start on multiples of 8 nodes, so a
// vector never straddles two).  Eight consecutive nodes take the top 16 bits
// of their uniforms Q from one Philox block.  The state's 16-byte record (the
// top 15 bits of the eight F values around d = 0) decides the draw from Q's
// top 15 bits unless d lies beyond +-3 or a prefix ties (about 0.2% of nodes
// near equilibrium); then the rest of Q is drawn and Q compared with the
// row's u64 entries (mclg_slice.cuh).  The records of the states a lattice
// near equilibrium visits take a few hundred kilobytes, so most lookups hit
// the SM's L1 cache.
//
// A node heavier than the tables' n_max takes the sequential sampler's C
// decisions (the bits that sampler gives it) in a second, small pass of the
// same step: the table kernel writes such a node unchanged and appends its
// position to a device list; k_step_heavy collides the listed nodes.  If the
// list overflows, the pass scans the whole range instead: collisions keep N,
// so exactly the heavy nodes have N > n_max after the table kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "mclg_device.cuh"
#include "mclg_internal.h"
#include "mclg_slice.cuh"

namespace mclg {

// The table draws of one thread's V consecutive nodes [x0, x0 + V) of a
// replica (nv of them valid, the rest padding that stays empty), from the
// streamed planes em, e0, ep (device form) and the two halo values: nxt =
// B_-1(x0 + V) and prv = B_+1(x0 - 1), periodic.  Writes the post-collision
// values; returns a bit per node left for the heavy-node pass.  One Philox
// block per node pair (slice_draws).
template <int V>
__device__ __forceinline__ uint32_t slice_vector(const uint32_t (&em)[V], const uint32_t (&e0)[V],
                                                 const uint32_t (&ep)[V], uint32_t nxt,
                                                 uint32_t prv, bool stream, uint32_t x0,
                                                 uint32_t nv, uint32_t r, uint32_t t,
                                                 const PlainArgs &p, const SliceTables &tab,
                                                 uint32_t (&om)[V], uint32_t (&o0)[V],
                                                 uint32_t (&op)[V], uint32_t &err)
{
    // pre-collision occupations n_i(x) = B_i(x - v_i); padding stays empty
#pragma unroll
    for (int j = 0; j < V; ++j) {
        if (stream) {
            om[j] = (uint32_t(j) + 1u < nv) ? em[(j + 1) % V] : nxt;
            op[j] = (j > 0) ? ep[(j + V - 1) % V] : prv;
        } else {
            om[j] = em[j];
            op[j] = ep[j];
        }
        o0[j] = e0[j];
        if (uint32_t(j) >= nv) om[j] = o0[j] = op[j] = 0u;
    }
    return slice_draws<V>(om, o0, op, x0, r, t, p.rk, p.k0, p.k1, tab, p.C, err);
}

// The same draws as slice_vector for a full or partial vector read from a
// shared-memory stage: `inputs_used` runs once the record loads, whose
// addresses depend on every input value (the halo values included), have been
// issued: by then the inputs have arrived in registers, so their stage can be
// handed back.
template <int V, typename InputsUsed>
__device__ __forceinline__ uint32_t slice_vector_phased(
    const uint32_t (&em)[V], const uint32_t (&e0)[V], const uint32_t (&ep)[V], uint32_t nxt,
    uint32_t prv, bool stream, uint32_t x0, uint32_t nv, uint32_t r, uint32_t t, const PlainArgs &p,
    const SliceTables &tab, uint32_t (&om)[V], uint32_t (&o0)[V], uint32_t (&op)[V], uint32_t &err,
    InputsUsed &&inputs_used)
{
    // pre-collision occupations n_i(x) = B_i(x - v_i), for a full vector ...
#pragma unroll
    for (int j = 0; j < V; ++j) {
        om[j] = stream ? (j + 1 < V ? em[j + 1] : nxt) : em[j];
        o0[j] = e0[j];
        op[j] = stream ? (j > 0 ? ep[j - 1] : prv) : ep[j];
    }
    // ... and at the end of a replica: the last node wraps around, padding stays empty
    if (nv < uint32_t(V)) {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            if (stream && uint32_t(j) + 1u == nv) om[j] = nxt;
            if (uint32_t(j) >= nv) om[j] = o0[j] = op[j] = 0u;
        }
    }
    return slice_draws<V>(om, o0, op, x0, r, t, p.rk, p.k0, p.k1, tab, p.C, err, inputs_used);
}

// Append the warp's heavy nodes (bit j of `heavy`: node node0 + j) to the list
// of the sequential pass: one atomic per warp and node slot that has any.
template <int V>
__device__ __forceinline__ void list_heavy(uint32_t heavy, uint64_t node0, uint32_t lane,
                                           const SliceTables &tab)
{
    if (!__any_sync(0xFFFFFFFFu, heavy != 0u)) return;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, (heavy >> j) & 1u);
        if (!m) continue;
        const uint32_t leader = __ffs(m) - 1u;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(tab.heavy_ctl, uint32_t(__popc(m)));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (m & (1u << lane)) {
            const uint32_t i = base + __popc(m & ((1u << lane) - 1u));
            if (i < tab.heavy_cap) tab.heavy_pos[i] = node0 + uint32_t(j);
            else atomicOr(tab.heavy_ctl + 1, 1u);
        }
    }
}

// kMinBlocks counts CTAs of 256 threads (the register bound of the variant
// table); the kernel runs CTAs of kSliceThreads.  kStream: pull-stream before
// colliding (else collide only).  kOne: a single replica, whose node indices
// fit 32 bits.
template <int V, int kMinBlocks, bool kOne, bool kStream>
__global__ void __launch_bounds__(kSliceThreads, kMinBlocks * 256 / kSliceThreads)
    k_step_slice(PlainArgs p, SliceTables tab)
{
    static_assert(V == 2 || V == 4 || V == 8, "V nodes per thread: 2, 4 or 8");
    using T = typename VecT<V>::T;
    using Index = typename std::conditional<kOne, uint32_t, uint64_t>::type;
    const uint32_t lane = threadIdx.x & 31u;
    const Index v_begin = Index(p.g_begin) * (8 / V), v_end = Index(p.g_end) * (8 / V);
    const Index g = v_begin + Index(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool active = g < v_end;
    const Index gv = active ? g : v_end - 1;  // idle lanes mirror the last vector
    const Index node0 = gv * V;

    Index off;
    uint32_t L, rid;
    if (kOne) {
        off = Index(p.one_off);
        L = p.one_L;
        rid = p.one_rid;
    } else {
        const uint32_t k = p.chunk_rep[node0 / 8u];
        off = p.rep_off[k];
        L = p.rep_L[k];
        rid = p.rep_id[k];
    }
    const uint32_t x0 = uint32_t(node0 - off);  // replica-local, a multiple of V

    const uint16_t *__restrict__ inm = p.in;
    const uint16_t *__restrict__ in0 = p.in + p.P;
    const uint16_t *__restrict__ inp = p.in + 2 * p.P;
    // halo: lanes at a warp or replica edge load theirs directly, issued together
    // with the vector loads; the others take them from the neighbouring lanes
    const bool own_next = !(lane < 31u && x0 + V < L), own_prev = !(lane > 0u && x0 > 0u);
    uint32_t nxt_own = 0u, prv_own = 0u;
    if (kStream && own_next)
        nxt_own = x0 + V < L ? inm[off + x0 + V] : (kOne && p.halo_in ? p.halo_in[1] : inm[off]);
    if (kStream && own_prev)
        prv_own = x0 > 0u ? inp[off + x0 - 1u] : (kOne && p.halo_in ? p.halo_in[0] : inp[off + L - 1u]);
    uint32_t em[V], e0[V], ep[V];
    unpack(__ldcs(reinterpret_cast<const T *>(inm + node0)), em);
    unpack(__ldcs(reinterpret_cast<const T *>(in0 + node0)), e0);
    unpack(__ldcs(reinterpret_cast<const T *>(inp + node0)), ep);
    uint32_t nxt = __shfl_down_sync(0xFFFFFFFFu, em[0], 1);
    uint32_t prv = __shfl_up_sync(0xFFFFFFFFu, ep[V - 1], 1);
    if (kStream && own_next) nxt = nxt_own;
    if (kStream && own_prev) prv = prv_own;
    // valid nodes here (none when the whole vector is replica padding)
    const uint32_t nv = x0 >= L ? 0u : (L - x0 < uint32_t(V) ? L - x0 : uint32_t(V));
    const uint32_t t = p.t_dev ? *p.t_dev + p.t : p.t;

    uint32_t err = 0;
    uint32_t om[V], o0[V], op[V];
    uint32_t heavy = slice_vector<V>(em, e0, ep, nxt, prv, kStream, p.x_base + x0, nv,
                                              rid + p.r0, t, p, tab, om, o0, op, err);
    if (active) {
        T vo;
        pack(om, vo);
        __stcs(reinterpret_cast<T *>(p.out + node0), vo);
        pack(o0, vo);
        __stcs(reinterpret_cast<T *>(p.out + p.P + node0), vo);
        pack(op, vo);
        __stcs(reinterpret_cast<T *>(p.out + 2 * p.P + node0), vo);
        flag_error(p.err, err);
    }
    // heavy nodes (written unchanged) join the list of the sequential pass
    if (!active) heavy = 0u;
    list_heavy<V>(heavy, uint64_t(node0), lane, tab);
}

// ---------------------------------------------------------------------------
// Grid-stride form for one replica (the single-lattice step): a grid sized to
// the resident CTAs; each warp walks tiles of 32 V nodes, loading the next
// tile's three vectors (and its edge values) into registers before it draws
// the current one, so the HBM latency overlaps the table lookups.  The
// per-launch values (round keys, table pointers) stay in registers for all of
// a warp's tiles.
// ---------------------------------------------------------------------------
template <int V, int kMinBlocks, bool kStream>
__global__ void __launch_bounds__(kSliceThreads, kMinBlocks * 256 / kSliceThreads)
    k_step_slice_loop(PlainArgs p, SliceTables tab)
{
    static_assert(V == 2 || V == 4 || V == 8, "V nodes per thread: 2, 4 or 8");
    using T = typename VecT<V>::T;
    constexpr uint32_t TW = 32u * uint32_t(V);  // nodes per warp tile
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t wpb = kSliceThreads / 32u;
    const uint32_t wid = blockIdx.x * wpb + (threadIdx.x >> 5), nw = gridDim.x * wpb;
    const uint64_t off = p.one_off;
    const uint32_t L = p.one_L, Pn = (L + 7u) & ~7u;
    const uint32_t tiles = (Pn + TW - 1u) / TW;
    const uint16_t *__restrict__ inm = p.in + off;
    const uint16_t *__restrict__ in0 = p.in + p.P + off;
    const uint16_t *__restrict__ inp = p.in + 2 * p.P + off;
    const uint32_t t = p.t_dev ? *p.t_dev + p.t : p.t;
    const uint32_t r = p.one_rid + p.r0;
    uint32_t err = 0;

    // a tile's three vectors for this lane (lanes past the replica mirror its
    // last vector and store nothing) and the edge values the lane needs from
    // beyond its warp: B_-1(x0 + V) for the last lane (or the replica's end),
    // B_+1(x0 - 1) for the first (or the replica's start)
    auto load = [&](uint32_t tile, T &vm, T &vz, T &vp, uint32_t &hn, uint32_t &hp) {
        const uint32_t x0 = tile * TW + lane * uint32_t(V);
        const uint32_t xs = x0 < Pn ? x0 : Pn - uint32_t(V);
        vm = __ldcs(reinterpret_cast<const T *>(inm + xs));
        vz = __ldcs(reinterpret_cast<const T *>(in0 + xs));
        vp = __ldcs(reinterpret_cast<const T *>(inp + xs));
        hn = hp = 0u;
        if (kStream && !(lane < 31u && x0 + V < L))
            hn = x0 + V < L ? inm[x0 + V] : (p.halo_in ? p.halo_in[1] : inm[0]);
        if (kStream && !(lane > 0u && x0 > 0u))
            hp = x0 > 0u && x0 - 1u < L ? inp[x0 - 1u] : (p.halo_in ? p.halo_in[0] : inp[L - 1u]);
    };

    uint32_t tile = wid;
    T cm, cz, cp;
    uint32_t chn = 0, chp = 0;
    if (tile < tiles) load(tile, cm, cz, cp, chn, chp);
    for (; tile < tiles; tile += nw) {
        T nm, nz, np;
        uint32_t nhn = 0, nhp = 0;
        if (tile + nw < tiles) load(tile + nw, nm, nz, np, nhn, nhp);
        const uint32_t x0 = tile * TW + lane * uint32_t(V);
        uint32_t em[V], e0[V], ep[V];
        unpack(cm, em);
        unpack(cz, e0);
        unpack(cp, ep);
        uint32_t nxt = __shfl_down_sync(0xFFFFFFFFu, em[0], 1);
        uint32_t prv = __shfl_up_sync(0xFFFFFFFFu, ep[V - 1], 1);
        if (kStream && !(lane < 31u && x0 + V < L)) nxt = chn;
        if (kStream && !(lane > 0u && x0 > 0u)) prv = chp;
        const uint32_t nv = x0 >= L ? 0u : (L - x0 < uint32_t(V) ? L - x0 : uint32_t(V));
        uint32_t om[V], o0[V], op[V];
        uint32_t heavy = slice_vector<V>(em, e0, ep, nxt, prv, kStream, p.x_base + x0, nv, r, t, p,
                                         tab, om, o0, op, err);
        const bool active = x0 < Pn;
        if (active) {
            T vo;
            pack(om, vo);
            __stcs(reinterpret_cast<T *>(p.out + off + x0), vo);
            pack(o0, vo);
            __stcs(reinterpret_cast<T *>(p.out + p.P + off + x0), vo);
            pack(op, vo);
            __stcs(reinterpret_cast<T *>(p.out + 2 * p.P + off + x0), vo);
        } else {
            heavy = 0u;
        }
        list_heavy<V>(heavy, off + x0, lane, tab);
        cm = nm;
        cz = nz;
        cp = np;
        chn = nhn;
        chp = nhp;
    }
    flag_error(p.err, err);
}

template <int V, int kMinBlocks>
static cudaError_t launch_slice_loop_v(const PlainArgs &p, const SliceTables &tab, cudaStream_t s)
{
    auto kern = p.stream ? k_step_slice_loop<V, kMinBlocks, true> : k_step_slice_loop<V, kMinBlocks, false>;
    static int resident[2] = {0, 0};  // CTAs per SM of the two forms
    int &res = resident[p.stream ? 1 : 0];
    cudaError_t e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (res == 0) {
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, int(kSliceThreads), 0)) !=
            cudaSuccess)
            return e;
        res = std::max(per_sm, 1);
    }
    const uint32_t Pn = (p.one_L + 7u) & ~7u;
    const uint32_t tiles = (Pn + 32u * V - 1u) / (32u * V);
    const uint32_t warps = kSliceThreads / 32u;
    const uint32_t grid = std::max<uint32_t>(1u, std::min<uint32_t>((tiles + warps - 1u) / warps,
                                                                    uint32_t(sms * res)));
    kern<<<grid, kSliceThreads, 0, s>>>(p, tab);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Temporally blocked form for one replica: a CTA of kThreads threads holds a
// window of E = kThreads V consecutive nodes of the periodic lattice in
// registers (V per thread) and advances it up to K steps in one launch.  Each
// step a node needs B_-1 of its right neighbour and B_+1 of its left one
// (Sec. III streaming); inside a warp they come by shuffle, across warps
// through a shared slot per warp (double-buffered by step parity, one barrier
// per step).  The window's ends have no neighbours, so after s steps only
// [s, E - s) holds the lattice's values; nodes outside that cone are set to
// zero before each draw (they report nothing and never reach the tables'
// fallback or the sequential draws).  After the launch's n <= K steps the
// middle T = E - 2K nodes, the CTA's own tile, are written.  Every node's
// random numbers depend on its global index and time step only, so the nodes
// that two windows both compute get the same values; nodes beyond the tables
// take the sequential draws in place.  The state crosses HBM once per launch
// instead of once per step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t wrap_node(int64_t x, uint32_t L)
{
    const int64_t m = x % int64_t(L);
    return uint32_t(m < 0 ? m + int64_t(L) : m);
}

// kSync: how a window's warps meet each step.  kTbBarrier: the CTA is the
// window, one barrier per step.  kTbWarp: every warp is a window of its own
// (E = 32 V, nothing to wait for: a warp held up by a rare exact draw holds up
// nobody else).  kTbNeighbours: the CTA is the window, and each warp waits
// only for its two neighbours' edge values of the step (flags in shared
// memory; the double-buffered slots let a warp run at most one step ahead of
// a neighbour, which is what keeps a slot from being overwritten before it is
// read); every wait gives up after kTbWaitCycles with MCLG_ERR_TIMEOUT.
constexpr int kTbBarrier = 0, kTbWarp = 1, kTbNeighbours = 2;
constexpr long long kTbWaitCycles = 2000000000ll;  // about a second

template <int V, int K, int kThreads, int kMinCtas, int kSync>
__global__ void __launch_bounds__(kThreads, kMinCtas)
    k_step_slice_tb(PlainArgs p, SliceTables tab, uint32_t n_steps)
{
    constexpr bool kWarp = kSync == kTbWarp;
    static_assert(V == 2 || V == 4 || V == 8, "V nodes per thread: 2, 4 or 8");
    static_assert(K % V == 0 && K % 2 == 0, "the halo holds whole vectors");
    constexpr uint32_t E = uint32_t(kWarp ? 32 : kThreads) * V, TT = E - 2u * K, W = kThreads / 32;
    static_assert(TT % 8u == 0u && TT > 0u, "tiles start on multiples of 8 nodes");
    using T = typename VecT<V>::T;
    __shared__ uint32_t s_first[2][W], s_last[2][W];  // per warp: B_-1 of its first node, B_+1 of its last
    __shared__ uint32_t s_flag[W];                     // kTbNeighbours: steps whose edges are out
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (kSync == kTbNeighbours) {
        if (lane == 0u) s_flag[warp] = 0u;
        __syncthreads();
    }
    const uint64_t off = p.one_off;
    const uint32_t L = p.one_L, Pn = (L + 7u) & ~7u;
    const uint32_t tile = kWarp ? blockIdx.x * W + warp : blockIdx.x;
    const uint32_t x0 = tile * TT;                       // the tile's first node
    const uint32_t e0 = (kWarp ? lane : threadIdx.x) * uint32_t(V);  // this thread's first window position
    if (kWarp && x0 >= Pn) return;                       // a whole warp past the last tile
    const int64_t xs = int64_t(x0) + int64_t(e0) - K;    // its node before wrapping
    const bool plain = xs >= 0 && xs + V <= int64_t(L);  // no wrap inside (xs is even, a multiple of V)
    const uint16_t *__restrict__ inm = p.in + off;
    const uint16_t *__restrict__ in0 = p.in + p.P + off;
    const uint16_t *__restrict__ inp = p.in + 2 * p.P + off;
    uint32_t em[V], ez[V], ep[V], xj[V];
    if (plain) {
        unpack(__ldcs(reinterpret_cast<const T *>(inm + xs)), em);
        unpack(__ldcs(reinterpret_cast<const T *>(in0 + xs)), ez);
        unpack(__ldcs(reinterpret_cast<const T *>(inp + xs)), ep);
#pragma unroll
        for (int j = 0; j < V; ++j) xj[j] = uint32_t(xs) + uint32_t(j);
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            xj[j] = wrap_node(xs + j, L);
            em[j] = inm[xj[j]];
            ez[j] = in0[xj[j]];
            ep[j] = inp[xj[j]];
        }
    }
#pragma unroll
    for (int j = 0; j < V; ++j) xj[j] += p.x_base;  // the random numbers' node index
    const uint32_t t0 = p.t_dev ? *p.t_dev + p.t : p.t;
    const uint32_t r = p.one_rid + p.r0;
    const bool stream = p.stream != 0u;
    uint32_t err = 0;
    for (uint32_t s = 0; s < n_steps; ++s) {
        const uint32_t t = t0 + s;
        uint32_t a[V], b[V], c[V];
        if (stream) {
            if (kSync == kTbBarrier) {
                if (lane == 0u) s_first[s & 1u][warp] = em[0];
                if (lane == 31u) s_last[s & 1u][warp] = ep[V - 1];
                __syncthreads();
            } else if (kSync == kTbNeighbours) {
                if (lane == 0u) s_first[s & 1u][warp] = em[0];
                if (lane == 31u) s_last[s & 1u][warp] = ep[V - 1];
                __syncwarp();
                bool ok = true;
                if (lane == 0u) {
                    volatile uint32_t *flag = s_flag;
                    __threadfence_block();
                    flag[warp] = s + 1u;  // this warp's edges of step s are out
                    const long long start = clock64();
                    while ((warp > 0u && flag[warp - 1u] < s + 1u) ||
                           (warp + 1u < W && flag[warp + 1u] < s + 1u)) {
                        if (clock64() - start > kTbWaitCycles) {
                            ok = false;
                            break;
                        }
                        __nanosleep(32);
                    }
                    __threadfence_block();
                }
                if (!__shfl_sync(0xFFFFFFFFu, ok ? 1u : 0u, 0)) {
                    err |= kErrTimeout;  // a neighbour never came: give up (state unspecified)
                    break;
                }
                __syncwarp();
            }
            uint32_t nxt = __shfl_down_sync(0xFFFFFFFFu, em[0], 1);
            uint32_t prv = __shfl_up_sync(0xFFFFFFFFu, ep[V - 1], 1);
            const volatile uint32_t *vf = &s_first[s & 1u][0], *vl = &s_last[s & 1u][0];
            if (lane == 31u) nxt = !kWarp && warp + 1u < W ? vf[warp + 1u] : 0u;
            if (lane == 0u) prv = !kWarp && warp > 0u ? vl[warp - 1u] : 0u;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                a[j] = j + 1 < V ? em[j + 1] : nxt;
                b[j] = ez[j];
                c[j] = j > 0 ? ep[j - 1] : prv;
            }
            // outside the cone of valid values: nothing
            if (e0 <= s || e0 + V + s >= E) {
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const uint32_t e = e0 + uint32_t(j);
                    if (e < s + 1u || e + s + 1u >= E) a[j] = b[j] = c[j] = 0u;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                a[j] = em[j];
                b[j] = ez[j];
                c[j] = ep[j];
            }
        }
        const uint32_t heavy =
            plain ? slice_draws<V>(a, b, c, xj[0], r, t, p.rk, p.k0, p.k1, tab, p.C, err)
                  : slice_draws_scattered<V>(a, b, c, xj, r, t, p.rk, p.k0, p.k1, tab, p.C, err);
        if (heavy) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                if (!((heavy >> j) & 1u)) continue;
                const NodeKey nk{xj[j], r, t, p.k0, p.k1};
                uint32_t ln, ld;
                node_rate(p.galilean != 0u, a[j], b[j], c[j], p.lam_n, p.lam_d, ln, ld);
                collide_node(a[j], b[j], c[j], nk, p.rk, p.C, ln, ld, err);
            }
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
            em[j] = a[j];
            ez[j] = b[j];
            ep[j] = c[j];
        }
    }
    // the tile's own nodes (padding beyond the replica's end written as zero)
    if (e0 >= K && e0 + V <= K + TT) {
        const uint32_t x = x0 + e0 - K;
        if (x < Pn) {
            if (x + V > L) {
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (x + uint32_t(j) >= L) em[j] = ez[j] = ep[j] = 0u;
            }
            T vo;
            pack(em, vo);
            __stcs(reinterpret_cast<T *>(p.out + off + x), vo);
            pack(ez, vo);
            __stcs(reinterpret_cast<T *>(p.out + p.P + off + x), vo);
            pack(ep, vo);
            __stcs(reinterpret_cast<T *>(p.out + 2 * p.P + off + x), vo);
        }
    }
    flag_error(p.err, err);
}

template <int V, int K, int kThreads, int kMinCtas, int kSync>
static cudaError_t launch_slice_tb_v(const PlainArgs &p, const SliceTables &tab, uint32_t n_steps,
                                     cudaStream_t s)
{
    constexpr bool kWarp = kSync == kTbWarp;
    constexpr uint32_t TT = uint32_t(kWarp ? 32 : kThreads) * V - 2u * K;
    constexpr uint32_t kPerCta = kWarp ? kThreads / 32 : 1;  // tiles per CTA
    if (n_steps == 0u || n_steps > uint32_t(K)) return cudaErrorInvalidValue;
    const uint32_t Pn = (p.one_L + 7u) & ~7u;
    const uint32_t tiles = (Pn + TT - 1u) / TT;
    k_step_slice_tb<V, K, kThreads, kMinCtas, kSync>
        <<<(tiles + kPerCta - 1u) / kPerCta, kThreads, 0, s>>>(p, tab, n_steps);
    return cudaGetLastError();
}

// Temporally blocked configurations: (nodes per thread, steps per launch,
// threads per CTA, minimum CTAs per SM, windows per warp or per CTA).
static const uint32_t kTbSteps[kSliceTbConfigs] = {16, 8, 4, 8, 16, 16};

uint32_t slice_tb_steps(uint32_t config) { return kTbSteps[config < kSliceTbConfigs ? config : 0]; }

cudaError_t launch_slice_tb(const PlainArgs &p, const SliceTables &tab, uint32_t n_steps,
                            uint32_t config, cudaStream_t s)
{
    switch (config) {
    case 0: return launch_slice_tb_v<4, 16, 256, 4, kTbNeighbours>(p, tab, n_steps, s);
    case 1: return launch_slice_tb_v<4, 8, 128, 6, kTbBarrier>(p, tab, n_steps, s);
    case 2: return launch_slice_tb_v<4, 4, 256, 4, kTbWarp>(p, tab, n_steps, s);
    case 3: return launch_slice_tb_v<4, 8, 256, 4, kTbWarp>(p, tab, n_steps, s);
    case 4: return launch_slice_tb_v<4, 16, 128, 6, kTbBarrier>(p, tab, n_steps, s);
    default: return launch_slice_tb_v<4, 16, 256, 3, kTbNeighbours>(p, tab, n_steps, s);
    }
}

// ---------------------------------------------------------------------------
// Warp-specialised form for one replica (the single-lattice step).  A
// producer warp streams tiles of T = W x 32 x 8 nodes of the three planes into
// a ring of S shared-memory stages with bulk asynchronous copies
// (cp.async.bulk, each stage's bytes counted on its "full" mbarrier); W
// consumer warps read a stage into registers, hand it back through its
// "empty" mbarrier at once, draw every node's C sub-collisions from the tables
// and store the post-collision vectors straight to global memory.  The bytes
// in flight live in shared memory instead of registers, so HBM streaming no
// longer competes with the table lookups for warps.  Every wait is bounded:
// after about two seconds it sets the timeout bit of the error word and the
// CTA stops (the producer first lets the copies it issued land).
// ---------------------------------------------------------------------------
namespace {

constexpr long long kWaitCycles = 4000000000ll;  // bounded mbarrier waits (~2 s at 2 GHz)

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

// Wait for the phase of `parity` to complete; false after kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_test(bar, parity)) return true;
    const long long start = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - start > kWaitCycles) return false;
    return true;
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completion counted on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace

// Shared memory of one stage: plane -1 holds nodes [x0, x0 + T + 8), plane 0
// nodes [x0, x0 + T), plane +1 nodes [x0 - 8, x0 + T) (one 16-byte halo vector
// on the side each plane streams from).
template <int W, int V>
struct WsTile {
    static constexpr uint32_t T = uint32_t(W) * 32u * uint32_t(V);  // nodes per tile
    static constexpr uint32_t kBuf = T + 8u;                // nodes per plane buffer
    static constexpr uint32_t kStage = 3u * kBuf;           // uint16 per stage
};

template <int W, int V, int S, int kMinBlocks>
__global__ void __launch_bounds__((W + 1) * 32, kMinBlocks)
    k_step_slice_ws(PlainArgs p, SliceTables tab)
{
    static_assert(V == 4 || V == 8, "V nodes per consumer thread: 4 or 8");
    using Tl = WsTile<W, V>;
    using Vec = typename VecT<V>::T;
    constexpr uint32_t T = Tl::T, kBuf = Tl::kBuf;
    extern __shared__ __align__(128) uint16_t ring[];
    __shared__ __align__(8) uint64_t full[S], empty[S];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint64_t off = p.one_off;
    const uint32_t L = p.one_L;
    const uint32_t Pn = (L + 7u) & ~7u;  // the replica's nodes with padding
    const uint32_t tiles = (Pn + T - 1u) / T;
    const uint16_t *__restrict__ inm = p.in + off;
    const uint16_t *__restrict__ in0 = p.in + p.P + off;
    const uint16_t *__restrict__ inp = p.in + 2 * p.P + off;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1u);
            mbar_init(&empty[s], uint32_t(W));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == uint32_t(W)) {
        // producer: one lane issues the copies of this CTA's tiles in order
        if (lane != 0u) return;
        uint32_t i = 0, issued = 0;
        bool ok = true;
        for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++i) {
            const uint32_t s = i % S, round = i / S;
            if (round > 0u && !mbar_wait(&empty[s], (round - 1u) & 1u)) {
                ok = false;
                break;
            }
            const uint32_t x0 = tile * T, n = min(T, Pn - x0);
            const uint32_t nm = min(n + 8u, Pn - x0);             // plane -1: one vector beyond
            const uint32_t lo = x0 >= 8u ? 8u : 0u;               // plane +1: one vector before
            uint16_t *st = ring + size_t(s) * Tl::kStage;
            mbar_expect_tx(&full[s], 2u * (nm + n + n + lo));
            bulk_load(st, inm + x0, 2u * nm, &full[s]);
            bulk_load(st + kBuf, in0 + x0, 2u * n, &full[s]);
            bulk_load(st + 2u * kBuf + (8u - lo), inp + x0 - lo, 2u * (n + lo), &full[s]);
            ++issued;
        }
        if (!ok) {
            flag_error(p.err, kErrTimeout);
            // let the copies already issued land before the CTA's memory goes away
            for (uint32_t k = issued > uint32_t(S) ? issued - S : 0u; k < issued; ++k)
                mbar_wait(&full[k % S], (k / S) & 1u);
        }
        return;
    }

    // consumers
    const bool kStream = p.stream != 0u;
    const uint32_t t = p.t_dev ? *p.t_dev + p.t : p.t;
    const uint32_t r = p.one_rid + p.r0;
    const uint32_t xl = (warp * 32u + lane) * uint32_t(V);  // tile-local first node of this thread
    uint32_t err = 0, i = 0;
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++i) {
        const uint32_t s = i % S, round = i / S;
        if (!mbar_wait(&full[s], round & 1u)) {
            err |= kErrTimeout;
            break;
        }
        const uint32_t x0t = tile * T, n = min(T, Pn - x0t);
        const uint32_t x0 = x0t + xl;  // replica-local first node of this thread
        const uint16_t *st = ring + size_t(s) * Tl::kStage;
        const uint16_t *sm = st, *sz = st + kBuf, *sp = st + 2u * kBuf + 8u;  // index x - x0t
        uint32_t em[V], e0[V], ep[V];
        unpack(*reinterpret_cast<const Vec *>(sm + xl), em);
        unpack(*reinterpret_cast<const Vec *>(sz + xl), e0);
        unpack(*reinterpret_cast<const Vec *>(sp + xl), ep);
        // halo: B_-1(x0 + V) and B_+1(x0 - 1), from the neighbouring lanes, the
        // stage's halo vectors, or (at the ends of the lattice) the periodic image
        const bool own_next = !(lane < 31u && x0 + V < L), own_prev = !(lane > 0u && x0 > 0u);
        uint32_t nxt = __shfl_down_sync(0xFFFFFFFFu, em[0], 1);
        uint32_t prv = __shfl_up_sync(0xFFFFFFFFu, ep[V - 1], 1);
        if (kStream && own_next)
            nxt = x0 + V < L ? uint32_t(sm[xl + V]) : uint32_t(p.halo_in ? p.halo_in[1] : inm[0]);
        if (kStream && own_prev)
            prv = x0 > 0u ? uint32_t(sp[int(xl) - 1]) : uint32_t(p.halo_in ? p.halo_in[0] : inp[L - 1u]);

        const bool active = xl < n;
        const uint32_t nv = x0 >= L ? 0u : (L - x0 < uint32_t(V) ? L - x0 : uint32_t(V));
        uint32_t om[V], o0[V], op[V];
        // the stage goes back to the producer once every lane's reads of it have
        // been consumed (arriving right after issuing the shared-memory loads let
        // the next bulk copy overwrite values still in flight)
        uint32_t heavy = slice_vector_phased<V>(
            em, e0, ep, nxt, prv, kStream, p.x_base + x0, nv, r, t, p, tab, om, o0, op, err, [&]() {
                __syncwarp();
                if (lane == 0u) mbar_arrive(&empty[s]);
            });
        const uint64_t node0 = off + x0;
        if (active) {
            Vec vo;
            pack(om, vo);
            __stcs(reinterpret_cast<Vec *>(p.out + node0), vo);
            pack(o0, vo);
            __stcs(reinterpret_cast<Vec *>(p.out + p.P + node0), vo);
            pack(op, vo);
            __stcs(reinterpret_cast<Vec *>(p.out + 2 * p.P + node0), vo);
        }
        if (!active) heavy = 0u;
        list_heavy<V>(heavy, node0, lane, tab);
    }
    flag_error(p.err, err);
}

template <int W, int V, int S, int kMinBlocks>
static cudaError_t launch_slice_ws_v(const PlainArgs &p, const SliceTables &tab, cudaStream_t s)
{
    using Tl = WsTile<W, V>;
    const size_t smem = size_t(S) * Tl::kStage * sizeof(uint16_t);
    auto kern = k_step_slice_ws<W, V, S, kMinBlocks>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (W + 1) * 32, smem)) !=
        cudaSuccess)
        return e;
    const uint32_t Pn = (p.one_L + 7u) & ~7u;
    const uint32_t tiles = (Pn + Tl::T - 1u) / Tl::T;
    const uint32_t grid = std::min<uint32_t>(tiles, uint32_t(sms * std::max(per_sm, 1)));
    kern<<<grid, (W + 1) * 32, smem, s>>>(p, tab);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Statistics form (MCLG_STATS with the slice sampler): one pass per step that
// both steps the replicas and adds the statistics of the field it reads,
// n(x, t) (Sec. V: sums of n_i, n_i n_j at a node and n_i(x) n_j(x + 1)), so
// the state is not read a second time.  A CTA of 8 warps takes 64 positions
// of KR x 8 replicas: warp w steps replicas w, w + 8, ... (2 nodes per lane,
// as k_step_slice does) and adds each node's 18 quantities to its lane's
// 32-bit counters in shared memory (exact while every value is below 2^14 and
// KR <= 16: 16 products below 2^28 fit 32 bits; a node with a larger value
// adds its quantities to the global 64-bit sums at once); at the end the CTA
// folds its 8 warps' counters into the batch sums with one 64-bit atomic per
// position and quantity.  The kernel of step t adds its input only when
// t >= *stats_from (the library's last call ended with n(t) already added, or
// n(t) is the field at a reset): every field after a reset is counted once.
// ---------------------------------------------------------------------------
constexpr int kStatQty = 18;  // 3 sums + 6 same-node products + 9 neighbour products

__device__ __forceinline__ void node_quantities(uint32_t a, uint32_t b, uint32_t c, uint32_t a1,
                                                uint32_t b1, uint32_t c1, uint32_t (&q)[kStatQty])
{
    q[0] = a; q[1] = b; q[2] = c;
    q[3] = a * a; q[4] = a * b; q[5] = a * c; q[6] = b * b; q[7] = b * c; q[8] = c * c;
    q[9] = a * a1; q[10] = a * b1; q[11] = a * c1;
    q[12] = b * a1; q[13] = b * b1; q[14] = b * c1;
    q[15] = c * a1; q[16] = c * b1; q[17] = c * c1;
}

template <int KR, bool kRed, bool kStream>
__global__ void __launch_bounds__(256, 4) k_step_slice_stats(PlainArgs p, SliceTables tab, StatsArgs sa)
{
    static_assert(KR >= 1 && KR <= 16, "32-bit counters hold at most 16 products below 2^28");
    constexpr int V = 2;
    __shared__ uint32_t cnt[8][V * kStatQty][32];  // per warp, (node, quantity), lane
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t L = p.one_L, Pn = (L + 7u) & ~7u;
    const uint32_t x0 = blockIdx.x * 64u + lane * V;       // replica-local first node of the lane
    const bool inside = x0 < Pn;
    const uint32_t xv = inside ? x0 : Pn - V;              // lanes past the replica mirror its end
    const uint32_t t = p.t_dev ? *p.t_dev + p.t : p.t;
    const bool acc = t >= *sa.stats_from;
#pragma unroll
    for (int k = 0; k < V * kStatQty; ++k) cnt[warp][k][lane] = 0u;
    uint32_t err = 0;
    const uint16_t *__restrict__ inm = p.in;
    const uint16_t *__restrict__ in0 = p.in + p.P;
    const uint16_t *__restrict__ inp = p.in + 2 * p.P;
    for (int k = 0; k < KR; ++k) {
        const uint32_t r = blockIdx.y * (8u * KR) + warp + 8u * uint32_t(k);
        if (r >= sa.R) break;  // the same for the whole warp
        const uint64_t off = uint64_t(r) * sa.stride, node0 = off + xv;
        const bool own_next = !(lane < 31u && xv + V < L), own_prev = !(lane > 0u && xv > 0u);
        uint32_t nxt_own = 0u, prv_own = 0u;
        if (kStream && own_next) nxt_own = inm[off + (xv + V < L ? xv + V : 0u)];
        if (kStream && own_prev) prv_own = inp[off + (xv > 0u ? xv - 1u : L - 1u)];
        uint32_t em[V], e0[V], ep[V];
        unpack(__ldcs(reinterpret_cast<const uint32_t *>(inm + node0)), em);
        unpack(__ldcs(reinterpret_cast<const uint32_t *>(in0 + node0)), e0);
        unpack(__ldcs(reinterpret_cast<const uint32_t *>(inp + node0)), ep);
        uint32_t nxt = __shfl_down_sync(0xFFFFFFFFu, em[0], 1);
        uint32_t prv = __shfl_up_sync(0xFFFFFFFFu, ep[V - 1], 1);
        if (kStream && own_next) nxt = nxt_own;
        if (kStream && own_prev) prv = prv_own;
        const uint32_t nv = (!inside || xv >= L) ? 0u : (L - xv < uint32_t(V) ? L - xv : uint32_t(V));
        // the input field n(x, t) of the lane's nodes (the values the step collides)
        uint32_t na[V], nb[V], nc[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            na[j] = kStream ? ((uint32_t(j) + 1u < nv) ? em[(j + 1) % V] : nxt) : em[j];
            nb[j] = e0[j];
            nc[j] = kStream ? ((j > 0) ? ep[(j + V - 1) % V] : prv) : ep[j];
        }
        uint32_t om[V], o0[V], op[V];
        uint32_t heavy = slice_vector<V>(em, e0, ep, nxt, prv, kStream, p.x_base + xv, nv,
                                                  r + p.r0, t, p, tab, om, o0, op, err);
        if (inside) {
            __stcs(reinterpret_cast<uint32_t *>(p.out + node0), om[0] | (om[1] << 16));
            __stcs(reinterpret_cast<uint32_t *>(p.out + p.P + node0), o0[0] | (o0[1] << 16));
            __stcs(reinterpret_cast<uint32_t *>(p.out + 2 * p.P + node0), op[0] | (op[1] << 16));
        }
        if (!inside) heavy = 0u;
        list_heavy<V>(heavy, node0, lane, tab);
        if (!acc) continue;
        // the right neighbour of the lane's last node: the next lane's first node,
        // or (at the end of a warp or of the replica) read from the input field
        uint32_t a1 = __shfl_down_sync(0xFFFFFFFFu, na[0], 1);
        uint32_t b1 = __shfl_down_sync(0xFFFFFFFFu, nb[0], 1);
        uint32_t c1 = __shfl_down_sync(0xFFFFFFFFu, nc[0], 1);
        if (nv > 0u && (lane == 31u || xv + nv >= L)) {
            const uint32_t y = xv + nv < L ? xv + nv : 0u;   // node after the last valid one
            const uint32_t yr = kStream ? (y + 1u < L ? y + 1u : 0u) : y;
            const uint32_t yl = kStream ? (y > 0u ? y - 1u : L - 1u) : y;
            a1 = inm[off + yr];
            b1 = in0[off + y];
            c1 = inp[off + yl];
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
            if (uint32_t(j) >= nv) break;
            const bool last = uint32_t(j) + 1u == nv;
            uint32_t q[kStatQty];
            node_quantities(na[j], nb[j], nc[j], last ? a1 : na[j + 1 < V ? j + 1 : j],
                            last ? b1 : nb[j + 1 < V ? j + 1 : j],
                            last ? c1 : nc[j + 1 < V ? j + 1 : j], q);
            const uint32_t big = na[j] | nb[j] | nc[j] | (last ? (a1 | b1 | c1) : 0u) |
                                 (j + 1 < V ? na[j + 1] | nb[j + 1] | nc[j + 1] : 0u);
            if (big < (1u << 14)) {
#pragma unroll
                for (int m = 0; m < kStatQty; ++m) {  // the lane's own counter: no contention
                    if (kRed) atomicAdd(&cnt[warp][j * kStatQty + m][lane], q[m]);
                    else cnt[warp][j * kStatQty + m][lane] += q[m];
                }
            } else {
                // values of 2^14 or more: exact 64-bit products straight into the batch
                const uint64_t v[3] = {na[j], nb[j], nc[j]};
                const int jn = j + 1 < V ? j + 1 : j;  // the next node when it is this lane's
                const uint64_t w[3] = {last ? a1 : na[jn], last ? b1 : nb[jn], last ? c1 : nc[jn]};
                unsigned long long *dst = sa.batch + uint64_t(xv + j) * kStatQty;
                int m = 0;
                for (int i = 0; i < 3; ++i) atomicAdd(dst + m++, v[i]);
                for (int i = 0; i < 3; ++i)
                    for (int i2 = i; i2 < 3; ++i2) atomicAdd(dst + m++, v[i] * v[i2]);
                for (int i = 0; i < 3; ++i)
                    for (int i2 = 0; i2 < 3; ++i2) atomicAdd(dst + m++, v[i] * w[i2]);
            }
        }
    }
    flag_error(p.err, err);
    if (!acc) return;
    __syncthreads();
    // fold the 8 warps' counters: item (node j, quantity m, lane) per thread
    for (uint32_t it = threadIdx.x; it < uint32_t(V * kStatQty) * 32u; it += blockDim.x) {
        const uint32_t l = it & 31u, jm = it >> 5, j = jm / kStatQty, m = jm % kStatQty;
        const uint32_t x = blockIdx.x * 64u + l * V + j;
        if (x >= L) continue;
        unsigned long long sum = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) sum += cnt[w][jm][l];
        if (sum) atomicAdd(sa.batch + uint64_t(x) * kStatQty + m, sum);
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
        atomicAdd(sa.batch_count, (unsigned long long)sa.R);  // one sample of every replica
}

// The sequential pass over the step's heavy nodes (see above).  Reads the
// table kernel's output, where heavy nodes still hold their pre-collision
// state, and overwrites them with their sequential collisions.  The last CTA
// to finish resets the list for the next step.
template <bool kOne>
__global__ void __launch_bounds__(kPlainThreads) k_step_heavy(PlainArgs p, SliceTables tab)
{
    const uint32_t count = *(volatile uint32_t *)tab.heavy_ctl;
    const bool scan = *(volatile uint32_t *)(tab.heavy_ctl + 1) != 0u;
    const uint32_t t = p.t_dev ? *p.t_dev + p.t : p.t;
    const uint64_t first = p.g_begin * 8u, end = p.g_end * 8u;
    const uint64_t n = scan ? end - first : min(count, tab.heavy_cap);
    if (n == 0 && !scan) return;  // nothing listed: the list is already clear
    uint32_t err = 0;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t pos = scan ? first + i : tab.heavy_pos[i];
        uint64_t off;
        uint32_t L, rid;
        if (kOne) {
            off = p.one_off;
            L = p.one_L;
            rid = p.one_rid;
        } else {
            const uint32_t k = p.chunk_rep[pos / 8u];
            off = p.rep_off[k];
            L = p.rep_L[k];
            rid = p.rep_id[k];
        }
        const uint32_t x = uint32_t(pos - off);
        uint32_t a = p.out[pos], b = p.out[p.P + pos], c = p.out[2 * p.P + pos];
        if (x >= L || a + b + c <= tab.n_max) continue;  // padding, or a table node (scan)
        const NodeKey nk{p.x_base + x, rid + p.r0, t, p.k0, p.k1};
        uint32_t ln, ld;
        node_rate(p.galilean != 0u, a, b, c, p.lam_n, p.lam_d, ln, ld);
        collide_node(a, b, c, nk, p.rk, p.C, ln, ld, err);
        p.out[pos] = uint16_t(a);
        p.out[p.P + pos] = uint16_t(b);
        p.out[2 * p.P + pos] = uint16_t(c);
    }
    flag_error(p.err, err);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(tab.heavy_ctl + 2, 1u) == gridDim.x - 1u) {  // every CTA has read the list
            tab.heavy_ctl[0] = 0u;
            tab.heavy_ctl[1] = 0u;
            tab.heavy_ctl[2] = 0u;
            __threadfence();
        }
    }
}

template <int V, int kMinBlocks>
static void launch_slice_v(const PlainArgs &p, bool one, const SliceTables &tab, cudaStream_t s)
{
    const uint64_t threads = (p.g_end - p.g_begin) * (8u / V);
    const dim3 grid(uint32_t((threads + kSliceThreads - 1) / kSliceThreads));
    const bool stream = p.stream != 0u;
    if (one && stream) k_step_slice<V, kMinBlocks, true, true><<<grid, kSliceThreads, 0, s>>>(p, tab);
    else if (one) k_step_slice<V, kMinBlocks, true, false><<<grid, kSliceThreads, 0, s>>>(p, tab);
    else if (stream) k_step_slice<V, kMinBlocks, false, true><<<grid, kSliceThreads, 0, s>>>(p, tab);
    else k_step_slice<V, kMinBlocks, false, false><<<grid, kSliceThreads, 0, s>>>(p, tab);
}

// Slice-kernel variants 0-5: k_step_slice with (nodes per thread, minimum
// CTAs of 256 threads per SM, i.e. a register bound); variants 6-9: the
// warp-specialised k_step_slice_ws with (consumer warps, stages, minimum CTAs
// per SM), 4 nodes per consumer thread; variants 10-13: the grid-stride
// k_step_slice_loop with (nodes per thread, minimum CTAs of 256 threads per
// SM); variants 14-19: the temporally blocked k_step_slice_tb (configurations
// 0-5), which the step loop drives several steps per launch.  Variants 6-19
// apply to single-replica launches (a launch over several replicas takes
// variant 4 instead).  The autotuner picks one per handle; every variant gives
// the same bits.
static const uint32_t kSliceVec[kSliceVariants] = {2, 2, 4, 4, 8, 8, 4, 4, 4, 4, 2, 4, 4, 8, 4, 4, 4, 4, 4, 4};

uint32_t slice_variant_vec(uint32_t variant)
{
    return kSliceVec[variant < kSliceVariants ? variant : 0];
}

cudaError_t launch_slice(const PlainArgs &p, bool one, const SliceTables &tab, cudaStream_t s)
{
    if (p.g_end == p.g_begin) return cudaSuccess;
    if (p.variant >= kSliceVariants) return cudaErrorInvalidValue;
    // the single-replica forms; the blocked one treats its replica as periodic,
    // so a block of a larger lattice takes a classic variant
    const bool other = !one || (p.variant >= kSliceTbFirst && p.halo_in);
    const uint32_t v = (other && p.variant >= kSliceClassicVariants) ? 4u : p.variant;
    cudaError_t e = cudaSuccess;
    switch (v) {
    case 0: launch_slice_v<2, 8>(p, one, tab, s); break;  // <= 32 registers
    case 1: launch_slice_v<2, 6>(p, one, tab, s); break;  // <= 40 registers
    case 2: launch_slice_v<4, 5>(p, one, tab, s); break;  // <= 48 registers
    case 3: launch_slice_v<4, 4>(p, one, tab, s); break;  // <= 64 registers
    case 4: launch_slice_v<8, 3>(p, one, tab, s); break;  // <= 80 registers
    case 5: launch_slice_v<8, 2>(p, one, tab, s); break;  // <= 128 registers
    // (consumer warps, nodes per consumer thread, stages, CTAs per SM)
    case 6: e = launch_slice_ws_v<16, 4, 6, 2>(p, tab, s); break;  // <= 60 registers
    case 7: e = launch_slice_ws_v<4, 4, 8, 6>(p, tab, s); break;   // <= 68
    case 8: e = launch_slice_ws_v<8, 4, 6, 4>(p, tab, s); break;   // <= 56
    case 9: e = launch_slice_ws_v<2, 4, 12, 10>(p, tab, s); break; // <= 68
    // grid-stride form: (nodes per thread, minimum CTAs of 256 threads per SM)
    case 10: e = launch_slice_loop_v<2, 6>(p, tab, s); break;  // <= 40 registers
    case 11: e = launch_slice_loop_v<4, 5>(p, tab, s); break;  // <= 48
    case 12: e = launch_slice_loop_v<4, 4>(p, tab, s); break;  // <= 64
    case 13: e = launch_slice_loop_v<8, 3>(p, tab, s); break;  // <= 80
    // temporally blocked form, one step (the step loop gives it more); heavy
    // nodes are collided in place, so no second pass
    default: return launch_slice_tb(p, tab, 1u, v - kSliceTbFirst, s);
    }
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (one) k_step_heavy<true><<<kHeavyBlocks, kPlainThreads, 0, s>>>(p, tab);
    else k_step_heavy<false><<<kHeavyBatchBlocks, kPlainThreads, 0, s>>>(p, tab);
    return cudaGetLastError();
}

}  // namespace mclg

namespace mclg {

template <int KR, bool kRed>
static void launch_slice_stats_v(const PlainArgs &p, const SliceTables &tab, const StatsArgs &sa,
                                 cudaStream_t s)
{
    const uint32_t Pn = (p.one_L + 7u) & ~7u;
    const dim3 grid((Pn + 63u) / 64u, (sa.R + 8u * KR - 1u) / (8u * KR));
    if (p.stream) k_step_slice_stats<KR, kRed, true><<<grid, 256, 0, s>>>(p, tab, sa);
    else k_step_slice_stats<KR, kRed, false><<<grid, 256, 0, s>>>(p, tab, sa);
}

// Statistics-form configurations (replicas per warp, shared-memory counter
// updates as reductions or as load-add-store), chosen by the autotuner.
cudaError_t launch_slice_stats(const PlainArgs &p, const SliceTables &tab, const StatsArgs &sa,
                               cudaStream_t s)
{
    switch (sa.config) {
    case 0: launch_slice_stats_v<4, false>(p, tab, sa, s); break;
    case 1: launch_slice_stats_v<8, false>(p, tab, sa, s); break;
    case 2: launch_slice_stats_v<4, true>(p, tab, sa, s); break;
    default: launch_slice_stats_v<8, true>(p, tab, sa, s); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the heavy-node pass runs over the whole range of replicas
    if (p.g_end == p.g_begin) return cudaSuccess;
    k_step_heavy<false><<<kHeavyBlocks, kPlainThreads, 0, s>>>(p, tab);
    return cudaGetLastError();
}

}  // namespace mclg
