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
// vector never straddles two).  Node pair (2i, 2i + 1) shares one Philox
// block: node 2i takes words (0, 1), node 2i + 1 words (2, 3) as Q.  The
// row's guide entry for the top 9 bits of Q gives the count directly unless
// an F[k] falls inside Q's bucket (about 1.6% of nodes near equilibrium); then
// the entry also holds that F[k]'s next 8 bits, which decide Q against it
// unless Q has the same 17 top bits (or several entries share the bucket,
// mostly in the tails): then Q is compared with the row's u64 entries from
// the guide's count on (about 0.5% of nodes near equilibrium).
//
// A node heavier than the tables' n_max takes the sequential sampler's C
// decisions (the bits that sampler gives it) in a second, small pass of the
// same step: the table kernel writes such a node unchanged and appends its
// position to a device list; k_step_heavy collides the listed nodes.  If the
// list overflows, the pass scans the whole range instead: collisions keep N,
// so exactly the heavy nodes have N > n_max after the table kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "mclg_device.cuh"
#include "mclg_internal.h"

namespace mclg {

// One node's table draw.  Returns true, leaving the node as it is, when its
// mass is beyond the tables (the sequential pass collides it).
template <bool kNarrow>
__device__ __forceinline__ bool slice_node(uint32_t &a, uint32_t &b, uint32_t &c, uint32_t lo,
                                           uint32_t hi, const SliceTables &tab, uint32_t C,
                                           uint32_t &err)
{
    const uint32_t N = a + b + c;
    if (N < 2u) return false;
    if (N > tab.n_max) return true;
    const uint32_t Jp = a > c ? a - c : c - a;
    const uint32_t below = (b - ((N - Jp) & 1u)) >> 1;
    const uint32_t row = __ldg(tab.rowstart + N * (tab.n_max + 1u) + Jp) + below;
    // guide entry of Q's bucket; kNarrow: the table's entries are indexed in 32 bits
    const uint32_t bucket = hi >> (32 - kSliceBucketBits);
    const uint32_t e = kNarrow
        ? __ldg(tab.guide + (row * uint32_t(kSliceBuckets) + bucket))
        : __ldg(tab.guide + ((uint64_t(row) << kSliceBucketBits) + bucket));
    uint32_t count = e & 0x1Fu;
    const uint32_t inside = (e >> 5) & 3u;  // entries in Q's bucket (3: three or more)
    const uint32_t qn = (hi >> (24 - kSliceBucketBits)) & 0xFFu, fn = e >> 8;  // Q bits 54..47
    if (inside == 1u && qn != fn) {
        count += qn > fn ? 1u : 0u;  // the next 8 bits decide Q against that entry
    } else if (inside != 0u) {
        // finish on the exact 64-bit values
        const uint32_t above = (N - Jp - b) >> 1;
        const uint32_t nvalid = min(C, above) + min(C, below);  // entries dmin .. dmax - 1
        const uint64_t Q = (uint64_t(hi) << 32) | lo;
        const unsigned long long *F = tab.secondary + uint64_t(row) * kSliceRowU64;
        uint64_t f = 0;
        while (count < nvalid && (f = __ldg(F + count)) < Q) ++count;
        if (count < nvalid && f == Q) {
            err |= kErrSampler;
            return false;
        }
    }
    // d = dmin + count with dmin = -min(C, below): b' = b + 2 d and, with N and
    // J kept, a' = a - d, c' = c - d (arithmetic modulo 2^32)
    const uint32_t d = count - min(C, below);
    a -= d;
    b += 2u * d;
    c -= d;
    return false;
}

// kMinBlocks counts CTAs of 256 threads (the register bound of the variant
// table); the kernel runs CTAs of kSliceThreads.
template <int V, int kMinBlocks, bool kOne, bool kNarrow>
__global__ void __launch_bounds__(kSliceThreads, kMinBlocks * 256 / kSliceThreads)
    k_step_slice(PlainArgs p, SliceTables tab)
{
    static_assert(V == 2 || V == 4 || V == 8, "V nodes per thread: 2, 4 or 8");
    const bool kStream = p.stream != 0u;
    using T = typename VecT<V>::T;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t v_begin = p.g_begin * (8 / V), v_end = p.g_end * (8 / V);
    const uint64_t g = v_begin + uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool active = g < v_end;
    const uint64_t gv = active ? g : v_end - 1;  // idle lanes mirror the last vector
    const uint64_t node0 = gv * V;

    uint64_t off;
    uint32_t L, rid;
    if (kOne) {
        off = p.one_off;
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
    if (kStream && own_next) nxt_own = inm[off + (x0 + V < L ? x0 + V : 0u)];
    if (kStream && own_prev) prv_own = inp[off + (x0 > 0u ? x0 - 1u : L - 1u)];
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

    uint32_t err = 0, heavy = 0;
    uint32_t om[V], o0[V], op[V];
#pragma unroll
    for (int i = 0; i < V / 2; ++i) {
        uint32_t w0 = (x0 >> 1) + uint32_t(i), w1 = rid + p.r0, w2 = t, w3 = kPurposeSlice << 28;
        philox4x32_10(w0, w1, w2, w3, p.rk);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * i + h;
            // pre-collision occupations n_i(x) = B_i(x - v_i); padding stays empty
            uint32_t a, b, c;
            if (kStream) {
                a = (uint32_t(j) + 1u < nv) ? em[(j + 1) % V] : nxt;
                c = (j > 0) ? ep[(j + V - 1) % V] : prv;
            } else {
                a = em[j];
                c = ep[j];
            }
            b = e0[j];
            if (uint32_t(j) >= nv) a = b = c = 0u;
            if (slice_node<kNarrow>(a, b, c, h ? w2 : w0, h ? w3 : w1, tab, p.C, err))
                heavy |= 1u << j;
            om[j] = a;
            o0[j] = b;
            op[j] = c;
        }
    }
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
    // heavy nodes (written unchanged) join the list of the sequential pass:
    // one atomic per warp and node slot that has any
    if (!active) heavy = 0u;
    if (__any_sync(0xFFFFFFFFu, heavy != 0u)) {
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
        const NodeKey nk{x, rid + p.r0, t, p.k0, p.k1};
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
    if (tab.guide_narrow) {
        if (one) k_step_slice<V, kMinBlocks, true, true><<<grid, kSliceThreads, 0, s>>>(p, tab);
        else k_step_slice<V, kMinBlocks, false, true><<<grid, kSliceThreads, 0, s>>>(p, tab);
    } else {
        if (one) k_step_slice<V, kMinBlocks, true, false><<<grid, kSliceThreads, 0, s>>>(p, tab);
        else k_step_slice<V, kMinBlocks, false, false><<<grid, kSliceThreads, 0, s>>>(p, tab);
    }
}

// Slice-kernel variants: (nodes per thread, minimum CTAs of 256 threads per
// SM, i.e. a register bound).  The autotuner picks one per handle.
static const uint32_t kSliceVec[kSliceVariants] = {2, 2, 4, 4, 8, 8};

uint32_t slice_variant_vec(uint32_t variant)
{
    return kSliceVec[variant < kSliceVariants ? variant : 0];
}

cudaError_t launch_slice(const PlainArgs &p, bool one, const SliceTables &tab, cudaStream_t s)
{
    if (p.g_end == p.g_begin) return cudaSuccess;
    if (p.variant >= kSliceVariants) return cudaErrorInvalidValue;
    switch (p.variant) {
    case 0: launch_slice_v<2, 8>(p, one, tab, s); break;  // <= 32 registers
    case 1: launch_slice_v<2, 6>(p, one, tab, s); break;  // <= 40 registers
    case 2: launch_slice_v<4, 5>(p, one, tab, s); break;  // <= 48 registers
    case 3: launch_slice_v<4, 4>(p, one, tab, s); break;  // <= 64 registers
    case 4: launch_slice_v<8, 3>(p, one, tab, s); break;  // <= 80 registers
    default: launch_slice_v<8, 2>(p, one, tab, s); break; // <= 128 registers
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (one) k_step_heavy<true><<<kHeavyBlocks, kPlainThreads, 0, s>>>(p, tab);
    else k_step_heavy<false><<<kHeavyBlocks, kPlainThreads, 0, s>>>(p, tab);
    return cudaGetLastError();
}

}  // namespace mclg
