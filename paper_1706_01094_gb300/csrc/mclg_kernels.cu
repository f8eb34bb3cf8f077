// sm_103a kernels of the D1Q3 Monte Carlo Lattice Gas time step (Sec. III).
//
// Device state layout ("pre-streamed" form).  Each of the three planes
// (v = -1, 0, +1) is a uint16 array of P nodes; replica k of the internal
// order occupies [off_k, off_k + L_k) with off_k a multiple of 8 (16-byte
// aligned vectors), padding nodes hold 0.  A buffer B holds the occupations
// one streaming step *before* the canonical pre-collision field: the field of
// the paper's evolution equation is n_i(x, t) = B_i(x - v_i), i.e.
//     n_-1(x) = B_-1(x + 1),  n_0(x) = B_0(x),  n_+1(x) = B_+1(x - 1)
// (periodic).  One time step is then a pull: read the three streamed values
// of node x, run the C sub-collisions of time t, write the post-collision
// values back to node x of the other buffer.  Every read is a coalesced
// vector load plus two halo values per warp, every write an aligned vector
// store.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mclg_device.cuh"
#include "mclg_internal.h"
#include "mclg_slice.cuh"

namespace mclg {


// ---------------------------------------------------------------------------
// Plain kernel: one thread per V consecutive nodes, any set of whole replicas
// laid out contiguously (node range [8 g_begin, 8 g_end)).  kOne: a single
// replica whose offset, length and id come from the arguments (no tables).
// ---------------------------------------------------------------------------
template <int V, int kMinBlocks, bool kOne>
__global__ void __launch_bounds__(kPlainThreads, kMinBlocks)
    k_step_plain(PlainArgs p)
{
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
    const uint32_t x0 = uint32_t(node0 - off);  // replica-local

    const uint16_t *__restrict__ inm = p.in;
    const uint16_t *__restrict__ in0 = p.in + p.P;
    const uint16_t *__restrict__ inp = p.in + 2 * p.P;

    // Halo: the v = -1 value right of the vector and the v = +1 value left of it.
    // Lanes at a warp or replica edge load theirs directly, issued together with
    // the vector loads (the addresses do not depend on loaded data); the others
    // take them from the neighbouring lanes.
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
    const uint32_t e = x0 >= L ? 0u : (L - x0 < uint32_t(V) ? L - x0 : uint32_t(V));
    const uint32_t t = p.t_dev ? *p.t_dev + p.t : p.t;

    uint32_t err = 0;
    uint32_t om[V], o0[V], op[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        uint32_t a, b, c;
        if (kStream) {
            a = (uint32_t(j) + 1u < e) ? em[(j + 1) % V] : nxt;
            b = e0[j];
            c = (j > 0) ? ep[(j + V - 1) % V] : prv;
        } else {
            a = em[j];
            b = e0[j];
            c = ep[j];
        }
        if (uint32_t(j) < e) {
            const NodeKey nk{p.x_base + x0 + uint32_t(j), rid + p.r0, t, p.k0, p.k1};
            uint32_t ln, ld;
            node_rate(p.galilean != 0u, a, b, c, p.lam_n, p.lam_d, ln, ld);
            collide_node(a, b, c, nk, p.rk, p.C, ln, ld, err);
        } else {
            a = b = c = 0u;
        }
        om[j] = a;
        o0[j] = b;
        op[j] = c;
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
}

// ---------------------------------------------------------------------------
// Persistent kernel: each CTA takes work units (runs of whole replicas of at
// most `cap` padded nodes, largest first) from an atomic counter and keeps a
// unit in shared memory for all n_steps steps.  Two shared buffers alternate;
// one barrier per step.  Each thread updates node pairs (2i, 2i+1), which never
// straddle a replica because replicas start on multiples of 8 nodes.  kSlice:
// the slice sampler (one table draw per node for masses up to the tables'
// n_max, the node pair's top bits from one word of its eight-node group's
// Philox block; the sequential draws above it).
// ---------------------------------------------------------------------------
template <int kMinBlocks, bool kSlice>
__global__ void __launch_bounds__(kPersistentMaxThreads, kMinBlocks) k_step_persistent(PersistentArgs p)
{
    const bool kStream = p.stream != 0u;
    extern __shared__ __align__(16) uint16_t smem[];
    __shared__ uint32_t s_lo[kMaxUnitReplicas + 1];  // unit-local replica starts
    __shared__ uint32_t s_L[kMaxUnitReplicas];
    __shared__ uint32_t s_rid[kMaxUnitReplicas];
    __shared__ uint32_t s_unit;

    uint16_t *buf[2] = {smem, smem + 3 * size_t(p.cap)};
    uint32_t err = 0;
    for (;;) {
        __syncthreads();  // the previous unit is written back before the tables change
        if (threadIdx.x == 0) s_unit = atomicAdd(p.unit_counter, 1u);
        __syncthreads();
        const uint32_t ui = s_unit;
        if (ui >= p.n_units) break;
        const Unit u = p.units[ui];
        const uint32_t nn = u.nodes;  // padded nodes of this unit (multiple of 8)
        const uint32_t nrep = u.rep_end - u.rep_begin;
        for (uint32_t k = threadIdx.x; k < nrep; k += blockDim.x) {
            const uint32_t kk = u.rep_begin + k;
            s_lo[k] = uint32_t(p.rep_off[kk] - u.node_begin);
            s_L[k] = p.rep_L[kk];
            s_rid[k] = p.rep_id[kk];
        }
        if (threadIdx.x == 0) s_lo[nrep] = nn;
        // Load the unit: 3 planes x nn nodes, 16-byte vectors.
        for (uint32_t v = threadIdx.x; v < 3u * (nn / 8u); v += blockDim.x) {
            const uint32_t plane = v / (nn / 8u), w = v % (nn / 8u);
            const uint4 val = *reinterpret_cast<const uint4 *>(p.in + plane * p.P + u.node_begin +
                                                               8u * w);
            *reinterpret_cast<uint4 *>(buf[0] + plane * p.cap + 8u * w) = val;
        }
        __syncthreads();

        int cur = 0;
        for (uint32_t s = 0; s < p.n_steps; ++s) {
            const uint32_t t = p.t0 + s;
            const uint16_t *bm = buf[cur], *bz = buf[cur] + p.cap, *bp = buf[cur] + 2 * p.cap;
            uint16_t *om = buf[cur ^ 1], *oz = buf[cur ^ 1] + p.cap, *op = buf[cur ^ 1] + 2 * p.cap;
            for (uint32_t i = 2u * threadIdx.x; i < nn; i += 2u * blockDim.x) {
                // replica of node i: largest k with s_lo[k] <= i
                uint32_t lo = 0, hi = nrep;
                while (hi - lo > 1u) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (s_lo[mid] <= i) lo = mid; else hi = mid;
                }
                const uint32_t base = s_lo[lo], L = s_L[lo], x = i - base;
                const bool v0 = x < L, v1 = x + 1u < L;  // padding nodes stay 0
                const uint32_t bpair = *reinterpret_cast<const uint32_t *>(bz + i);
                uint32_t a0, c0, a1, c1;
                if (kStream) {
                    a0 = v0 ? bm[base + (x + 1u < L ? x + 1u : 0u)] : 0u;
                    c0 = v0 ? bp[base + (x > 0u ? x - 1u : L - 1u)] : 0u;
                    a1 = v1 ? bm[base + (x + 2u < L ? x + 2u : 0u)] : 0u;
                    c1 = v1 ? bp[base + x] : 0u;
                } else {
                    a0 = v0 ? bm[i] : 0u;
                    c0 = v0 ? bp[i] : 0u;
                    a1 = v1 ? bm[i + 1] : 0u;
                    c1 = v1 ? bp[i + 1] : 0u;
                }
                uint32_t b0 = v0 ? lo16(bpair) : 0u, b1 = v1 ? hi16(bpair) : 0u;
                const uint32_t rid = s_rid[lo] + p.r0;
                const NodeKey nk0{x, rid, t, p.k0, p.k1};
                const NodeKey nk1{x + 1u, rid, t, p.k0, p.k1};
                uint32_t ln, ld;
                bool seq0 = true, seq1 = true;
                if (kSlice) {
                    // the node pair's table draws (x is even: both nodes' top bits are
                    // the two halves of one word of their eight-node group's block)
                    uint32_t a2[2] = {a0, a1}, b2[2] = {b0, b1}, c2[2] = {c0, c1};
                    const uint32_t heavy =
                        slice_draws<2>(a2, b2, c2, x, rid, t, p.rk, p.k0, p.k1, p.tab, p.C, err);
                    a0 = a2[0]; b0 = b2[0]; c0 = c2[0];
                    a1 = a2[1]; b1 = b2[1]; c1 = c2[1];
                    seq0 = heavy & 1u;
                    seq1 = (heavy >> 1) & 1u;
                }
                if (seq0) {
                    node_rate(p.galilean != 0u, a0, b0, c0, p.lam_n, p.lam_d, ln, ld);
                    collide_node(a0, b0, c0, nk0, p.rk, p.C, ln, ld, err);
                }
                if (seq1) {
                    node_rate(p.galilean != 0u, a1, b1, c1, p.lam_n, p.lam_d, ln, ld);
                    collide_node(a1, b1, c1, nk1, p.rk, p.C, ln, ld, err);
                }
                *reinterpret_cast<uint32_t *>(om + i) = a0 | (a1 << 16);
                *reinterpret_cast<uint32_t *>(oz + i) = b0 | (b1 << 16);
                *reinterpret_cast<uint32_t *>(op + i) = c0 | (c1 << 16);
            }
            cur ^= 1;
            __syncthreads();
        }
        for (uint32_t v = threadIdx.x; v < 3u * (nn / 8u); v += blockDim.x) {
            const uint32_t plane = v / (nn / 8u), w = v % (nn / 8u);
            const uint4 val = *reinterpret_cast<const uint4 *>(buf[cur] + plane * p.cap + 8u * w);
            *reinterpret_cast<uint4 *>(p.out + plane * p.P + u.node_begin + 8u * w) = val;
        }
    }
    flag_error(p.err, err);
}

// ---------------------------------------------------------------------------
// Layout conversions between the ABI field n[3][S] (canonical, replica order)
// and the pre-streamed device form, and the node moments.  One thread per
// 8-node chunk of the device form: the replica tables are read once per
// chunk, the device side moves 16-byte vectors, the ABI side (arbitrary
// offsets) moves uint16 values, consecutive across the warp.
// ---------------------------------------------------------------------------
struct ChunkInfo {
    uint64_t base;  // device-form offset of the replica
    uint64_t a0;    // ABI offset of the replica
    uint32_t L, x0; // replica length, replica-local first node of the chunk
};

__device__ __forceinline__ ChunkInfo chunk_info(uint64_t g, const uint64_t *abi_off,
                                                const uint64_t *rep_off, const uint32_t *rep_L,
                                                const uint32_t *chunk_rep, const uint32_t *rep_id)
{
    const uint32_t k = chunk_rep[g];
    ChunkInfo c;
    c.base = rep_off[k];
    c.L = rep_L[k];
    c.a0 = abi_off[rep_id[k]];
    c.x0 = uint32_t(g * 8u - c.base);
    return c;
}

__global__ void k_to_device_form(const uint16_t *__restrict__ n, uint64_t S, uint16_t *__restrict__ B,
                                 uint64_t P, const uint64_t *__restrict__ abi_off,
                                 const uint64_t *__restrict__ rep_off, const uint32_t *__restrict__ rep_L,
                                 const uint32_t *__restrict__ chunk_rep, uint64_t chunks,
                                 const uint32_t *__restrict__ rep_id, int stream)
{
    const uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= chunks) return;
    const ChunkInfo c = chunk_info(g, abi_off, rep_off, rep_L, chunk_rep, rep_id);
    uint32_t em[8], ez[8], ep[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t y = c.x0 + uint32_t(j);
        if (y < c.L) {
            // B_-1(y) = n_-1(y - 1), B_0(y) = n_0(y), B_+1(y) = n_+1(y + 1)
            const uint32_t ym = stream ? (y == 0u ? c.L - 1u : y - 1u) : y;
            const uint32_t yp = stream ? (y + 1u == c.L ? 0u : y + 1u) : y;
            em[j] = n[c.a0 + ym];
            ez[j] = n[S + c.a0 + y];
            ep[j] = n[2 * S + c.a0 + yp];
        } else {
            em[j] = ez[j] = ep[j] = 0u;  // padding
        }
    }
    uint4 v;
    pack(em, v);
    *reinterpret_cast<uint4 *>(B + g * 8u) = v;
    pack(ez, v);
    *reinterpret_cast<uint4 *>(B + P + g * 8u) = v;
    pack(ep, v);
    *reinterpret_cast<uint4 *>(B + 2 * P + g * 8u) = v;
}

__global__ void k_from_device_form(const uint16_t *__restrict__ B, uint64_t P, uint16_t *__restrict__ n,
                                   uint64_t S, const uint64_t *__restrict__ abi_off,
                                   const uint64_t *__restrict__ rep_off, const uint32_t *__restrict__ rep_L,
                                   const uint32_t *__restrict__ chunk_rep, uint64_t chunks,
                                   const uint32_t *__restrict__ rep_id, int stream,
                                   const uint16_t *__restrict__ halo)
{
    const uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= chunks) return;
    const ChunkInfo c = chunk_info(g, abi_off, rep_off, rep_L, chunk_rep, rep_id);
    uint32_t ez[8];
    unpack(*reinterpret_cast<const uint4 *>(B + P + g * 8u), ez);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t x = c.x0 + uint32_t(j);
        if (x < c.L) {
            const uint32_t xr = stream ? (x + 1u == c.L ? 0u : x + 1u) : x;
            const uint32_t xl = stream ? (x == 0u ? c.L - 1u : x - 1u) : x;
            // a block of a larger lattice: its edges' arriving values come from the halo
            n[c.a0 + x] = (halo && stream && x + 1u == c.L) ? halo[1] : B[c.base + xr];
            n[S + c.a0 + x] = uint16_t(ez[j]);
            n[2 * S + c.a0 + x] = (halo && stream && x == 0u) ? halo[0] : B[2 * P + c.base + xl];
        }
    }
}

// Node moments N = a + b + c, J = c - a of the canonical field, in ABI order,
// and exact int64 totals (block partial sums, then one 64-bit atomic each).
__global__ void k_moments(const uint16_t *__restrict__ B, uint64_t P, int32_t *__restrict__ N,
                          int32_t *__restrict__ J, const uint64_t *__restrict__ abi_off,
                          const uint64_t *__restrict__ rep_off, const uint32_t *__restrict__ rep_L,
                          const uint32_t *__restrict__ chunk_rep, uint64_t chunks,
                          const uint32_t *__restrict__ rep_id, int stream,
                          const uint16_t *__restrict__ halo, unsigned long long *__restrict__ totals)
{
    const uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    long long sn = 0, sj = 0;
    if (g < chunks) {
        const ChunkInfo c = chunk_info(g, abi_off, rep_off, rep_L, chunk_rep, rep_id);
        uint32_t ez[8];
        unpack(*reinterpret_cast<const uint4 *>(B + P + g * 8u), ez);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t x = c.x0 + uint32_t(j);
            if (x < c.L) {
                const uint32_t xr = stream ? (x + 1u == c.L ? 0u : x + 1u) : x;
                const uint32_t xl = stream ? (x == 0u ? c.L - 1u : x - 1u) : x;
                const int32_t a = (halo && stream && x + 1u == c.L) ? halo[1] : B[c.base + xr];
                const int32_t b = int32_t(ez[j]);
                const int32_t cc = (halo && stream && x == 0u) ? halo[0] : B[2 * P + c.base + xl];
                const uint64_t o = c.a0 + x;
                if (N) N[o] = a + b + cc;
                if (J) J[o] = cc - a;
                sn += a + b + cc;
                sj += cc - a;
            }
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        sn += __shfl_down_sync(0xFFFFFFFFu, sn, d);
        sj += __shfl_down_sync(0xFFFFFFFFu, sj, d);
    }
    __shared__ long long ws[2][32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { ws[0][w] = sn; ws[1][w] = sj; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tn = 0, tj = 0;
        for (int k = 0; k < int(blockDim.x >> 5); ++k) { tn += ws[0][k]; tj += ws[1][k]; }
        atomicAdd(&totals[0], (unsigned long long)tn);
        atomicAdd(&totals[1], (unsigned long long)tj);
    }
}

// Ensemble statistics of the canonical field, per replica-local position x,
// pooled over R equal-length replicas (contiguous, offset stride `stride`).
// Pass 1: a block covers 32 positions x (blockDim / 32) replica groups of one
// replica slice and adds its partial sums (18 per position) to the step's
// batch sums batch[x][18] with 64-bit integer atomics (exact, so the result
// does not depend on their order).  Pass 2 (k_stats_merge): one thread per
// position adds the batch to the int64 accumulators, merges it into the FP32
// running means and co-moments and clears it for the next step.
constexpr int kStatQ = 18;  // 3 sums + 6 products + 9 neighbour products

__global__ void __launch_bounds__(256) k_stats_partial(const uint16_t *__restrict__ B, uint64_t P,
                                                       uint32_t L, uint32_t R, uint64_t stride,
                                                       int stream, uint32_t slices,
                                                       unsigned long long *__restrict__ batch,
                                                       unsigned long long *__restrict__ batch_count)
{
    const uint32_t xl = threadIdx.x & 31u, grp = threadIdx.x >> 5, ngrp = blockDim.x >> 5;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
        atomicAdd(batch_count, (unsigned long long)R);  // one sample of every replica
    const uint32_t x = blockIdx.x * 32u + xl;
    const uint32_t slice = blockIdx.y;
    const uint32_t r_begin = uint32_t(uint64_t(R) * slice / slices);
    const uint32_t r_end = uint32_t(uint64_t(R) * (slice + 1) / slices);
    __shared__ unsigned long long red[8][32][kStatQ + 1];  // <= 8 groups; +1 avoids bank conflicts
    unsigned long long *mine = red[grp][xl];
#pragma unroll
    for (int q = 0; q < kStatQ; ++q) mine[q] = 0ull;
    if (x < L) {
        const uint32_t x1 = x + 1u == L ? 0u : x + 1u;  // neighbour position
        const uint32_t xr = stream ? (x + 1u == L ? 0u : x + 1u) : x;
        const uint32_t xlft = stream ? (x == 0u ? L - 1u : x - 1u) : x;
        const uint32_t x1r = stream ? (x1 + 1u == L ? 0u : x1 + 1u) : x1;
        const uint32_t x1l = stream ? (x1 == 0u ? L - 1u : x1 - 1u) : x1;
        // At most 16 replicas per thread (the launch sizes the slices so): with
        // every value below 2^14 each product is below 2^28 and 16 of them fit
        // 32 bits, so the sums run in 32-bit multiply-adds; a thread that saw a
        // larger value redoes its replicas with 64-bit sums (in shared memory).
        uint32_t a32[kStatQ];
#pragma unroll
        for (int q = 0; q < kStatQ; ++q) a32[q] = 0u;
        uint32_t big = 0;
#pragma unroll 4
        for (uint32_t r = r_begin + grp; r < r_end; r += ngrp) {
            const uint16_t *row = B + r * stride;
            const uint32_t v0 = row[xr], v1 = row[P + x], v2 = row[2 * P + xlft];
            const uint32_t w0 = row[x1r], w1 = row[P + x1], w2 = row[2 * P + x1l];
            big |= v0 | v1 | v2 | w0 | w1 | w2;
            a32[0] += v0; a32[1] += v1; a32[2] += v2;
            a32[3] += v0 * v0; a32[4] += v0 * v1; a32[5] += v0 * v2;
            a32[6] += v1 * v1; a32[7] += v1 * v2; a32[8] += v2 * v2;
            a32[9] += v0 * w0; a32[10] += v0 * w1; a32[11] += v0 * w2;
            a32[12] += v1 * w0; a32[13] += v1 * w1; a32[14] += v1 * w2;
            a32[15] += v2 * w0; a32[16] += v2 * w1; a32[17] += v2 * w2;
        }
        if (big < (1u << 14)) {
#pragma unroll
            for (int q = 0; q < kStatQ; ++q) mine[q] = a32[q];
        } else {
            for (uint32_t r = r_begin + grp; r < r_end; r += ngrp) {
                const uint16_t *row = B + r * stride;
                const uint64_t v[3] = {row[xr], row[P + x], row[2 * P + xlft]};
                const uint64_t w[3] = {row[x1r], row[P + x1], row[2 * P + x1l]};
                for (int i = 0; i < 3; ++i) mine[i] += v[i];
                int q = 3;
                for (int i = 0; i < 3; ++i)
                    for (int j = i; j < 3; ++j) mine[q++] += v[i] * v[j];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) mine[q++] += v[i] * w[j];
            }
        }
    }
    __syncthreads();
    if (grp != 0 || x >= L) return;
    unsigned long long acc[kStatQ];
#pragma unroll
    for (int q = 0; q < kStatQ; ++q) acc[q] = mine[q];
    for (uint32_t g2 = 1; g2 < ngrp; ++g2)
#pragma unroll
        for (int q = 0; q < kStatQ; ++q) acc[q] += red[g2][xl][q];
    unsigned long long *out = batch + uint64_t(x) * kStatQ;
#pragma unroll
    for (int q = 0; q < kStatQ; ++q) atomicAdd(out + q, acc[q]);
}

// Pass 2: thread (position, quantity) adds its batch sum to the int64
// accumulator and clears it; then one thread per position merges the batch
// into the FP32 running means and co-moments (Chan et al.), with Kahan
// compensation, reading the batch from shared memory.  count[0] holds the
// samples per position so far, count[1] is the blocks' finishing ticket and
// count[2] the samples in the batch (added by the passes that filled it).
constexpr uint32_t kMergePositions = 14;  // 14 x 18 = 252 threads per block

__global__ void __launch_bounds__(256) k_stats_merge(unsigned long long *__restrict__ batch,
                                                     uint32_t L, StatsBuffers st)
{
    __shared__ long long sb[kMergePositions][kStatQ];
    const uint64_t n = *(volatile unsigned long long *)(st.count + 2);  // samples in this batch
    const uint32_t lp = threadIdx.x / kStatQ, q = threadIdx.x % kStatQ;
    const uint32_t x = blockIdx.x * kMergePositions + lp;
    if (lp < kMergePositions && x < L) {
        unsigned long long *in = batch + uint64_t(x) * kStatQ + q;
        const long long v = (long long)*in;
        *in = 0ull;
        sb[lp][q] = v;
        if (q < 3) st.s1[3u * x + q] += v;
        else if (q < 9) st.s2[6u * x + (q - 3)] += v;
        else st.snb[9u * x + (q - 9)] += v;
    }
    __syncthreads();
    const uint32_t xm = blockIdx.x * kMergePositions + threadIdx.x;
    if (threadIdx.x < kMergePositions && xm < L && n > 0u) {
        const long long *acc = sb[threadIdx.x];
        // the merge weights from the exact integer counts, rounded to FP32 once
        // (so they stay exact to FP32 rounding beyond 2^24 samples per position)
        const uint64_t na = *st.count;  // samples per position before this batch
        const float Rb = float(n);      // samples per position in this batch (divisor of exact sums)
        const float wb = float(double(n) / double(na + n));                 // Rb / Mt
        const float wab = float(double(na) * double(n) / double(na + n));   // Ma Rb / Mt
        float delta[3];
        for (int i = 0; i < 3; ++i) {
            const float mb = float(acc[i]) / Rb;
            const float m = st.mean32[3u * xm + i];
            delta[i] = mb - m;
            const float inc = delta[i] * wb - st.mean32c[3u * xm + i];
            const float nm = m + inc;
            st.mean32c[3u * xm + i] = (nm - m) - inc;
            st.mean32[3u * xm + i] = nm;
        }
        const int pi[6] = {0, 0, 0, 1, 1, 2}, pj[6] = {0, 1, 2, 1, 2, 2};
        for (int k = 0; k < 6; ++k) {
            const int i = pi[k], j = pj[k];
            // batch co-moment sum (n_i - mb_i)(n_j - mb_j) = (n s_ij - s_i s_j) / n, exact numerator
            const __int128 num = (__int128)n * acc[3 + k] - (__int128)acc[i] * acc[j];
            const float cb = float(num) / Rb;
            const float inc = cb + delta[i] * delta[j] * wab - st.m2c[6u * xm + k];
            const float m2 = st.m2[6u * xm + k];
            const float nm2 = m2 + inc;
            st.m2c[6u * xm + k] = (nm2 - m2) - inc;
            st.m2[6u * xm + k] = nm2;
        }
    }
    // the last block to finish, after every block has read the count, adds
    // this batch's n samples to it
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(st.count + 1, 1ull) == gridDim.x - 1u) {
            st.count[0] += n;
            st.count[1] = 0ull;
            st.count[2] = 0ull;
            __threadfence();
        }
    }
}

__global__ void k_set_time(uint32_t *t_dev, uint32_t value) { *t_dev = value; }
__global__ void k_advance_time(uint32_t *t_dev, uint32_t by) { *t_dev += by; }

__global__ void k_philox(const uint4 *__restrict__ ctr, uint64_t n, uint32_t k0, uint32_t k1,
                         uint4 *__restrict__ out)
{
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint4 c = ctr[i];
    philox4x32_10(c.x, c.y, c.z, c.w, k0, k1);
    out[i] = c;
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
template <int V, int kMinBlocks>
static void launch_plain_v(const PlainArgs &p, bool one, dim3 grid, cudaStream_t s)
{
    if (one) k_step_plain<V, kMinBlocks, true><<<grid, kPlainThreads, 0, s>>>(p);
    else k_step_plain<V, kMinBlocks, false><<<grid, kPlainThreads, 0, s>>>(p);
}

// Plain-kernel variants: (nodes per thread, minimum CTAs per SM).  More
// nodes per thread give more independent work per thread; a higher CTA bound
// caps registers for occupancy.  The autotuner picks one per handle.
static const uint32_t kVariantVec[kPlainVariants] = {1, 1, 2, 2, 2, 2};

uint32_t plain_variant_vec(uint32_t variant)
{
    return kVariantVec[variant < kPlainVariants ? variant : 0];
}

cudaError_t launch_plain(const PlainArgs &p, bool one, cudaStream_t s)
{
    const uint64_t chunks = p.g_end - p.g_begin;
    if (chunks == 0) return cudaSuccess;
    if (p.variant >= kPlainVariants) return cudaErrorInvalidValue;
    const uint32_t V = plain_variant_vec(p.variant);
    const uint64_t threads = chunks * (8u / V);
    const dim3 grid(uint32_t((threads + kPlainThreads - 1) / kPlainThreads));
    switch (p.variant) {
    case 0: launch_plain_v<1, 6>(p, one, grid, s); break;   // <= 40 registers
    case 1: launch_plain_v<1, 8>(p, one, grid, s); break;   // <= 32 registers
    case 2: launch_plain_v<2, 4>(p, one, grid, s); break;   // <= 64 registers
    case 3: launch_plain_v<2, 5>(p, one, grid, s); break;   // <= 51 registers
    case 4: launch_plain_v<2, 6>(p, one, grid, s); break;   // <= 42 registers
    default: launch_plain_v<2, 1>(p, one, grid, s); break;
    }
    return cudaGetLastError();
}

size_t persistent_smem_bytes(uint32_t cap) { return 2u * 3u * size_t(cap) * sizeof(uint16_t); }

// Persistent-kernel variants: minimum CTAs of kPersistentMaxThreads threads
// per SM, i.e. register bounds of 128, 64 and 42 per thread.
template <int kMinBlocks>
static cudaError_t launch_persistent_v(const PersistentArgs &p, uint32_t n_units, uint32_t threads,
                                       cudaStream_t s)
{
    const size_t smem = persistent_smem_bytes(p.cap);
    auto kern = p.slice ? k_step_persistent<kMinBlocks, true> : k_step_persistent<kMinBlocks, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    // as many CTAs as can be resident at once; they pull the units
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, int(threads), smem)) !=
        cudaSuccess)
        return e;
    const uint32_t resident = uint32_t(std::max(1, sms * std::max(per_sm, 1)));
    PersistentArgs a = p;
    a.n_units = n_units;
    if ((e = cudaMemsetAsync(a.unit_counter, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
    kern<<<std::min(n_units, resident), threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_persistent(const PersistentArgs &p, uint32_t n_units, uint32_t threads,
                              cudaStream_t s)
{
    if (n_units == 0) return cudaSuccess;
    switch (p.variant) {
    case 0: return launch_persistent_v<1>(p, n_units, threads, s);
    case 1: return launch_persistent_v<2>(p, n_units, threads, s);
    default: return launch_persistent_v<3>(p, n_units, threads, s);
    }
}

cudaError_t launch_to_device_form(const uint16_t *n, uint64_t S, uint16_t *B, const Layout &lay,
                                  int stream, cudaStream_t s)
{
    const uint64_t chunks = lay.P / 8u;
    const uint32_t th = 256;
    k_to_device_form<<<uint32_t((chunks + th - 1) / th), th, 0, s>>>(
        n, S, B, lay.P, lay.d_abi_off, lay.d_rep_off, lay.d_rep_L, lay.d_chunk_rep, chunks,
        lay.d_rep_id, stream);
    return cudaGetLastError();
}

cudaError_t launch_from_device_form(const uint16_t *B, uint16_t *n, uint64_t S, const Layout &lay,
                                    int stream, const uint16_t *halo, cudaStream_t s)
{
    const uint64_t chunks = lay.P / 8u;
    const uint32_t th = 256;
    k_from_device_form<<<uint32_t((chunks + th - 1) / th), th, 0, s>>>(
        B, lay.P, n, S, lay.d_abi_off, lay.d_rep_off, lay.d_rep_L, lay.d_chunk_rep, chunks,
        lay.d_rep_id, stream, halo);
    return cudaGetLastError();
}

cudaError_t launch_moments(const uint16_t *B, int32_t *N, int32_t *J, const Layout &lay, int stream,
                           const uint16_t *halo, unsigned long long *totals, cudaStream_t s)
{
    const uint64_t chunks = lay.P / 8u;
    const uint32_t th = 256;
    k_moments<<<uint32_t((chunks + th - 1) / th), th, 0, s>>>(
        B, lay.P, N, J, lay.d_abi_off, lay.d_rep_off, lay.d_rep_L, lay.d_chunk_rep, chunks,
        lay.d_rep_id, stream, halo, totals);
    return cudaGetLastError();
}

// Replica slices of the partial-sum pass: each of its 8 thread groups takes at
// most kStatReplicas replicas of a slice (<= 16, the bound its 32-bit sums rely
// on; 4 measured slower on the statistics workload: the atomics outweigh the
// extra CTAs).
constexpr uint32_t kStatReplicas = 16;
uint32_t stats_slices(uint32_t R) { return std::max<uint32_t>(1u, (R + 8u * kStatReplicas - 1u) / (8u * kStatReplicas)); }

size_t stats_partials_bytes(uint32_t L, uint32_t R)
{
    (void)R;
    return size_t(L) * kStatQ * sizeof(unsigned long long);
}

cudaError_t launch_stats_partial(const uint16_t *B, uint64_t P, uint32_t L, uint32_t R,
                                 uint64_t stride, int stream, unsigned long long *batch,
                                 unsigned long long *batch_count, cudaStream_t s)
{
    const uint32_t slices = stats_slices(R);
    const dim3 grid((L + 31) / 32, slices);
    k_stats_partial<<<grid, 256, 0, s>>>(B, P, L, R, stride, stream, slices, batch, batch_count);
    return cudaGetLastError();
}

cudaError_t launch_stats_merge(unsigned long long *batch, uint32_t L, const StatsBuffers &st,
                               cudaStream_t s)
{
    k_stats_merge<<<(L + kMergePositions - 1) / kMergePositions, 256, 0, s>>>(batch, L, st);
    return cudaGetLastError();
}

cudaError_t launch_set_time(uint32_t *t_dev, uint32_t value, cudaStream_t s)
{
    k_set_time<<<1, 1, 0, s>>>(t_dev, value);
    return cudaGetLastError();
}

cudaError_t launch_advance_time(uint32_t *t_dev, uint32_t by, cudaStream_t s)
{
    k_advance_time<<<1, 1, 0, s>>>(t_dev, by);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, uint64_t n, uint32_t k0, uint32_t k1, uint32_t *out,
                          cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint32_t th = 256;
    k_philox<<<uint32_t((n + th - 1) / th), th, 0, s>>>(reinterpret_cast<const uint4 *>(ctr), n, k0,
                                                          k1, reinterpret_cast<uint4 *>(out));
    return cudaGetLastError();
}

}  // namespace mclg
