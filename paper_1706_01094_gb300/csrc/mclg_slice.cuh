// The slice sampler's draw of one node (Sec. III: the C sub-collisions of a
// node drawn at once from the exact C-step law of its (N, J) slice, Sec.
// III.A), shared by the per-step slice kernels and the persistent kernel.
//
// A node in state (N, |J|, b) draws d = dmin + #{k : Q > F[k]} with its 64-bit
// uniform Q, F[k] = floor(CDF[dmin + k] 2^64) and dmin = -min(C, b / 2)
// (Q == F[k]: sampler error).  Q's top 16 bits for node x are bits
// [16 (x & 1), 16 (x & 1) + 16) of word (x >> 1) & 3 of Philox block
// (x >> 3, r, t, kPurposeSliceTop << 28), so eight consecutive nodes share one
// block; its low 48 bits are word 0 and the low half of word 1 (even x) or
// words 2 and 3 (odd x) of block (x >> 1, r, t, kPurposeSlice << 28), computed
// only when the record below leaves the draw open.
//
// The kernels decide almost every draw from the state's 16-byte record: the
// top 15 bits t_j of the eight values F[c0 - 4 + j], j = 0..7, c0 = -dmin (0
// where that index is below the row, 0x7FFF where it is past its end), which
// bracket the outcomes d = -3 .. 3.  With q the top 15 bits of Q, q > t_j
// implies Q > F and q < t_j implies Q < F; so if no t_j equals q and q lies
// above t_0 and below t_7, the number g of t_j below q gives d = g - 4 exactly
// (the values below the window are all below Q, those above it all above).
// Otherwise (about 0.2% of nodes near equilibrium: the tails beyond |d| = 3
// and prefix ties) the draw is finished on the row's u64 values.
#pragma once
#include <cstdint>

#include "mclg_device.cuh"
#include "mclg_internal.h"

namespace mclg {

// Record of state (N, |J|, b): (N (n_max + 1) + |J|) (n_max / 2 + 1) + b / 2
// (b has the parity of N - |J|, so b / 2 tells the state within its slice).
__device__ __forceinline__ uint32_t slice_record_index(uint32_t N, uint32_t Jp, uint32_t b,
                                                       const SliceTables &tab)
{
    return (N * (tab.n_max + 1u) + Jp) * tab.rec_hb + (b >> 1);
}

// Count of the record's eight values below q = Q >> 49, in 16-bit lanes of
// four words (lane j: half j & 1 of word j / 2).  Each lane of q2 - w holds
// 2^15 + q - t_j in [1, 2^16), so its bit 15 is set iff q >= t_j; the lane is
// exactly 2^15 iff q == t_j, which subtracting one from it reveals in bit 15.
// `open`: the record leaves the draw undecided.
__device__ __forceinline__ uint32_t slice_record_count(const uint4 &r, uint32_t hi, bool &open)
{
    const uint32_t q2 = ((hi >> 17) * 0x10001u) | 0x80008000u;
    const uint32_t l0 = q2 - r.x, l1 = q2 - r.y, l2 = q2 - r.z, l3 = q2 - r.w;
    const uint32_t ge = (l0 & 0x80008000u) | ((l1 >> 1) & 0x40004000u) |
                        ((l2 >> 2) & 0x20002000u) | ((l3 >> 3) & 0x10001000u);
    const uint32_t tie = ((l0 ^ (l0 - 0x10001u)) | (l1 ^ (l1 - 0x10001u)) |
                          (l2 ^ (l2 - 0x10001u)) | (l3 ^ (l3 - 0x10001u))) & 0x80008000u;
    const uint32_t g = __popc(ge);
    open = tie != 0u || g - 1u >= 7u;
    return g;
}

// The Philox block of the eight-node group holding node x (top 16 bits of Q).
__device__ __forceinline__ void slice_top_block(uint32_t x, uint32_t r, uint32_t t,
                                                const RoundKeys &rk, uint32_t (&w)[4])
{
    w[0] = x >> 3;
    w[1] = r;
    w[2] = t;
    w[3] = kPurposeSliceTop << 28;
    philox4x32_10(w[0], w[1], w[2], w[3], rk);
}

// Word k (0..3) of a block, by selection (no indexed register array).
__device__ __forceinline__ uint32_t pick_word(const uint32_t (&w)[4], uint32_t k)
{
    return (k & 2u) ? ((k & 1u) ? w[3] : w[2]) : ((k & 1u) ? w[1] : w[0]);
}

// Node x's top 16 bits of Q from its group's block.
__device__ __forceinline__ uint32_t slice_top16(const uint32_t (&w)[4], uint32_t x)
{
    const uint32_t word = pick_word(w, (x >> 1) & 3u);
    return (x & 1u) ? word >> 16 : word & 0xFFFFu;
}

// The exact finish on the u64 values of the state's row (the record r left
// the draw open): returns (d, error bits).  Q's low 48 bits come from node x's
// pair block under the seed words (k0, k1).  The record brackets the answer:
// with gt lanes strictly below q and ge lanes at or below it, every entry up
// to index c0 - 5 + gt lies below Q and entry c0 - 4 + ge above it, so the
// count #{k : Q > F[k]} lies in [c0 - 4 + gt, c0 - 4 + ge] (clamped to the
// row); it is found by scanning from the side the record bounds (usually one
// or two loads).  Every argument is passed by value.
__device__ __forceinline__ uint2 slice_exact_body(uint32_t N, uint32_t Jp, uint32_t b,
                                                  uint32_t top16, uint32_t x, uint32_t rr,
                                                  uint32_t t, uint32_t k0, uint32_t k1,
                                                  const uint4 r, const uint32_t *rowstart,
                                                  const unsigned long long *secondary,
                                                  uint32_t n_max, uint32_t C)
{
    uint32_t w0 = x >> 1, w1 = rr, w2 = t, w3 = kPurposeSlice << 28;
    philox4x32_10(w0, w1, w2, w3, k0, k1);
    const bool odd = x & 1u;
    const uint32_t lo = odd ? w2 : w0, hi = (top16 << 16) | ((odd ? w3 : w1) & 0xFFFFu);
    const uint32_t below = b >> 1, above = (N - Jp - b) >> 1;
    const int c0 = int(min(C, below)), nvalid = int(min(C, above)) + c0;
    const uint32_t row = __ldg(rowstart + N * (n_max + 1u) + Jp) + below;
    const unsigned long long *F = secondary + uint64_t(row) * kSliceRowU64;
    const uint64_t Q = (uint64_t(hi) << 32) | lo;
    const uint32_t q = hi >> 17, w[4] = {r.x, r.y, r.z, r.w};
    int gt = 0, ge = 0;  // the lanes ascend, so both are prefixes
#pragma unroll
    for (int j = 0; j < kSliceRecordLanes; ++j) {
        const uint32_t tj = (w[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
        gt += q > tj;
        ge += q >= tj;
    }
    const int kmin = gt > 0 ? max(0, min(nvalid, c0 - 4 + gt)) : 0;
    const int kmax = ge < kSliceRecordLanes ? max(kmin, min(nvalid, c0 - 4 + ge)) : nvalid;
    int count;
    uint64_t f = 0;
    bool seen = false;  // f = F[count] was loaded (and is >= Q)
    if (gt > 0) {
        // upward from the lower bound
        for (count = kmin; count < kmax; ++count) {
            f = __ldg(F + count);
            if (f >= Q) {
                seen = true;
                break;
            }
        }
    } else {
        // downward from the upper bound
        for (count = kmax; count > kmin; --count) {
            const uint64_t g = __ldg(F + count - 1);
            if (g < Q) break;
            f = g;
            seen = true;
        }
    }
    return make_uint2(uint32_t(count - c0), (seen && f == Q) ? kErrSampler : 0u);
}

static __device__ __noinline__ uint2 slice_exact(uint32_t N, uint32_t Jp, uint32_t b,
                                                 uint32_t top16, uint32_t x, uint32_t rr,
                                                 uint32_t t, uint32_t k0, uint32_t k1,
                                                 const uint4 r, const uint32_t *rowstart,
                                                 const unsigned long long *secondary,
                                                 uint32_t n_max, uint32_t C)
{
    return slice_exact_body(N, Jp, b, top16, x, rr, t, k0, k1, r, rowstart, secondary, n_max, C);
}

// Node x's random-number identity: its global index, random-stream index and
// time step, and the seed words.
struct SliceKey {
    uint32_t x, r, t, k0, k1;
};

__device__ __forceinline__ uint32_t slice_exact_d(uint32_t N, uint32_t Jp, uint32_t b,
                                                  uint32_t top16, const SliceKey &key,
                                                  const uint4 &r, const SliceTables &tab,
                                                  uint32_t C, uint32_t &err)
{
    const uint2 de = slice_exact(N, Jp, b, top16, key.x, key.r, key.t, key.k0, key.k1, r,
                                 tab.rowstart, tab.secondary, tab.n_max, C);
    err |= de.y;
    return de.x;
}

// One node's table draw from its top 16 bits.  Returns true, leaving the node
// as it is, when its mass is beyond the tables (the sequential pass collides
// it).  Nodes with N < 2 have identity records (d = 0).
__device__ __forceinline__ bool slice_node(uint32_t &a, uint32_t &b, uint32_t &c, uint32_t top16,
                                           const SliceKey &key, const SliceTables &tab,
                                           uint32_t C, uint32_t &err)
{
    const uint32_t N = a + b + c;
    if (N > tab.n_max) return true;
    const uint32_t Jp = a > c ? a - c : c - a;
    const uint4 r = __ldg(tab.record + slice_record_index(N, Jp, b, tab));
    bool open;
    const uint32_t g = slice_record_count(r, top16 << 16, open);
    // d: b' = b + 2 d and, with N and J kept, a' = a - d, c' = c - d (modulo 2^32)
    const uint32_t d = open ? slice_exact_d(N, Jp, b, top16, key, r, tab, C, err) : g - 4u;
    a -= d;
    b += 2u * d;
    c -= d;
    return false;
}

struct NoHook {
    __device__ void operator()() const {}
};

// The table draws of V consecutive nodes x0 .. x0 + V - 1 (x0 a multiple of
// V; pre-collision a, b, c in registers): the record loads of all V nodes are
// issued first (then `loads_issued` runs), the group block of their top bits
// computed while the loads are in flight, then every record is decoded without
// branches; the draws a record leaves open (rare) are finished afterwards in
// one branch per thread.  Returns a bit per node beyond the tables (left
// unchanged for the sequential pass).
template <int V, typename Hook = NoHook>
__device__ __forceinline__ uint32_t slice_draws(uint32_t (&a)[V], uint32_t (&b)[V], uint32_t (&c)[V],
                                                uint32_t x0, uint32_t r, uint32_t t,
                                                const RoundKeys &rk, uint32_t k0, uint32_t k1,
                                                const SliceTables &tab, uint32_t C, uint32_t &err,
                                                Hook &&loads_issued = Hook())
{
    static_assert(V == 2 || V == 4 || V == 8, "V nodes: 2, 4 or 8");
    uint32_t heavy = 0, open = 0, d[V];
    uint4 rec[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const uint32_t N = a[j] + b[j] + c[j], Jp = a[j] > c[j] ? a[j] - c[j] : c[j] - a[j];
        const bool in = N <= tab.n_max;
        heavy |= uint32_t(!in) << j;
        rec[j] = __ldg(tab.record + (in ? slice_record_index(N, Jp, b[j], tab) : 0u));
    }
    loads_issued();
    uint32_t w[4];
    slice_top_block(x0, r, t, rk, w);
    // the V / 2 words of this thread's nodes: from word (x0 >> 1) & 3 on
    uint32_t u[V / 2];
    if (V == 8) {
#pragma unroll
        for (int i = 0; i < V / 2; ++i) u[i] = w[i];
    } else {
        const uint32_t k = (x0 >> 1) & 3u;
#pragma unroll
        for (int i = 0; i < V / 2; ++i) u[i] = pick_word(w, k + uint32_t(i));
    }
    uint32_t top[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        top[j] = (j & 1) ? u[j >> 1] >> 16 : u[j >> 1] & 0xFFFFu;
        bool o;
        const uint32_t g = slice_record_count(rec[j], top[j] << 16, o);
        const bool in = !((heavy >> j) & 1u);
        d[j] = in ? g - 4u : 0u;
        open |= uint32_t(o && in) << j;
    }
    // the open draws one at a time, inline: the node's values taken by
    // selection, so nothing goes through local memory or a call
    while (open) {
        const uint32_t j = __ffs(open) - 1u;
        open &= open - 1u;
        uint32_t aj = a[0], bj = b[0], cj = c[0], tj = top[0];
        uint4 rj = rec[0];
#pragma unroll
        for (int k = 1; k < V; ++k)
            if (j == uint32_t(k)) {
                aj = a[k];
                bj = b[k];
                cj = c[k];
                tj = top[k];
                rj = rec[k];
            }
        const uint32_t N = aj + bj + cj, Jp = aj > cj ? aj - cj : cj - aj;
        const uint2 de = slice_exact_body(N, Jp, bj, tj, x0 + j, r, t, k0, k1, rj, tab.rowstart,
                                          tab.secondary, tab.n_max, C);
        err |= de.y;
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (j == uint32_t(k)) d[k] = de.x;
    }
#pragma unroll
    for (int j = 0; j < V; ++j) {
        // b' = b + 2 d and, with N and J kept, a' = a - d, c' = c - d (modulo 2^32)
        a[j] -= d[j];
        b[j] += 2u * d[j];
        c[j] -= d[j];
    }
    return heavy;
}

// The same draws for V nodes whose global indices x[j] are arbitrary (a
// thread's nodes straddling the periodic wrap): one group block per node.
template <int V>
__device__ __forceinline__ uint32_t slice_draws_scattered(uint32_t (&a)[V], uint32_t (&b)[V],
                                                          uint32_t (&c)[V],
                                                          const uint32_t (&x)[V], uint32_t r,
                                                          uint32_t t, const RoundKeys &rk,
                                                          uint32_t k0, uint32_t k1,
                                                          const SliceTables &tab, uint32_t C,
                                                          uint32_t &err)
{
    uint32_t heavy = 0;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        uint32_t w[4];
        slice_top_block(x[j], r, t, rk, w);
        const SliceKey key{x[j], r, t, k0, k1};
        if (slice_node(a[j], b[j], c[j], slice_top16(w, x[j]), key, tab, C, err)) heavy |= 1u << j;
    }
    return heavy;
}

}  // namespace mclg
