// Device building blocks of the D1Q3 MCLG step: Philox4x32-10 in registers and
// the exact integer sampler of one sub-collision (Sec. III, Sec. III.A).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#ifndef MCLG_HD
#define MCLG_HD __host__ __device__ __forceinline__
#endif

namespace mclg {

constexpr uint32_t kPurposeCollide = 0u;
constexpr uint32_t kPurposeRefine = 1u;
constexpr uint32_t kPurposeInit = 2u;
constexpr uint32_t kPurposeSlice = 4u;     // slice sampler: the uniform's low 48 bits
constexpr uint32_t kPurposeSliceTop = 6u;  // slice sampler: the uniform's top 16 bits
constexpr int kChunksPerBlock = 10;  // 12-bit primary chunks in one 128-bit Philox block
constexpr int kMaxRefine = 4;        // 16-bit refinement chunks allowed per decision

constexpr uint32_t kErrOverflow = 1u;
constexpr uint32_t kErrSampler = 2u;
constexpr uint32_t kErrTimeout = 4u;  // a bounded device-side wait gave up

// Philox4x32-10 (Salmon et al., SC'11): ten rounds; each multiplies words 0 and
// 2 by the two round constants, swaps the halves and xors in the round key;
// the key advances by the Weyl increments between rounds.
MCLG_HD void philox4x32_10(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3, uint32_t k0,
                           uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = uint64_t(0xD2511F53u) * x0, p1 = uint64_t(0xCD9E8D57u) * x2;
        const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
        const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
        const uint32_t y0 = hi1 ^ x1 ^ k0;
        const uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
}

// The ten round keys of Philox4x32-10 for one seed, precomputed once per launch
// (they are the same for every counter); the two words of a round side by
// side, so that a kernel reads a round's keys with one 8-byte load.
struct RoundKeys {
    uint2 k[10];  // .x: key word 0, .y: key word 1 of round i
};

MCLG_HD RoundKeys make_round_keys(uint64_t seed)
{
    RoundKeys rk;
    uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        rk.k[i].x = k0;
        rk.k[i].y = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return rk;
}

// philox4x32_10 with precomputed round keys.
MCLG_HD void philox4x32_10(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3,
                           const RoundKeys &rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = uint64_t(0xD2511F53u) * x0, p1 = uint64_t(0xCD9E8D57u) * x2;
        const uint32_t y0 = uint32_t(p1 >> 32) ^ x1 ^ rk.k[round].x;
        const uint32_t y2 = uint32_t(p0 >> 32) ^ x3 ^ rk.k[round].y;
        x1 = uint32_t(p1);
        x3 = uint32_t(p0);
        x0 = y0;
        x2 = y2;
    }
}

// Bits [12m, 12m + 12) of the 128-bit block (w0 least significant), m in 0..9.
template <int m>
__device__ __forceinline__ uint32_t chunk12(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3)
{
    constexpr int off = 12 * m, word = off / 32, sh = off % 32;
    const uint32_t w[4] = {w0, w1, w2, w3};
    if constexpr (sh + 12 <= 32) {
        return (w[word] >> sh) & 0xFFFu;
    } else {
        return __funnelshift_r(w[word], w[word + 1], sh) & 0xFFFu;
    }
}

struct NodeKey {
    uint32_t x, r, t, k0, k1;
};

// Refinement chunk s of the node-step: bits [16(s%8), 16(s%8)+16) of block
// (x, r, t, kPurposeRefine << 28 | s/8).
__device__ __forceinline__ uint32_t refine_chunk(const NodeKey &nk, uint32_t s)
{
    uint32_t w0 = nk.x, w1 = nk.r, w2 = nk.t, w3 = (kPurposeRefine << 28) | (s >> 3);
    philox4x32_10(w0, w1, w2, w3, nk.k0, nk.k1);
    const uint32_t m = s & 7u;
    const uint32_t word = (m >> 1) == 0 ? w0 : (m >> 1) == 1 ? w1 : (m >> 1) == 2 ? w2 : w3;
    return (word >> ((m & 1u) * 16u)) & 0xFFFFu;
}

// Finish a decision whose 12-bit primary chunk left U's region open.
// R1 = T1 * 2^12 - q D and R2 = T2 * 2^12 - q D (signed): with `bits` bits of U
// known, U*D*2^bits - T*2^bits lies in [-R, D - R), so R >= D means U < T/D
// for certain and R <= 0 means U >= T/D for certain.  A resolved remainder is
// clamped to 0 or D (it stays resolved under R <- R 2^16 - q D) which keeps
// |R| 2^16 < 2^63 for D < 2^47.  Returns the region (0, 1, 2) or 3 when the
// refinement cap is reached.
static __device__ __noinline__ uint32_t refine_decision(int64_t R1, int64_t R2, int64_t D,
                                                 const NodeKey &nk, uint32_t &next_ref)
{
    for (int k = 0; k < kMaxRefine; ++k) {
        R1 = R1 >= D ? D : (R1 <= 0 ? 0 : R1);
        R2 = R2 >= D ? D : (R2 <= 0 ? 0 : R2);
        const int64_t q = int64_t(refine_chunk(nk, next_ref));
        ++next_ref;
        R1 = R1 * 65536 - q * D;
        R2 = R2 * 65536 - q * D;
        if (R1 >= D) return 0u;
        if (R1 <= 0 && R2 >= D) return 1u;
        if (R2 <= 0) return 2u;
    }
    return 3u;
}

// Exact region of one decision from its 12-bit primary chunk q (64-bit integer
// thresholds, refinement when the chunk leaves the region open).  Returns 0
// (down), 1 (up), 2 (nothing) or 3 (refinement cap).
static __device__ __noinline__ uint32_t exact_decision(uint32_t a, uint32_t b, uint32_t c, uint32_t q,
                                                       uint32_t lam_n, uint32_t lam_d,
                                                       const NodeKey &nk, uint32_t &next_ref)
{
    const uint64_t N = uint64_t(a) + b + c;
    const uint64_t D = 8ull * N * N * lam_d;
    const uint64_t T1 = (uint64_t(a * c) << 4) * lam_n;
    const uint64_t T2 = T1 + uint64_t(b * (b - 1u)) * lam_n;
    const uint64_t X = uint64_t(q) * D;
    const uint64_t S1 = T1 << 12, S2 = T2 << 12;
    if (X + D <= S1) return 0u;
    if (X >= S1 && X + D <= S2) return 1u;
    if (X >= S2) return 2u;
    return refine_decision(int64_t(S1 - X), int64_t(S2 - X), int64_t(D), nk, next_ref);
}

// C sequential sub-collisions at one node, exact 64-bit integer arithmetic for
// every decision.  (a, b, c) = (n_-1, n_0, n_+1), all <= 65535 on entry; on
// return the post-collision state.  Error bits go to err (the node stops at
// the first error).  Used near the uint16 limit, where every transition must
// be checked.
template <bool kLambdaOne>
__device__ __noinline__ void collide_node_checked(uint32_t &a, uint32_t &b, uint32_t &c,
                                             const NodeKey &nk, uint32_t C, uint32_t lam_n,
                                             uint32_t lam_d, uint32_t &err)
{
    const uint32_t N = a + b + c;
    if (N < 2u) return;
    const uint64_t D = kLambdaOne ? 8ull * N * N : 8ull * N * N * lam_d;
    uint32_t next_ref = 0;
    for (uint32_t blk = 0; blk * kChunksPerBlock < C; ++blk) {
        uint32_t w0 = nk.x, w1 = nk.r, w2 = nk.t, w3 = (kPurposeCollide << 28) | blk;
        philox4x32_10(w0, w1, w2, w3, nk.k0, nk.k1);
        const uint32_t base = blk * kChunksPerBlock;
        uint32_t q[kChunksPerBlock];
        q[0] = chunk12<0>(w0, w1, w2, w3);
        q[1] = chunk12<1>(w0, w1, w2, w3);
        q[2] = chunk12<2>(w0, w1, w2, w3);
        q[3] = chunk12<3>(w0, w1, w2, w3);
        q[4] = chunk12<4>(w0, w1, w2, w3);
        q[5] = chunk12<5>(w0, w1, w2, w3);
        q[6] = chunk12<6>(w0, w1, w2, w3);
        q[7] = chunk12<7>(w0, w1, w2, w3);
        q[8] = chunk12<8>(w0, w1, w2, w3);
        q[9] = chunk12<9>(w0, w1, w2, w3);
#pragma unroll
        for (int m = 0; m < kChunksPerBlock; ++m) {
            if (base + m >= C) break;
            const uint64_t ac = uint64_t(a * c);          // < 2^32
            const uint64_t bb = uint64_t(b * (b - 1u));   // b(b-1) < 2^32, 0 for b = 0
            const uint64_t T1 = kLambdaOne ? ac << 4 : (ac << 4) * lam_n;
            const uint64_t T2 = T1 + (kLambdaOne ? bb : bb * lam_n);
            const uint64_t X = uint64_t(q[m]) * D;
            const uint64_t S1 = T1 << 12, S2 = T2 << 12;
            uint32_t region;
            if (X + D <= S1) {
                region = 0u;
            } else if (X >= S1 && X + D <= S2) {
                region = 1u;
            } else if (X >= S2) {
                region = 2u;
            } else {
                region = refine_decision(int64_t(S1 - X), int64_t(S2 - X), int64_t(D), nk,
                                         next_ref);
                if (region == 3u) {
                    err |= kErrSampler;
                    return;
                }
            }
            if (region == 0u) {  // {-1, +1} -> {0, 0}
                if (b + 2u > 65535u) {
                    err |= kErrOverflow;
                    return;
                }
                a -= 1u;
                b += 2u;
                c -= 1u;
            } else if (region == 1u) {  // {0, 0} -> {-1, +1}
                if (a + 1u > 65535u || c + 1u > 65535u) {
                    err |= kErrOverflow;
                    return;
                }
                a += 1u;
                b -= 2u;
                c += 1u;
            }
        }
    }
}


// Chunk m (bits [12m, 12m+12)) of the block, placed at bits [11, 23).
template <int m>
__device__ __forceinline__ uint32_t chunk12_at11(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3)
{
    constexpr int off = 12 * m, word = off / 32, sh = off % 32;
    const uint32_t w[4] = {w0, w1, w2, w3};
    uint32_t v;
    if constexpr (sh + 12 <= 32) {
        v = sh >= 11 ? (w[word] >> (sh - 11)) : (w[word] << (11 - sh));
    } else {
        v = __funnelshift_r(w[word], w[word + 1], sh - 11);
    }
    return v & 0x007FF800u;
}

// One sub-collision of the FP32 fast path (see fast_block); qbits = q << 11.
__device__ __forceinline__ void fast_sub_collision(float &af, float &bm1, float &cf, float K1,
                                                   float K2, uint32_t qbits, const NodeKey &nk,
                                                   uint32_t lam_n, uint32_t lam_d,
                                                   uint32_t &next_ref, bool &failed)
{
    const float lo = __uint_as_float(qbits + 0x3F7FFFF8u);  // 1 + q/4096 - 2^-20
    const float hi = __uint_as_float(qbits + 0x3F800808u);  // 1 + (q+1)/4096 + 2^-20
    const float t1 = fmaf(af * cf, K1, 1.0f);
    const float t2 = fmaf(fmaf(bm1, bm1, bm1), K2, t1);     // b (b - 1) = bm1^2 + bm1
    const bool down = hi <= t1;
    const bool up = lo >= t1 && hi <= t2;
    const bool none = lo >= t2;
    float s = down ? -1.0f : (up ? 1.0f : 0.0f);
    if (!(down || up || none)) {
        const uint32_t a = __float_as_uint(af + 8388608.0f) & 0x7FFFFFu;
        const uint32_t b = __float_as_uint(bm1 + 8388609.0f) & 0x7FFFFFu;
        const uint32_t c = __float_as_uint(cf + 8388608.0f) & 0x7FFFFFu;
        const uint32_t region = exact_decision(a, b, c, qbits >> 11, lam_n, lam_d, nk, next_ref);
        failed |= region == 3u;
        s = region == 0u ? -1.0f : (region == 1u ? 1.0f : 0.0f);
    }
    af += s;
    cf += s;
    bm1 = fmaf(-2.0f, s, bm1);
}

// The sub-collisions of one node that one Philox block serves, FP32 fast path.
//
// 1 + U lies in [1 + q/4096, 1 + (q+1)/4096) and is compared with
// t1 ~ 1 + T1/D and t2 ~ 1 + T2/D.  Their FP32 error is below 7 * 2^-24:
// K1 = 2 lam / (N^2 lam_d) carries two roundings and a 2-ulp __fdividef,
// a*c and b(b-1) one rounding each, each fused multiply-add one.  `lo` and
// `hi` sit outside U's interval by at least 2^-21 (2^-20 except lo at q = 0),
// so every comparison they decide is decided exactly as the integer test
// would; when a threshold lies within that margin of the interval the
// decision goes to the exact 64-bit path (probability about 2^-11).
// State: a, b - 1 and c as FP32 integers (exact below 2^24).
template <int kC>
__device__ __forceinline__ void fast_block(float &af, float &bm1, float &cf, float K1, float K2,
                                           uint32_t blk, uint32_t C, const NodeKey &nk,
                                           const RoundKeys &rk, uint32_t lam_n, uint32_t lam_d,
                                           uint32_t &next_ref, bool &failed)
{
    uint32_t w0 = nk.x, w1 = nk.r, w2 = nk.t, w3 = (kPurposeCollide << 28) | blk;
    philox4x32_10(w0, w1, w2, w3, rk);
    const uint32_t left = kC ? 0u : C - blk * kChunksPerBlock;
#define MCLG_SUB(m)                                                                         \
    if (kC ? (m < kC) : (uint32_t(m) < left))                                               \
        fast_sub_collision(af, bm1, cf, K1, K2, chunk12_at11<m>(w0, w1, w2, w3), nk, lam_n, \
                           lam_d, next_ref, failed);
    MCLG_SUB(0) MCLG_SUB(1) MCLG_SUB(2) MCLG_SUB(3) MCLG_SUB(4)
    MCLG_SUB(5) MCLG_SUB(6) MCLG_SUB(7) MCLG_SUB(8) MCLG_SUB(9)
#undef MCLG_SUB
}

// C sequential sub-collisions at one node (Sec. III; D1Q3 table of
// Sec. III.A), same results as collide_node_checked.  A node within 2C of
// the uint16 limit takes collide_node_checked, which checks every transition.
__device__ __forceinline__ void collide_node(uint32_t &a, uint32_t &b, uint32_t &c,
                                             const NodeKey &nk, const RoundKeys &rk, uint32_t C,
                                             uint32_t lam_n, uint32_t lam_d, uint32_t &err)
{
    const uint32_t N = a + b + c;
    if (N < 2u) return;
    if (max(a, max(b, c)) + 2u * C > 65535u) {
        collide_node_checked<false>(a, b, c, nk, C, lam_n, lam_d, err);
        return;
    }
    // exact int -> float through the exponent bits (all values < 2^23)
    const float fN = __uint_as_float(N | 0x4B000000u) - 8388608.0f;
    const float K1 = __fdividef(float(2u * lam_n), (fN * fN) * float(lam_d));
    const float K2 = K1 * 0.0625f;
    float af = __uint_as_float(a | 0x4B000000u) - 8388608.0f;
    float bm1 = __uint_as_float(b | 0x4B000000u) - 8388609.0f;
    float cf = __uint_as_float(c | 0x4B000000u) - 8388608.0f;
    uint32_t next_ref = 0;
    bool failed = false;
    if (C == 10u) {
        fast_block<10>(af, bm1, cf, K1, K2, 0u, C, nk, rk, lam_n, lam_d, next_ref, failed);
    } else {
        for (uint32_t blk = 0; blk * kChunksPerBlock < C; ++blk)
            fast_block<0>(af, bm1, cf, K1, K2, blk, C, nk, rk, lam_n, lam_d, next_ref, failed);
    }
    // a decision that hit the refinement cap is reported like the checked path
    // reports it (the state after an error is unspecified)
    if (failed) err |= kErrSampler;
    a = __float_as_uint(af + 8388608.0f) & 0x7FFFFFu;
    b = __float_as_uint(bm1 + 8388609.0f) & 0x7FFFFFu;
    c = __float_as_uint(cf + 8388608.0f) & 0x7FFFFFu;
}

// Galilean-invariant collision rate (end of Sec. IV.A): lambda = lt / sqrt(1 + 3 u^2)
// with the node's velocity u = J / N and lt = lt_n / lt_d, quantised down to q / 256:
// the largest q with q^2 lt_d^2 (N^2 + 3 J^2) <= (256 lt_n N)^2.  A single-precision
// first guess is settled by exact 128-bit comparisons (host and device).
__host__ __device__ inline uint32_t galilean_q(uint32_t N, int32_t J, uint32_t lt_n, uint32_t lt_d)
{
    if (N == 0u) return 0u;
    const uint64_t R = uint64_t(N) * N + 3ull * uint64_t(int64_t(J) * J);
    const uint64_t s = 256ull * lt_n * N;
    const unsigned __int128 rhs = (unsigned __int128)s * s;
    const float guess = 256.0f * float(lt_n) * float(N) / (float(lt_d) * sqrtf(float(R)));
    uint64_t q = guess >= 256.0f ? 256u : uint64_t(guess);
    while (q > 0u && (unsigned __int128)(q * q * lt_d * lt_d) * R > rhs) --q;
    while (q < 256u && (unsigned __int128)((q + 1u) * (q + 1u) * lt_d * lt_d) * R <= rhs) ++q;
    return uint32_t(q);
}

// The handle's rate, or the node's Galilean-invariant one, as (numerator, denominator).
__device__ __forceinline__ void node_rate(bool galilean, uint32_t a, uint32_t b, uint32_t c,
                                          uint32_t lam_n, uint32_t lam_d, uint32_t &ln, uint32_t &ld)
{
    ln = lam_n;
    ld = lam_d;
    if (galilean) {
        ln = galilean_q(a + b + c, int32_t(c) - int32_t(a), lam_n, lam_d);
        ld = 256u;
    }
}

// Vector access helpers shared by the per-step kernels.
__device__ __forceinline__ uint32_t lo16(uint32_t w) { return w & 0xFFFFu; }
__device__ __forceinline__ uint32_t hi16(uint32_t w) { return w >> 16; }

// V consecutive uint16 values per thread: one 2-, 4-, 8- or 16-byte vector.
template <int V> struct VecT;
template <> struct VecT<1> { using T = uint16_t; };
template <> struct VecT<2> { using T = uint32_t; };
template <> struct VecT<4> { using T = uint2; };
template <> struct VecT<8> { using T = uint4; };

__device__ __forceinline__ void unpack(uint16_t v, uint32_t e[1]) { e[0] = v; }
__device__ __forceinline__ void unpack(uint32_t v, uint32_t e[2]) { e[0] = lo16(v); e[1] = hi16(v); }
__device__ __forceinline__ void unpack(uint2 v, uint32_t e[4])
{
    e[0] = lo16(v.x); e[1] = hi16(v.x); e[2] = lo16(v.y); e[3] = hi16(v.y);
}
__device__ __forceinline__ void unpack(uint4 v, uint32_t e[8])
{
    e[0] = lo16(v.x); e[1] = hi16(v.x); e[2] = lo16(v.y); e[3] = hi16(v.y);
    e[4] = lo16(v.z); e[5] = hi16(v.z); e[6] = lo16(v.w); e[7] = hi16(v.w);
}
__device__ __forceinline__ void pack(const uint32_t e[1], uint16_t &v) { v = uint16_t(e[0]); }
__device__ __forceinline__ void pack(const uint32_t e[2], uint32_t &v) { v = e[0] | (e[1] << 16); }
__device__ __forceinline__ void pack(const uint32_t e[4], uint2 &v)
{
    v = make_uint2(e[0] | (e[1] << 16), e[2] | (e[3] << 16));
}
__device__ __forceinline__ void pack(const uint32_t e[8], uint4 &v)
{
    v = make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16), e[4] | (e[5] << 16),
                   e[6] | (e[7] << 16));
}

__device__ __forceinline__ void flag_error(uint32_t *err, uint32_t bits)
{
    if (bits) atomicOr(err, bits);
}

}  // namespace mclg
