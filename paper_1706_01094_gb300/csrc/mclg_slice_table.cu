// Host builder of the slice sampler's tables: for every state (N, J >= 0, b)
// of the (N, J) slices with 2 <= N <= n_max, the cumulative law of the rest
// count after C sub-collisions (Sec. III, Sec. III.A: the C-th power of the
// one-sub-collision matrix), as exact fixed-point values
//     F[d] = min(floor(CDF[d] 2^64), 2^64 - 1),   d = dmin .. dmax - 1,
// stored per row re-based at dmin (the u64 secondary table), and a 16-byte
// record per state that the kernel reads first: the top 15 bits of the eight
// values around d = 0 (F[c0 - 4 + j], j = 0..7, c0 = -dmin; 0 below the
// row's first entry, 0x7FFF past its last), which decide almost every draw
// (mclg_slice.cuh).  States with N < 2 get identity records.  The law is
// symmetric under J -> -J (it depends on a c and b only), so only J >= 0 is
// stored.
//
// Exact arithmetic: numerators over D^C with D = 8 N^2 lam_d, in fixed-size
// unsigned big integers of 64-bit limbs.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "mclg_device.cuh"
#include "mclg_internal.h"

namespace mclg {
namespace {

constexpr int kLimbs = 8;  // 512 bits: D^C 2^64 < 2^512 for C <= 10 and D < 2^44

struct Big {
    uint64_t v[kLimbs];
};

inline void big_set(Big &a, uint64_t x)
{
    std::memset(a.v, 0, sizeof(a.v));
    a.v[0] = x;
}

inline void big_add(Big &r, const Big &a)
{
    unsigned __int128 c = 0;
    for (int i = 0; i < kLimbs; ++i) {
        c += (unsigned __int128)r.v[i] + a.v[i];
        r.v[i] = uint64_t(c);
        c >>= 64;
    }
}

// r = a * m
inline void big_mul(Big &r, const Big &a, uint64_t m)
{
    unsigned __int128 c = 0;
    for (int i = 0; i < kLimbs; ++i) {
        c += (unsigned __int128)a.v[i] * m;
        r.v[i] = uint64_t(c);
        c >>= 64;
    }
}

// r += a * m
inline void big_muladd(Big &r, const Big &a, uint64_t m)
{
    unsigned __int128 c = 0;
    for (int i = 0; i < kLimbs; ++i) {
        c += (unsigned __int128)a.v[i] * m + r.v[i];
        r.v[i] = uint64_t(c);
        c >>= 64;
    }
}

inline int big_cmp(const Big &a, const Big &b)
{
    for (int i = kLimbs - 1; i >= 0; --i)
        if (a.v[i] != b.v[i]) return a.v[i] < b.v[i] ? -1 : 1;
    return 0;
}

// a * 2^64 (shift by one limb; the top limb must be free)
inline Big big_shift64(const Big &a)
{
    Big r;
    r.v[0] = 0;
    for (int i = 1; i < kLimbs; ++i) r.v[i] = a.v[i - 1];
    return r;
}

inline int big_top(const Big &a)
{
    for (int i = kLimbs - 1; i >= 0; --i)
        if (a.v[i]) return i;
    return -1;
}

inline void big_sub(Big &r, const Big &a)  // r >= a
{
    unsigned __int128 borrow = 0;
    for (int i = 0; i < kLimbs; ++i) {
        const unsigned __int128 d = (unsigned __int128)r.v[i] - a.v[i] - borrow;
        r.v[i] = uint64_t(d);
        borrow = (d >> 64) ? 1 : 0;
    }
}

inline void big_shl1(Big &a)
{
    for (int i = kLimbs - 1; i > 0; --i) a.v[i] = (a.v[i] << 1) | (a.v[i - 1] >> 63);
    a.v[0] <<= 1;
}

// floor(num 2^64 / den) for num < den.  den < 2^64: one 128-bit division.
// Otherwise an estimate from the two leading limbs (error of a few units),
// corrected until den q <= num 2^64 < den (q + 1) holds, with bit-by-bit long
// division as the fallback should the estimate be far off.
uint64_t big_frac64(const Big &num, const Big &den)
{
    const int t = big_top(den);
    if (t == 0) return uint64_t(((unsigned __int128)num.v[0] << 64) / den.v[0]);
    const Big lhs = big_shift64(num);
    const long double two64 = 18446744073709551616.0L;
    const long double nl = (long double)lhs.v[t + 1] * two64 + (long double)lhs.v[t];
    const long double dl = (long double)den.v[t] + (long double)den.v[t - 1] / two64;
    const long double ratio = nl / dl;
    uint64_t q = ratio <= 0.0L ? 0 : (ratio >= 18446744073709551615.0L ? UINT64_MAX : uint64_t(ratio));
    Big prod, next;
    for (int it = 0; it < 8; ++it) {
        big_mul(prod, den, q);
        if (big_cmp(prod, lhs) > 0) {
            --q;
            continue;
        }
        next = prod;
        big_add(next, den);
        if (big_cmp(next, lhs) <= 0) {
            ++q;
            continue;
        }
        return q;  // den q <= lhs < den (q + 1)
    }
    // long division: one quotient bit per step
    Big rem = num;
    uint64_t qq = 0;
    for (int i = 63; i >= 0; --i) {
        big_shl1(rem);
        qq <<= 1;
        if (big_cmp(rem, den) >= 0) {
            big_sub(rem, den);
            qq |= 1;
        }
    }
    return qq;
}

struct SliceParams {
    uint32_t C, lam_n, lam_d;
};

inline void thresholds(int64_t N, int64_t J, int64_t b, uint32_t lam_n, uint64_t &down, uint64_t &up)
{
    down = up = 0;
    if (b < 0 || b > N - J || ((N - J - b) & 1)) return;  // J >= 0 here
    const int64_t a = (N - J - b) / 2, c = (N + J - b) / 2;
    down = 16ull * uint64_t(a) * uint64_t(c) * lam_n;
    up = (b > 0 ? uint64_t(b) * uint64_t(b - 1) : 0ull) * lam_n;
}

// One row: F[k] for d = dmin + k, k < dmax - dmin.
void build_row(uint32_t N, uint32_t J, uint32_t b, const SliceParams &sp, uint64_t *F, int &dmin,
               int &dmax)
{
    const int C = int(sp.C);
    const int64_t bmin = int64_t(N - J) & 1;
    dmin = int(std::max<int64_t>(-C, (bmin - int64_t(b)) / 2));
    dmax = int(std::min<int64_t>(C, (int64_t(N) - J - int64_t(b)) / 2));
    const uint64_t D = 8ull * N * N * sp.lam_d;  // < kSliceMaxD (callers check)
    constexpr int W = 2 * kSliceMaxC + 1;
    Big v[W], nv[W], den;
    for (int i = 0; i < W; ++i) big_set(v[i], 0);
    big_set(v[kSliceMaxC], 1);
    big_set(den, 1);
    uint64_t dn[W], up[W];
    for (int i = 0; i < W; ++i) thresholds(N, J, int64_t(b) + 2 * (i - kSliceMaxC), sp.lam_n, dn[i], up[i]);
    for (int step = 0; step < C; ++step) {
        for (int i = 0; i < W; ++i) {
            big_mul(nv[i], v[i], D - dn[i] - up[i]);
            if (i > 0 && dn[i - 1]) big_muladd(nv[i], v[i - 1], dn[i - 1]);
            if (i < W - 1 && up[i + 1]) big_muladd(nv[i], v[i + 1], up[i + 1]);
        }
        std::memcpy(v, nv, sizeof(v));
        Big t;
        big_mul(t, den, D);
        den = t;
    }
    Big cum;
    big_set(cum, 0);
    for (int i = 0; i < W; ++i) {
        const int d = i - kSliceMaxC;
        big_add(cum, v[i]);
        if (d >= dmin && d < dmax)
            F[d - dmin] = big_cmp(cum, den) >= 0 ? UINT64_MAX : big_frac64(cum, den);
    }
}

}  // namespace

void build_slice_row(uint32_t N, uint32_t J, uint32_t b, uint32_t C, uint32_t lam_n, uint32_t lam_d,
                     uint64_t *F, int &dmin, int &dmax)
{
    const SliceParams sp{C, lam_n, lam_d};
    build_row(N, J, b, sp, F, dmin, dmax);
}

uint64_t slice_rows(uint32_t n_max)
{
    uint64_t rows = 0;
    for (uint32_t N = 0; N <= n_max; ++N)
        for (uint32_t J = 0; J <= N; ++J) rows += (N - J) / 2 + 1;
    return rows;
}

uint64_t slice_records(uint32_t n_max)
{
    return uint64_t(n_max + 1) * (n_max + 1) * (n_max / 2 + 1);
}

// Record of one law with n entries, c0 = -dmin: lane j = the top 15 bits of
// F[c0 - 4 + j], or 0 below the first entry and 0x7FFF past the last.
void build_slice_record(const uint64_t *F, int n, int c0, uint16_t *record)
{
    for (int j = 0; j < kSliceRecordLanes; ++j) {
        const int k = c0 - 4 + j;
        record[j] = k < 0 ? uint16_t(0) : k >= n ? uint16_t(0x7FFF) : uint16_t(F[k] >> 49);
    }
}

// Fills rowstart[N * (n_max + 1) + J] (first row of the (N, J) slice),
// secondary[row * kSliceRowU64 + k] and the records, 8 lanes each, of every
// state (N, J, b) at (N (n_max + 1) + J) (n_max / 2 + 1) + b / 2.
void build_slice_tables(uint32_t n_max, uint32_t C, uint32_t lam_n, uint32_t lam_d, bool galilean,
                        std::vector<uint32_t> &rowstart, std::vector<uint16_t> &record,
                        std::vector<uint64_t> &secondary)
{
    const uint64_t rows = slice_rows(n_max);
    const uint64_t hb = n_max / 2 + 1;
    rowstart.assign(size_t(n_max + 1) * (n_max + 1), 0u);
    secondary.assign(rows * kSliceRowU64, UINT64_MAX);
    // identity records (d = 0 whatever Q's top bits: no entries around c0 = 0)
    record.resize(slice_records(n_max) * kSliceRecordLanes);
    for (uint64_t i = 0; i < record.size(); ++i)
        record[i] = (i % kSliceRecordLanes) < 4 ? uint16_t(0) : uint16_t(0x7FFF);
    uint64_t r = 0;
    for (uint32_t N = 0; N <= n_max; ++N)
        for (uint32_t J = 0; J <= N; ++J) {
            rowstart[size_t(N) * (n_max + 1) + J] = uint32_t(r);
            r += (N - J) / 2 + 1;
        }
    // spread the slices over the host cores, larger N first
    unsigned nth = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 64u));
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < nth; ++w)
        pool.emplace_back([&, w]() {
            uint64_t F[2 * kSliceMaxC + 1];
            uint32_t k = 0;
            for (int64_t N = n_max; N >= 2; --N)
                for (uint32_t J = 0; J <= uint32_t(N); ++J, ++k) {
                    if (k % nth != w) continue;
                    const uint32_t first = rowstart[size_t(N) * (n_max + 1) + J];
                    // the slice's rate: the handle's, or the Galilean-invariant one of (N, J)
                    const SliceParams sp = galilean
                        ? SliceParams{C, galilean_q(uint32_t(N), int32_t(J), lam_n, lam_d), 256u}
                        : SliceParams{C, lam_n, lam_d};
                    const uint32_t bmin = uint32_t(N - J) & 1u;
                    for (uint32_t b = bmin; b <= uint32_t(N) - J; b += 2) {
                        int dmin, dmax;
                        build_row(uint32_t(N), J, b, sp, F, dmin, dmax);
                        const uint64_t row = first + (b - bmin) / 2;
                        for (int i = 0; i < dmax - dmin; ++i) secondary[row * kSliceRowU64 + i] = F[i];
                        const uint64_t rec = (uint64_t(N) * (n_max + 1) + J) * hb + b / 2;
                        build_slice_record(F, dmax - dmin, -dmin, &record[rec * kSliceRecordLanes]);
                    }
                }
        });
    for (auto &th : pool) th.join();
}

}  // namespace mclg
