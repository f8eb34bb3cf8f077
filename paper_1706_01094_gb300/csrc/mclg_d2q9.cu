// D2Q9 Monte Carlo Lattice Gas (Sec. II.B, III.B, IV.B): the host side of the
// mclg2d_* calls in include/mclg.h and its kernels.
//
// Velocities v_i = (vx, vy), vx, vy in {-1, 0, 1}, numbered 0 = (0,0),
// 1 = (1,0), 2 = (0,1), 3 = (-1,0), 4 = (0,-1), 5 = (1,1), 6 = (-1,1),
// 7 = (-1,-1), 8 = (1,-1) (Fig. D2Q9vel); weights 4/9, 1/9, 1/36.
//
// A sub-collision follows the algorithm of Sec. III: two particle indices
// drawn uniformly from [0, N) (exact integer draws); the same particle twice
// collides nothing; otherwise the unordered velocity pair {s1, s2} may turn
// into one of the pairs with the same total momentum (the nine collision
// classes of Sec. III.B), with the class rate lambda_c towards the pair that
// is less likely at equilibrium seen from the more likely one scaled by the
// ratio of their equilibrium pick weights, so that detailed balance holds.
// One uniform integer below 128 lambda_den picks the outcome against the
// cumulative numerators.  The numbering of the classes is the one of the
// relaxation coefficients of Eq. D2Q9MOmega.
//
// Storage: canonical occupations n[9][S], S = R Lx Ly, node g = y Lx + x of
// replica r at r Lx Ly + g.  A step reads each node's own nine values,
// collides them and pushes population i to node x + v_i of the other buffer
// (periodic), so every read and write of a warp is contiguous per plane.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "../../include/mclg.h"
#include "mclg_device.cuh"

namespace {

constexpr int kVx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kVy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr uint32_t kPurposeD2Q9 = 5u;
constexpr uint32_t kThreads2 = 128;

__constant__ int c_vx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int c_vy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Outcomes of an ordered velocity pick (s1, s2), entry s1 * 9 + s2: n
// outcomes, target pair k in bits [8k, 8k + 8) of tgt (low nibble the first
// velocity, high nibble the second), cumulative numerators over 128 lam_den.
struct PairOut {
    uint32_t n;
    uint32_t tgt;
    uint32_t cum[4];
};

// ------------------------------------------------------------ host table ---
int velocity_index(int vx, int vy)
{
    for (int i = 0; i < 9; ++i)
        if (kVx[i] == vx && kVy[i] == vy) return i;
    return -1;
}

// pick weight of the unordered pair {i, j} at equilibrium, in units of 1/36^2:
// (i == j ? 1 : 2) w_i w_j with 36 w = 16, 4, 4, 4, 4, 1, 1, 1, 1
uint32_t pick_weight(int i, int j)
{
    const uint32_t w36[9] = {16, 4, 4, 4, 4, 1, 1, 1, 1};
    return (i == j ? 1u : 2u) * w36[i] * w36[j];
}

struct Collision {
    int a[2], b[2];  // the two unordered pairs, each sorted
    int cls;         // 0 .. 8 (rate lambda_{cls + 1})
};

// The 30 collisions: a representative of each class (Eq. D2Q9MOmega's
// numbering) mapped through the 8 symmetries of the square.
std::vector<Collision> collisions()
{
    static const int reps[9][4] = {
        {0, 5, 1, 2},  // 1: rest + diagonal <-> two axis velocities, momentum (1,1)
        {0, 0, 1, 3},  // 2: two rest <-> opposite axis pair
        {0, 0, 5, 7},  // 3: two rest <-> opposite diagonal pair
        {1, 3, 5, 7},  // 4: opposite axis pair <-> opposite diagonal pair
        {1, 3, 2, 4},  // 5: opposite axis pairs, turned by 90 degrees
        {5, 7, 6, 8},  // 6: opposite diagonal pairs, turned by 90 degrees
        {0, 1, 2, 8},  // 7: rest + axis <-> axis + diagonal, momentum (1,0)
        {1, 6, 3, 5},  // 8: axis + diagonal <-> axis + diagonal, momentum (0,1)
        {1, 1, 5, 8},  // 9: two equal axis velocities <-> two diagonals, momentum (2,0)
    };
    std::vector<Collision> out;
    for (int c = 0; c < 9; ++c)
        for (int sym = 0; sym < 8; ++sym) {
            int img[4];
            for (int q = 0; q < 4; ++q) {
                int x = kVx[reps[c][q]], y = kVy[reps[c][q]];
                if (sym & 4) std::swap(x, y);
                if (sym & 1) x = -x;
                if (sym & 2) y = -y;
                img[q] = velocity_index(x, y);
            }
            Collision k{{std::min(img[0], img[1]), std::max(img[0], img[1])},
                        {std::min(img[2], img[3]), std::max(img[2], img[3])}, c};
            bool seen = false;
            for (const Collision &e : out) {
                const bool same = (e.a[0] == k.a[0] && e.a[1] == k.a[1] && e.b[0] == k.b[0] &&
                                   e.b[1] == k.b[1]) ||
                                  (e.a[0] == k.b[0] && e.a[1] == k.b[1] && e.b[0] == k.a[0] &&
                                   e.b[1] == k.a[1]);
                seen = seen || same;
            }
            if (!seen) out.push_back(k);
        }
    return out;
}

// The outcome list of the unordered pair {s1, s2}: targets sorted by (first,
// second) velocity, numerators over 128 lam_den.  Returns false when the
// probabilities of the pair add up to more than 1.
bool pair_outcomes(int s1, int s2, const uint32_t lam_num[9], uint32_t lam_den,
                   const std::vector<Collision> &cols, int &n, int targets[4][2], uint64_t nums[4])
{
    const int a0 = std::min(s1, s2), a1 = std::max(s1, s2);
    struct Out { int b0, b1; uint64_t num; };
    std::vector<Out> outs;
    for (const Collision &e : cols) {
        const int *other = nullptr;
        if (e.a[0] == a0 && e.a[1] == a1) other = e.b;
        else if (e.b[0] == a0 && e.b[1] == a1) other = e.a;
        if (!other) continue;
        const uint64_t from = pick_weight(a0, a1), to = pick_weight(other[0], other[1]);
        // the class rate from the less likely pick; the other way scaled by the
        // weight ratio (a power of 2 down to 1/128: 128 * ratio is an integer)
        const uint64_t num = from <= to ? uint64_t(lam_num[e.cls]) * 128u
                                        : uint64_t(lam_num[e.cls]) * 128u * to / from;
        outs.push_back({other[0], other[1], num});
    }
    std::sort(outs.begin(), outs.end(), [](const Out &x, const Out &y) {
        return x.b0 != y.b0 ? x.b0 < y.b0 : x.b1 < y.b1;
    });
    uint64_t total = 0;
    n = int(outs.size());
    for (int k = 0; k < n; ++k) {
        targets[k][0] = outs[k].b0;
        targets[k][1] = outs[k].b1;
        nums[k] = outs[k].num;
        total += outs[k].num;
    }
    return total <= 128ull * lam_den;
}

// ---------------------------------------------------------------- device ---
// The node-step's stream of 32-bit words: word k is word k % 4 of Philox block
// (g, r, t, kPurposeD2Q9 << 28 | k / 4); at most `cap` words.
struct WordStream {
    uint32_t g, r, t, k, cap;
    uint32_t w[4];
};

__device__ __forceinline__ bool next_word(WordStream &s, const mclg::RoundKeys &rk, uint32_t &out)
{
    if (s.k >= s.cap) return false;
    if ((s.k & 3u) == 0u) {
        uint32_t x0 = s.g, x1 = s.r, x2 = s.t, x3 = (kPurposeD2Q9 << 28) | (s.k >> 2);
        mclg::philox4x32_10(x0, x1, x2, x3, rk);
        s.w[0] = x0;
        s.w[1] = x1;
        s.w[2] = x2;
        s.w[3] = x3;
    }
    const uint32_t j = s.k & 3u;
    out = j == 0u ? s.w[0] : (j == 1u ? s.w[1] : (j == 2u ? s.w[2] : s.w[3]));
    ++s.k;
    return true;
}

// A uniform integer in [0, m) (1 <= m < 2^32): Lemire's multiply-shift with
// rejection of the low words below (2^32 - m) mod m.
__device__ __forceinline__ bool uniform_below(WordStream &s, const mclg::RoundKeys &rk, uint32_t m,
                                              uint32_t &out)
{
    uint32_t x;
    if (!next_word(s, rk, x)) return false;
    uint64_t prod = uint64_t(x) * m;
    uint32_t lo = uint32_t(prod);
    if (lo < m) {
        const uint32_t thr = (0u - m) % m;
        while (lo < thr) {
            if (!next_word(s, rk, x)) return false;
            prod = uint64_t(x) * m;
            lo = uint32_t(prod);
        }
    }
    out = uint32_t(prod >> 32);
    return true;
}

struct Args2 {
    const uint16_t *in;
    uint16_t *out;
    uint64_t S;
    uint32_t Lx, Ly, R;
    uint32_t t, C, D, r0, stream;
    const uint32_t *t_dev;  // if set, the time step is *t_dev + t
    const PairOut *table;   // [81]
    uint32_t *err;
    mclg::RoundKeys rk;
};

__global__ void __launch_bounds__(kThreads2) k_step_d2q9(Args2 p)
{
    const uint64_t o = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (o >= p.S) return;
    const uint32_t G = p.Lx * p.Ly;
    const uint32_t r = uint32_t(o / G), g = uint32_t(o - uint64_t(r) * G);
    const uint32_t y = g / p.Lx, x = g - y * p.Lx;
    uint32_t n[9], N = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        n[i] = p.in[uint64_t(i) * p.S + o];
        N += n[i];
    }
    uint32_t err = 0;
    if (N >= 2u) {
        const uint32_t t = p.t_dev ? *p.t_dev + p.t : p.t;
        WordStream ws{g, r + p.r0, t, 0u, 16u * p.C + 64u, {0u, 0u, 0u, 0u}};
        for (uint32_t k = 0; k < p.C; ++k) {
            uint32_t q1, q2;
            if (!uniform_below(ws, p.rk, N, q1) || !uniform_below(ws, p.rk, N, q2)) {
                err |= mclg::kErrSampler;
                break;
            }
            if (q1 == q2) continue;  // the same particle twice
            // velocities of the two picks: the smallest s with q < n_0 + ... + n_s
            // (q < N, so both are found)
            int s1 = 9, s2 = 9;
            uint32_t cum = 0;
#pragma unroll
            for (int s = 0; s < 9; ++s) {
                cum += n[s];
                if (s1 == 9 && q1 < cum) s1 = s;
                if (s2 == 9 && q2 < cum) s2 = s;
            }
            const PairOut e = p.table[s1 * 9 + s2];
            if (e.n == 0u) continue;
            uint32_t u;
            if (!uniform_below(ws, p.rk, p.D, u)) {
                err |= mclg::kErrSampler;
                break;
            }
            for (uint32_t j = 0; j < e.n; ++j) {
                if (u < e.cum[j]) {
                    const uint32_t b = (e.tgt >> (8u * j)) & 0xFFu, b0 = b & 0xFu, b1 = b >> 4;
                    --n[s1];
                    --n[s2];
                    ++n[b0];
                    ++n[b1];
                    if (n[b0] > 65535u || n[b1] > 65535u) err |= mclg::kErrOverflow;
                    break;
                }
            }
            if (err) break;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        uint64_t dst = o;
        if (p.stream) {
            // push to x + v_i (periodic)
            const uint32_t xd = (x + p.Lx + uint32_t(c_vx[i])) % p.Lx;
            const uint32_t yd = (y + p.Ly + uint32_t(c_vy[i])) % p.Ly;
            dst = uint64_t(r) * G + uint64_t(yd) * p.Lx + xd;
        }
        p.out[uint64_t(i) * p.S + dst] = uint16_t(n[i]);
    }
    mclg::flag_error(p.err, err);
}

// Density and momentum per node; exact totals (block sums, one 64-bit atomic each).
__global__ void __launch_bounds__(256) k_moments_d2q9(const uint16_t *__restrict__ n, uint64_t S,
                                                      int32_t *rho, int32_t *jx, int32_t *jy,
                                                      unsigned long long *totals)
{
    const uint64_t o = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    long long s[3] = {0, 0, 0};
    if (o < S) {
        int32_t a = 0, bx = 0, by = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int32_t v = n[uint64_t(i) * S + o];
            a += v;
            bx += v * c_vx[i];
            by += v * c_vy[i];
        }
        if (rho) rho[o] = a;
        if (jx) jx[o] = bx;
        if (jy) jy[o] = by;
        s[0] = a;
        s[1] = bx;
        s[2] = by;
    }
    __shared__ long long red[3][8];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        for (int d = 16; d > 0; d >>= 1) s[q] += __shfl_down_sync(0xFFFFFFFFu, s[q], d);
        if ((threadIdx.x & 31u) == 0u) red[q][threadIdx.x >> 5] = s[q];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        long long v = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        atomicAdd(totals + threadIdx.x, (unsigned long long)v);
    }
}

bool is_device(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Entropic D2Q9 equilibrium (Eq. D2Q9eqdist) and Poisson sampling by inversion
// over parts of mean <= 32, in the FP64 operation order of the D1Q3 contract.
void equilibrium2(double rho, double ux, double uy, double f[9])
{
    static const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    const double sx = std::sqrt(1.0 + 3.0 * ux * ux) - 1.0, sy = std::sqrt(1.0 + 3.0 * uy * uy) - 1.0;
    for (int i = 0; i < 9; ++i) {
        const double vx = kVx[i], vy = kVy[i];
        const double gx = w1[kVx[i] + 1] * (1.0 + 3.0 * vx * ux + (3.0 * vx * vx - 1.0) * sx);
        const double gy = w1[kVy[i] + 1] * (1.0 + 3.0 * vy * uy + (3.0 * vy * vy - 1.0) * sy);
        f[i] = rho * gx * gy;
    }
}

uint32_t poisson_inversion(double mu, double U)
{
    double pk = std::exp(-mu), cdf = pk;
    uint32_t k = 0;
    while (U >= cdf && k < 200u) {
        ++k;
        pk = pk * (mu / double(k));
        cdf = cdf + pk;
    }
    return k;
}

}  // namespace

struct mclg2d_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t Lx = 0, Ly = 0, R = 0;
    uint64_t S = 0, seed = 0, t = 0;
    mclg2d_params prm{};
    uint16_t *d_n[2] = {nullptr, nullptr};
    int cur = 0;
    PairOut *d_table = nullptr;
    uint32_t *d_err = nullptr;
    unsigned long long *d_totals = nullptr;
    uint32_t sticky = 0;
    bool has_state = false;
};

namespace {

mclg_status ck(cudaError_t e) { return e == cudaSuccess ? MCLG_OK : MCLG_ERR_CUDA; }

#define MCLG2_CK(expr)                                 \
    do {                                               \
        cudaError_t _e = (expr);                       \
        if (_e != cudaSuccess) return ck(_e);          \
    } while (0)

mclg_status collect2(mclg2d_ctx *h)
{
    MCLG2_CK(cudaStreamSynchronize(h->stream));
    uint32_t bits = 0;
    MCLG2_CK(cudaMemcpy(&bits, h->d_err, sizeof(bits), cudaMemcpyDeviceToHost));
    h->sticky |= bits;
    if (h->sticky & mclg::kErrOverflow) return MCLG_ERR_OVERFLOW;
    if (h->sticky & mclg::kErrSampler) return MCLG_ERR_SAMPLER;
    return MCLG_OK;
}

mclg_status upload2(mclg2d_ctx *h, const uint16_t *n, uint64_t t)
{
    const bool dev = is_device(n);
    MCLG2_CK(cudaMemcpyAsync(h->d_n[h->cur], n, 9 * h->S * sizeof(uint16_t),
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    MCLG2_CK(cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream));
    if (!dev) MCLG2_CK(cudaStreamSynchronize(h->stream));
    h->t = t;
    h->sticky = 0;
    h->has_state = true;
    return MCLG_OK;
}

}  // namespace

extern "C" {

void mclg2d_default_params(mclg2d_params *p)
{
    if (!p) return;
    p->C = 10;
    // the rates of the paper's D2Q9 runs (Sec. IV.B): 15/128, 1/4 (classes 2-7), 1/8, 18/144
    const uint32_t num[9] = {15, 32, 32, 32, 32, 32, 32, 16, 16};
    std::memcpy(p->lambda_num, num, sizeof(num));
    p->lambda_den = 128;
    p->flags = 0;
    p->first_replica = 0;
}

mclg_status mclg2d_pair_outcomes(uint32_t s1, uint32_t s2, const mclg2d_params *p,
                                 uint32_t *count, uint32_t *targets, uint64_t *nums)
{
    if (!p || !count || s1 > 8 || s2 > 8 || p->lambda_den < 1 || p->lambda_den > 65536)
        return MCLG_ERR_ARG;
    const std::vector<Collision> cols = collisions();
    int n = 0, tg[4][2];
    uint64_t nm[4];
    if (!pair_outcomes(int(s1), int(s2), p->lambda_num, p->lambda_den, cols, n, tg, nm))
        return MCLG_ERR_ARG;
    *count = uint32_t(n);
    for (int k = 0; k < n; ++k) {
        if (targets) {
            targets[2 * k] = uint32_t(tg[k][0]);
            targets[2 * k + 1] = uint32_t(tg[k][1]);
        }
        if (nums) nums[k] = nm[k];
    }
    return MCLG_OK;
}

void mclg2d_destroy(mclg2d_handle h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->d_n[0]);
    cudaFree(h->d_n[1]);
    cudaFree(h->d_table);
    cudaFree(h->d_err);
    cudaFree(h->d_totals);
    delete h;
}

mclg_status mclg2d_create(uint32_t Lx, uint32_t Ly, uint32_t replicas, uint64_t seed,
                          const mclg2d_params *p, void *cuda_stream, mclg2d_handle *out)
{
    if (!out) return MCLG_ERR_ARG;
    *out = nullptr;
    mclg2d_params prm;
    mclg2d_default_params(&prm);
    if (p) prm = *p;
    if (Lx == 0 || Ly == 0 || replicas == 0) return MCLG_ERR_ARG;
    const uint64_t G = uint64_t(Lx) * Ly, S = G * replicas;
    if (G >= (uint64_t(1) << 32) || S >= (uint64_t(1) << 38)) return MCLG_ERR_ARG;
    if (uint64_t(prm.first_replica) + replicas > (uint64_t(1) << 32)) return MCLG_ERR_ARG;
    if (prm.lambda_den < 1 || prm.lambda_den > 65536 || prm.C > (1u << 24) ||
        (prm.flags & ~MCLG_NO_STREAM))
        return MCLG_ERR_ARG;
    for (int c = 0; c < 9; ++c)
        if (prm.lambda_num[c] > prm.lambda_den) return MCLG_ERR_ARG;
    // the outcome table; every pick's probabilities must add up to at most 1
    const std::vector<Collision> cols = collisions();
    PairOut table[81];
    for (int s1 = 0; s1 < 9; ++s1)
        for (int s2 = 0; s2 < 9; ++s2) {
            int n = 0, tg[4][2];
            uint64_t nm[4];
            if (!pair_outcomes(s1, s2, prm.lambda_num, prm.lambda_den, cols, n, tg, nm))
                return MCLG_ERR_ARG;
            PairOut e{};
            e.n = uint32_t(n);
            uint64_t cum = 0;
            for (int k = 0; k < n; ++k) {
                cum += nm[k];
                e.cum[k] = uint32_t(cum);
                e.tgt |= uint32_t(tg[k][0] | (tg[k][1] << 4)) << (8 * k);
            }
            table[s1 * 9 + s2] = e;
        }
    mclg2d_ctx *h = new (std::nothrow) mclg2d_ctx();
    if (!h) return MCLG_ERR_NOMEM;
    h->prm = prm;
    h->Lx = Lx;
    h->Ly = Ly;
    h->R = replicas;
    h->S = S;
    h->seed = seed;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    auto fail = [&](mclg_status s) {
        mclg2d_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(MCLG_ERR_CUDA);
    if (cudaMalloc(&h->d_n[0], 9 * S * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc(&h->d_n[1], 9 * S * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc(&h->d_table, sizeof(table)) != cudaSuccess ||
        cudaMalloc(&h->d_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&h->d_totals, 3 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return fail(MCLG_ERR_NOMEM);
    }
    if (cudaMemcpy(h->d_table, table, sizeof(table), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->d_err, 0, sizeof(uint32_t)) != cudaSuccess)
        return fail(MCLG_ERR_CUDA);
    *out = h;
    return MCLG_OK;
}

mclg_status mclg2d_init(mclg2d_handle h, const double *rho, const double *ux, const double *uy)
{
    if (!h || !rho || !ux || !uy) return MCLG_ERR_ARG;
    MCLG2_CK(cudaSetDevice(h->device));
    std::vector<uint16_t> n;
    try {
        n.resize(9 * h->S);
    } catch (...) {
        return MCLG_ERR_NOMEM;
    }
    const uint64_t G = uint64_t(h->Lx) * h->Ly;
    const uint32_t k0 = uint32_t(h->seed), k1 = uint32_t(h->seed >> 32);
    unsigned nth = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 64u));
    std::vector<int> errs(nth, 0);
    std::vector<std::thread> pool;
    for (unsigned wk = 0; wk < nth; ++wk)
        pool.emplace_back([&, wk]() {
            for (uint64_t o = wk; o < h->S; o += nth) {
                const uint32_t r = uint32_t(o / G), g = uint32_t(o - uint64_t(r) * G);
                const double rh = rho[o], u1 = ux[o], u2 = uy[o];
                if (!(rh >= 0.0) || !std::isfinite(rh) || !(std::fabs(u1) <= 1.0) ||
                    !(std::fabs(u2) <= 1.0)) {
                    errs[wk] |= 8;
                    continue;
                }
                double f[9];
                equilibrium2(rh, u1, u2, f);
                for (uint32_t i = 0; i < 9; ++i) {
                    const double mu = f[i] > 0.0 ? f[i] : 0.0;
                    uint32_t parts = uint32_t(std::ceil(mu / 32.0));
                    if (parts < 1) parts = 1;
                    const double part_mu = mu / double(parts);
                    uint64_t total = 0;
                    for (uint32_t q = 0; q < parts; ++q) {
                        uint32_t w0 = g, w1 = r + h->prm.first_replica, w2 = q / 2,
                                 w3 = (mclg::kPurposeInit << 28) | i;
                        mclg::philox4x32_10(w0, w1, w2, w3, k0, k1);
                        const uint32_t lo = (q & 1u) ? w2 : w0, hi = (q & 1u) ? w3 : w1;
                        const uint64_t m = ((uint64_t(hi) << 32) | lo) >> 11;
                        total += poisson_inversion(part_mu, double(m) * (1.0 / 9007199254740992.0));
                    }
                    if (total > 65535u) {
                        errs[wk] |= 1;
                        total = 65535u;
                    }
                    n[i * h->S + o] = uint16_t(total);
                }
            }
        });
    for (auto &th : pool) th.join();
    int err = 0;
    for (int e : errs) err |= e;
    if (err & 8) return MCLG_ERR_ARG;
    mclg_status s = upload2(h, n.data(), 0);
    if (s != MCLG_OK) return s;
    if (err & 1) {
        h->sticky |= mclg::kErrOverflow;
        return MCLG_ERR_OVERFLOW;
    }
    return MCLG_OK;
}

mclg_status mclg2d_set_state(mclg2d_handle h, const uint16_t *n, uint64_t t)
{
    if (!h || !n || t >= (uint64_t(1) << 32)) return MCLG_ERR_ARG;
    MCLG2_CK(cudaSetDevice(h->device));
    return upload2(h, n, t);
}

mclg_status mclg2d_get_state(mclg2d_handle h, uint16_t *n, uint64_t *t)
{
    if (!h || !n) return MCLG_ERR_ARG;
    if (!h->has_state) return MCLG_ERR_STATE;
    MCLG2_CK(cudaSetDevice(h->device));
    MCLG2_CK(cudaMemcpyAsync(n, h->d_n[h->cur], 9 * h->S * sizeof(uint16_t),
                             is_device(n) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             h->stream));
    if (t) *t = h->t;
    return collect2(h);
}

mclg_status mclg2d_step(mclg2d_handle h, uint64_t n_steps)
{
    if (!h) return MCLG_ERR_ARG;
    if (!h->has_state) return MCLG_ERR_STATE;
    if (h->t + n_steps > (uint64_t(1) << 32)) return MCLG_ERR_ARG;
    if (h->sticky) return collect2(h);
    MCLG2_CK(cudaSetDevice(h->device));
    Args2 a{};
    a.S = h->S;
    a.Lx = h->Lx;
    a.Ly = h->Ly;
    a.R = h->R;
    a.C = h->prm.C;
    a.D = 128u * h->prm.lambda_den;
    a.r0 = h->prm.first_replica;
    a.stream = (h->prm.flags & MCLG_NO_STREAM) ? 0u : 1u;
    a.t_dev = nullptr;
    a.table = h->d_table;
    a.err = h->d_err;
    a.rk = mclg::make_round_keys(h->seed);
    const uint32_t blocks = uint32_t((h->S + kThreads2 - 1) / kThreads2);
    for (uint64_t s = 0; s < n_steps; ++s) {
        a.in = h->d_n[h->cur];
        a.out = h->d_n[h->cur ^ 1];
        a.t = uint32_t(h->t);
        k_step_d2q9<<<blocks, kThreads2, 0, h->stream>>>(a);
        MCLG2_CK(cudaGetLastError());
        h->cur ^= 1;
        h->t += 1;
    }
    return MCLG_OK;
}

mclg_status mclg2d_moments(mclg2d_handle h, int32_t *rho, int32_t *jx, int32_t *jy,
                           int64_t *totals)
{
    if (!h) return MCLG_ERR_ARG;
    if (!h->has_state) return MCLG_ERR_STATE;
    if ((rho && !is_device(rho)) || (jx && !is_device(jx)) || (jy && !is_device(jy)))
        return MCLG_ERR_ARG;  // per-node moments into device arrays (the totals may be host)
    MCLG2_CK(cudaSetDevice(h->device));
    MCLG2_CK(cudaMemsetAsync(h->d_totals, 0, 3 * sizeof(unsigned long long), h->stream));
    const uint32_t blocks = uint32_t((h->S + 255) / 256);
    k_moments_d2q9<<<blocks, 256, 0, h->stream>>>(h->d_n[h->cur], h->S, rho, jx, jy, h->d_totals);
    MCLG2_CK(cudaGetLastError());
    unsigned long long tot[3] = {0, 0, 0};
    MCLG2_CK(cudaMemcpyAsync(tot, h->d_totals, sizeof(tot), cudaMemcpyDeviceToHost, h->stream));
    mclg_status s = collect2(h);
    if (totals)
        for (int q = 0; q < 3; ++q) totals[q] = (int64_t)tot[q];
    return s;
}

mclg_status mclg2d_sync(mclg2d_handle h)
{
    if (!h) return MCLG_ERR_ARG;
    MCLG2_CK(cudaSetDevice(h->device));
    return collect2(h);
}

uint64_t mclg2d_time(mclg2d_handle h) { return h ? h->t : 0; }

}  // extern "C"
