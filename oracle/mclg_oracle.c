/*
 * Plain CPU oracle for the D1Q3 Monte Carlo Lattice Gas (Blommel & Wagner,
 * "Integer lattice gas with Monte Carlo collision operator recovers the
 * entropic lattice Boltzmann method with Poisson distributed fluctuations").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library, its kernels or its Python
 * binding may include, link or call this file; only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark use it.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * Everything is written for clarity, not speed: nested loops over replicas,
 * nodes and sub-collisions in the order the paper states them, 128-bit integer
 * comparisons for the exact sampler, FP64 for the equilibrium and the Poisson
 * initialisation.  Build with -ffp-contract=off (no fused multiply-add) so the
 * FP64 initialisation is reproducible.
 *
 * The node loops of one time step (and of the initialisation) are shared out
 * over the host cores with OpenMP when it is available: every node reads the
 * field of the previous step and writes only its own entries, so the results
 * do not depend on the number of threads.  The slice sampler's exact laws are
 * remembered in a table keyed by their arguments (caching only: each law is
 * still computed by the plain big-integer recursion below the first time).
 *
 * State layout used by every function here: n[3 * S] uint16, S = sum of the
 * replica lengths L[r]; plane i (0, 1, 2) holds the particles with velocity
 * v = i - 1 (-1, 0, +1); replica r occupies nodes [off_r, off_r + L[r]) of
 * each plane, off_r = L[0] + ... + L[r-1].  Lattices are periodic.
 *
 * Parity status of each function (pins live in tests/):
 *   orc_philox        pinned: cuRAND host Philox4x32-10 (library call).
 *   orc_feq           pinned: H-function minimiser (scipy), zero-velocity
 *                     weights, Omega^(1) = 0 of Eq. collmatD1Q3.
 *   orc_poisson_inv   pinned: scipy.stats.poisson.ppf.
 *   orc_decide        pinned: exact enumeration of the chunk stream.
 *   orc_step          pinned: exact rational enumeration of the paper's
 *                     particle picks (Sec. III) for N <= 12; conservation and
 *                     n_0 parity invariants; stationary law; Poisson means and
 *                     variances against Eq. D1Q3equil and Eq. poisson.
 *   orc_literal_step  pinned: same enumeration (its own random stream).
 *   orc_init          pinned: sample mean/variance against Eq. D1Q3equil.
 *   orc_moments       pinned: hand-computed small cases.
 *   orc_stats_*       pinned: hand-computed small cases; numpy cross-check.
 *   orc_galilean_q    pinned: 50-digit decimal evaluation of lt / sqrt(1 + 3 u^2).
 *   orc_slice_*       pinned: rational matrix powers of the one-sub-collision
 *                     matrix (N <= 10, and N = 150 by propagated fractions);
 *                     one-step law by chi-square; invariants; n_max below
 *                     every mass reduces it to orc_step bit for bit.
 *   orc_block_*       pinned: blocks stitched together equal orc_step /
 *                     orc_slice_step of the whole lattice (gloo ranks too).
 *   orc2_* (D2Q9)     pinned: the collision table against brute-force
 *                     enumeration and its symmetry classes; the linearised
 *                     operator against the paper's printed Eq. D2Q9MOmega;
 *                     detailed balance of the product Poisson law (N <= 5);
 *                     one-collision law by chi-square; conservation; pure
 *                     streaming; Eq. D2Q9eqdist against the H minimiser.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ERR_OVERFLOW 1u /* a transition would leave [0, 65535] */
#define ORC_ERR_SAMPLER 2u  /* decision still open after the refinement cap */

#define ORC_FLAG_NO_STREAM 1u /* collide only: local equilibration (Sec. IV.A, Fig. decay) */
#define ORC_FLAG_GALILEAN 4u  /* per-node lambda = lambda~ / sqrt(1 + 3 u^2) (end of Sec. IV.A) */

/* Random-stream purposes (top 4 bits of the fourth Philox counter word). */
#define PURPOSE_COLLIDE 0u
#define PURPOSE_REFINE 1u
#define PURPOSE_INIT 2u
#define PURPOSE_LITERAL 3u

#define CHUNKS_PER_BLOCK 10 /* 12-bit primary chunks per 128-bit Philox block */
#define MAX_REFINE 4        /* 16-bit refinement chunks allowed per decision */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two      */
/* 32x32->64 multiplications; the key is advanced by the Weyl constants      */
/* between rounds.                                                          */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void seed_key(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
}

/* Threads of the node loops (1 without OpenMP); n <= 0 selects every core. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The 128-bit value of one Philox block, word 0 least significant. */
static unsigned __int128 block128(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                  const uint32_t key[2])
{
    uint32_t ctr[4] = {c0, c1, c2, c3}, w[4];
    orc_philox(ctr, key, w);
    unsigned __int128 b = 0;
    for (int i = 3; i >= 0; i--) b = (b << 32) | w[i];
    return b;
}

/* ------------------------------------------------------------------------ */
/* Entropic D1Q3 equilibrium, Eq. D1Q3equil:                                 */
/*   f_i = rho w_i [1 + 3 v_i u + (3 v_i^2 - 1)(sqrt(1 + 3u^2) - 1)],         */
/*   w_0 = 2/3, w_{+-1} = 1/6 (Eq. D1Q3wi).                                   */
/* ------------------------------------------------------------------------ */
void orc_feq(double rho, double u, double f[3])
{
    const double w[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    double s = sqrt(1.0 + 3.0 * u * u) - 1.0;
    for (int i = 0; i < 3; i++) {
        double v = (double)(i - 1);
        f[i] = rho * w[i] * (1.0 + 3.0 * v * u + (3.0 * v * v - 1.0) * s);
    }
}

/* Poisson(mu) by inversion of the CDF: the smallest k with U < F(k), with the
 * probabilities built by p_k = p_{k-1} * (mu / k) from p_0 = exp(-mu).  Used
 * with mu <= 32 only; capped at k = 200. */
uint32_t orc_poisson_inv(double mu, double U)
{
    double p = exp(-mu);
    double F = p;
    uint32_t k = 0;
    while (U >= F && k < 200) {
        k++;
        p = p * (mu / (double)k);
        F = F + p;
    }
    return k;
}

/* Initial occupations n_i ~ Poisson(f_i^eq(rho(x), u(x))) (Eq. poisson).
 * Each mean is split into P = max(1, ceil(mu/32)) equal parts and the part
 * samples are summed (a sum of independent Poisson variables is Poisson).
 * Part p of plane i at (replica r, local node x) takes the uniform
 *   U = ((w_hi << 32 | w_lo) >> 11) * 2^-53
 * from Philox block (x, r, p/2, PURPOSE_INIT << 28 | i), words (0, 1) for
 * even p and (2, 3) for odd p.  Returns ORC_ERR_OVERFLOW if a count exceeds
 * 65535, 8 for an invalid (rho, u) (negative, non-finite or |u| > 1). */
int orc_init(const uint32_t *L, uint32_t R, uint64_t seed, const double *rho, const double *u,
             uint16_t *n, uint32_t r0)
{
    uint32_t key[2];
    seed_key(seed, key);
    uint64_t S = 0;
    for (uint32_t r = 0; r < R; r++) S += L[r];
    int err = 0;
    uint64_t off = 0;
    for (uint32_t r = 0; r < R; r++) {
#pragma omp parallel for schedule(static) reduction(| : err)
        for (uint32_t x = 0; x < L[r]; x++) {
            double rh = rho[off + x], uu = u[off + x];
            if (!(rh >= 0.0) || !isfinite(rh) || !(fabs(uu) <= 1.0)) {
                err |= 8;
                continue;
            }
            double f[3];
            orc_feq(rh, uu, f);
            for (uint32_t i = 0; i < 3; i++) {
                double mu = f[i] > 0.0 ? f[i] : 0.0;
                uint32_t parts = (uint32_t)ceil(mu / 32.0);
                if (parts < 1) parts = 1;
                double mup = mu / (double)parts;
                uint64_t total = 0;
                for (uint32_t p = 0; p < parts; p++) {
                    uint32_t ctr[4] = {x, r0 + r, p / 2, (PURPOSE_INIT << 28) | i}, w[4];
                    orc_philox(ctr, key, w);
                    uint32_t lo = (p % 2 == 0) ? w[0] : w[2];
                    uint32_t hi = (p % 2 == 0) ? w[1] : w[3];
                    uint64_t m = (((uint64_t)hi << 32) | lo) >> 11;
                    double U = (double)m * (1.0 / 9007199254740992.0);
                    total += orc_poisson_inv(mup, U);
                }
                if (total > 65535) {
                    err |= ORC_ERR_OVERFLOW;
                    total = 65535;
                }
                n[i * S + off + x] = (uint16_t)total;
            }
        }
        off += L[r];
    }
    return (err & 8) ? 8 : err;
}

/* ------------------------------------------------------------------------ */
/* Exact sampler of one sub-collision.                                       */
/*                                                                          */
/* With particles picked by two independent uniform draws of a particle      */
/* index in [1, N] (Eq. select; picking the same particle twice collides     */
/* nothing) and the D1Q3 table of Sec. III.A:                                */
/*   P(down: (a,b,c) -> (a-1,b+2,c-1)) = 2ac/N^2 * lambda        = T1/D      */
/*   P(up:   (a,b,c) -> (a+1,b-2,c+1)) = b(b-1)/N^2 * lambda/8   = (T2-T1)/D */
/* with T1 = 16 a c lam_n, T2 = T1 + b (b-1) lam_n, D = 8 N^2 lam_d,          */
/* (a, b, c) = (n_-1, n_0, n_+1), lambda = lam_n / lam_d.                    */
/*                                                                          */
/* The outcome is the region of a uniform real U in [0,1) against T1/D and  */
/* T2/D: U < T1/D -> down, T1/D <= U < T2/D -> up, otherwise nothing.  U's   */
/* binary expansion is a 12-bit primary chunk q0 followed, only while the    */
/* region is still open, by 16-bit refinement chunks.  Knowing the first     */
/* `bits` bits Q places U in [Q, Q+1) / 2^bits, so U < T/D is certain when    */
/* (Q+1) D <= T 2^bits and U >= T/D is certain when Q D >= T 2^bits.          */
/*                                                                          */
/* Returns 0 (down), 1 (up), 2 (nothing), -1 when more refinement chunks are */
/* needed than `nref` supplies, -2 past the MAX_REFINE cap.  *used = number  */
/* of refinement chunks read.                                               */
/* ------------------------------------------------------------------------ */
typedef int (*chunk_source)(void *ctx, int k, uint16_t *chunk); /* 0 = no chunk k */

static int decide(uint64_t T1, uint64_t T2, uint64_t D, uint32_t q0, chunk_source src, void *ctx,
                  int *used)
{
    unsigned __int128 Q = q0;
    int bits = 12;
    *used = 0;
    for (int k = 0;; k++) {
        unsigned __int128 lo = Q * (unsigned __int128)D;
        unsigned __int128 hi = lo + D;
        unsigned __int128 s1 = (unsigned __int128)T1 << bits;
        unsigned __int128 s2 = (unsigned __int128)T2 << bits;
        if (hi <= s1) return 0;
        if (lo >= s1 && hi <= s2) return 1;
        if (lo >= s2) return 2;
        if (k == MAX_REFINE) return -2;
        uint16_t next;
        if (!src(ctx, k, &next)) return -1;
        Q = (Q << 16) | next;
        bits += 16;
        *used = k + 1;
    }
}

typedef struct {
    const uint16_t *chunks;
    int n;
} chunk_array;

static int from_array(void *ctx, int k, uint16_t *chunk)
{
    chunk_array *a = (chunk_array *)ctx;
    if (k >= a->n) return 0;
    *chunk = a->chunks[k];
    return 1;
}

int orc_decide(uint64_t T1, uint64_t T2, uint64_t D, uint32_t q0, const uint16_t *ref, int nref,
               int *used)
{
    chunk_array a = {ref, nref};
    return decide(T1, T2, D, q0, from_array, &a, used);
}

/* Refinement chunk s of the node-step (x, r, t): 16-bit chunk s % 8 of Philox
 * block (x, r, t, PURPOSE_REFINE << 28 | s / 8), chunk m = bits [16m, 16m+16). */
static uint16_t refine_chunk(uint32_t x, uint32_t r, uint32_t t, uint32_t s, const uint32_t key[2])
{
    unsigned __int128 b = block128(x, r, t, (PURPOSE_REFINE << 28) | (s / 8), key);
    return (uint16_t)((b >> (16 * (s % 8))) & 0xFFFF);
}

typedef struct {
    uint32_t x, r, t, first;
    const uint32_t *key;
} refine_stream;

static int from_refine_stream(void *ctx, int k, uint16_t *chunk)
{
    refine_stream *rs = (refine_stream *)ctx;
    *chunk = refine_chunk(rs->x, rs->r, rs->t, rs->first + (uint32_t)k, rs->key);
    return 1;
}

/* Primary chunk of sub-collision c of the node-step (x, r, t): 12-bit chunk
 * m = c % 10 (bits [12m, 12m+12)) of Philox block (x, r, t, c / 10). */
static uint32_t primary_chunk(uint32_t x, uint32_t r, uint32_t t, uint32_t c, const uint32_t key[2])
{
    unsigned __int128 b = block128(x, r, t, (PURPOSE_COLLIDE << 28) | (c / CHUNKS_PER_BLOCK), key);
    return (uint32_t)((b >> (12 * (c % CHUNKS_PER_BLOCK))) & 0xFFF);
}

/* C sequential sub-collisions at one node (Sec. III, Eqs. select and omega):
 * each sub-collision acts on the state left by the previous one.  A node with
 * N < 2 has no pair to collide and is left as it is. */
static int collide_node(uint16_t st[3], uint32_t x, uint32_t r, uint32_t t, uint32_t C,
                        uint32_t lam_n, uint32_t lam_d, const uint32_t key[2])
{
    uint64_t a = st[0], b = st[1], c = st[2];
    uint64_t N = a + b + c;
    if (N < 2) return 0;
    uint64_t D = 8 * N * N * lam_d;
    uint32_t next_ref = 0; /* refinement chunks are consumed in order across the node-step */
    for (uint32_t k = 0; k < C; k++) {
        uint64_t T1 = 16 * a * c * lam_n;
        uint64_t T2 = T1 + (b > 0 ? b * (b - 1) : 0) * lam_n;
        uint32_t q0 = primary_chunk(x, r, t, k, key);
        refine_stream rs = {x, r, t, next_ref, key};
        int used = 0;
        int region = decide(T1, T2, D, q0, from_refine_stream, &rs, &used);
        next_ref += (uint32_t)used;
        if (region == -2) {
            st[0] = (uint16_t)a; st[1] = (uint16_t)b; st[2] = (uint16_t)c;
            return ORC_ERR_SAMPLER;
        }
        if (region == 0) { /* {-1, 1} -> {0, 0} */
            if (b + 2 > 65535) {
                st[0] = (uint16_t)a; st[1] = (uint16_t)b; st[2] = (uint16_t)c;
                return ORC_ERR_OVERFLOW;
            }
            a -= 1; b += 2; c -= 1;
        } else if (region == 1) { /* {0, 0} -> {-1, 1} */
            if (a + 1 > 65535 || c + 1 > 65535) {
                st[0] = (uint16_t)a; st[1] = (uint16_t)b; st[2] = (uint16_t)c;
                return ORC_ERR_OVERFLOW;
            }
            a += 1; b -= 2; c += 1;
        }
    }
    st[0] = (uint16_t)a; st[1] = (uint16_t)b; st[2] = (uint16_t)c;
    return 0;
}

/* Streaming, from the evolution equation n_i(x + v_i, t + 1) = n_i(x, t) + Xi_i
 * (Sec. III): post-collision particles at x move to x + v_i, periodically. */
static void stream(const uint32_t *L, uint32_t R, uint64_t S, const uint16_t *post, uint16_t *n)
{
    uint64_t off = 0;
    for (uint32_t r = 0; r < R; r++) {
        uint32_t Lr = L[r];
#pragma omp parallel for schedule(static) if (Lr >= 65536)
        for (uint32_t x = 0; x < Lr; x++) {
            for (int i = 0; i < 3; i++) {
                int v = i - 1;
                uint32_t dest = (uint32_t)(((int64_t)x + v + Lr) % Lr);
                n[i * S + off + dest] = post[i * S + off + x];
            }
        }
        off += Lr;
    }
}

/* Galilean-invariant collision rate (end of Sec. IV.A): lambda = lt / sqrt(1 + 3 u^2)
 * with the node's velocity u = J / N and lt = lt_n / lt_d, quantised down to q / 256:
 * the largest integer q with  q lt_d sqrt(N^2 + 3 J^2) <= 256 lt_n N,  i.e.
 * q^2 lt_d^2 (N^2 + 3 J^2) <= (256 lt_n N)^2, decided in 128-bit integers after a
 * floating-point first guess. */
uint32_t orc_galilean_q(uint32_t N, int32_t J, uint32_t lt_n, uint32_t lt_d)
{
    if (N == 0) return 0;
    unsigned __int128 R = (unsigned __int128)N * N + (unsigned __int128)3 * ((int64_t)J * J);
    unsigned __int128 rhs = (unsigned __int128)(256ull * lt_n * N) * (256ull * lt_n * N);
    double guess = 256.0 * lt_n * N / (lt_d * sqrt((double)R));
    uint64_t q = guess >= 256.0 ? 256 : (uint64_t)guess;
    while (q > 0 && (unsigned __int128)(q * q * lt_d * lt_d) * R > rhs) q--;
    while (q < 256 && (unsigned __int128)((q + 1) * (q + 1) * lt_d * lt_d) * R <= rhs) q++;
    return (uint32_t)q;
}

/* The node's collision rate as (numerator, denominator): the handle's lambda, or the
 * Galilean-invariant one when flags ask for it. */
static void node_lambda(uint32_t flags, uint32_t N, int32_t J, uint32_t lam_n, uint32_t lam_d,
                        uint32_t *ln, uint32_t *ld)
{
    if (flags & ORC_FLAG_GALILEAN) {
        *ln = orc_galilean_q(N, J, lam_n, lam_d);
        *ld = 256;
    } else {
        *ln = lam_n;
        *ld = lam_d;
    }
}

/* n_steps time steps from time t0.  n holds the pre-collision occupations
 * n_i(x, t0) on entry and n_i(x, t0 + n_steps) on return.  Collision at
 * (replica r, local node x, time t) draws from Philox counters (x, r0 + r,
 * t, .) with key (seed low 32 bits, seed high 32 bits).  Returns ORC_ERR_* bits;
 * after an error the state is unspecified. */
int orc_step(const uint32_t *L, uint32_t R, uint64_t seed, uint32_t C, uint32_t lam_n,
             uint32_t lam_d, uint32_t flags, uint16_t *n, uint64_t t0, uint64_t n_steps,
             uint32_t r0)
{
    uint32_t key[2];
    seed_key(seed, key);
    uint64_t S = 0;
    for (uint32_t r = 0; r < R; r++) S += L[r];
    uint16_t *post = (uint16_t *)malloc(3 * S * sizeof(uint16_t) + 1);
    if (!post) return 16;
    int err = 0;
    for (uint64_t s = 0; s < n_steps; s++) {
        uint32_t t = (uint32_t)(t0 + s);
#pragma omp parallel reduction(| : err)
        {
            uint64_t off = 0;
            for (uint32_t r = 0; r < R; r++) {
#pragma omp for schedule(static) nowait
                for (uint32_t x = 0; x < L[r]; x++) {
                    uint16_t st[3] = {n[0 * S + off + x], n[1 * S + off + x], n[2 * S + off + x]};
                    uint32_t ln, ld;
                    node_lambda(flags, (uint32_t)st[0] + st[1] + st[2],
                                (int32_t)st[2] - (int32_t)st[0], lam_n, lam_d, &ln, &ld);
                    err |= collide_node(st, x, r0 + r, t, C, ln, ld, key);
                    for (int i = 0; i < 3; i++) post[i * S + off + x] = st[i];
                }
                off += L[r];
            }
        }
        if (flags & ORC_FLAG_NO_STREAM)
            memcpy(n, post, 3 * S * sizeof(uint16_t));
        else
            stream(L, R, S, post, n);
    }
    free(post);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Literal form of the paper's algorithm (Sec. III): two uniform particle    */
/* indices r1, r2 in [1, N]; r -> velocity by cumulative counts in the order */
/* (-1, 0, +1) (Eq. select); the same particle twice collides nothing; then  */
/* the D1Q3 table of Sec. III.A.  Its random numbers come from a stream of   */
/* its own (PURPOSE_LITERAL), so it is a distribution reference, not a       */
/* bit-exact one.                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t x, r, t, blk, pos;
    uint32_t w[4];
    const uint32_t *key;
} word_stream;

static uint32_t next_word(word_stream *ws)
{
    if (ws->pos == 4) {
        uint32_t ctr[4] = {ws->x, ws->r, ws->t, (PURPOSE_LITERAL << 28) | ws->blk};
        orc_philox(ctr, ws->key, ws->w);
        ws->blk++;
        ws->pos = 0;
    }
    return ws->w[ws->pos++];
}

/* Uniform integer in [0, m) by rejection of the incomplete top range. */
static uint32_t uniform_below(word_stream *ws, uint32_t m)
{
    uint32_t limit = (uint32_t)((((uint64_t)1 << 32) / m) * m - 1);
    for (;;) {
        uint32_t w = next_word(ws);
        if (w <= limit) return w % m;
    }
}

int orc_literal_step(const uint32_t *L, uint32_t R, uint64_t seed, uint32_t C, uint32_t lam_n,
                     uint32_t lam_d, uint32_t flags, uint16_t *n, uint64_t t0, uint64_t n_steps,
                     uint32_t r0)
{
    uint32_t key[2];
    seed_key(seed, key);
    uint64_t S = 0;
    for (uint32_t r = 0; r < R; r++) S += L[r];
    uint16_t *post = (uint16_t *)malloc(3 * S * sizeof(uint16_t) + 1);
    if (!post) return 16;
    int err = 0;
    for (uint64_t s = 0; s < n_steps; s++) {
        uint32_t t = (uint32_t)(t0 + s);
        uint64_t off = 0;
        for (uint32_t r = 0; r < R; r++) {
            for (uint32_t x = 0; x < L[r]; x++) {
                int64_t cnt[3] = {n[off + x], n[S + off + x], n[2 * S + off + x]};
                word_stream ws = {x, r0 + r, t, 0, 4, {0, 0, 0, 0}, key};
                uint32_t N = (uint32_t)(cnt[0] + cnt[1] + cnt[2]);
                uint32_t ln, ld;
                node_lambda(flags, N, (int32_t)(cnt[2] - cnt[0]), lam_n, lam_d, &ln, &ld);
                for (uint32_t k = 0; k < C && N >= 2; k++) {
                    uint32_t r1 = 1 + uniform_below(&ws, N);
                    uint32_t r2 = 1 + uniform_below(&ws, N);
                    int s1 = r1 <= cnt[0] ? 0 : (r1 <= cnt[0] + cnt[1] ? 1 : 2);
                    int s2 = r2 <= cnt[0] ? 0 : (r2 <= cnt[0] + cnt[1] ? 1 : 2);
                    if (r1 == r2) continue; /* one particle cannot collide with itself */
                    if ((s1 == 0 && s2 == 2) || (s1 == 2 && s2 == 0)) {
                        /* P_{-1 1 -> 0 0} = P_{1 -1 -> 0 0} = lambda */
                        if (uniform_below(&ws, ld) < ln) {
                            cnt[0] -= 1; cnt[1] += 2; cnt[2] -= 1;
                        }
                    } else if (s1 == 1 && s2 == 1) {
                        /* P_{00 -> -1 1} = P_{00 -> 1 -1} = lambda / 16 */
                        uint32_t v = uniform_below(&ws, 16 * ld);
                        if (v < 2 * ln) {
                            cnt[0] += 1; cnt[1] -= 2; cnt[2] += 1;
                        }
                    }
                }
                for (int i = 0; i < 3; i++) {
                    if (cnt[i] < 0 || cnt[i] > 65535) err |= ORC_ERR_OVERFLOW;
                    post[i * S + off + x] = (uint16_t)cnt[i];
                }
            }
            off += L[r];
        }
        if (flags & ORC_FLAG_NO_STREAM)
            memcpy(n, post, 3 * S * sizeof(uint16_t));
        else
            stream(L, R, S, post, n);
    }
    free(post);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Node moments: mass N = sum_i n_i (Sec. III) and momentum J = N U =         */
/* sum_i n_i v_i = n_+1 - n_-1 (Sec. IV.A); exact int64 totals.              */
/* ------------------------------------------------------------------------ */
void orc_moments(const uint32_t *L, uint32_t R, const uint16_t *n, int32_t *N, int32_t *J,
                 int64_t totals[2])
{
    uint64_t S = 0;
    for (uint32_t r = 0; r < R; r++) S += L[r];
    totals[0] = 0;
    totals[1] = 0;
    for (uint64_t x = 0; x < S; x++) {
        int32_t a = n[x], b = n[S + x], c = n[2 * S + x];
        N[x] = a + b + c;
        J[x] = c - a;
        totals[0] += N[x];
        totals[1] += J[x];
    }
}

/* ------------------------------------------------------------------------ */
/* Ensemble statistics for Eqs. poisson, Poisson2, corr and error: per node  */
/* position x (all replicas have the same length L and are pooled),          */
/*   s1[3*x + i]       += n_i(x)                                             */
/*   s2[6*x + p]       += n_i(x) n_j(x),     p over (i,j) = 00 01 02 11 12 22 */
/*   snb[9*x + 3*i+j]  += n_i(x) n_j(x+1 mod L)                              */
/* and the sample count.  Exact in int64.                                   */
/* ------------------------------------------------------------------------ */
void orc_stats_accumulate(uint32_t Lc, uint32_t R, const uint16_t *n, int64_t *s1, int64_t *s2,
                          int64_t *snb, uint64_t *count)
{
    static const int pi[6] = {0, 0, 0, 1, 1, 2}, pj[6] = {0, 1, 2, 1, 2, 2};
    uint64_t S = (uint64_t)Lc * R;
    for (uint32_t r = 0; r < R; r++) {
        for (uint32_t x = 0; x < Lc; x++) {
            uint64_t g = (uint64_t)r * Lc + x;
            uint64_t g1 = (uint64_t)r * Lc + (x + 1) % Lc;
            int64_t v[3] = {n[g], n[S + g], n[2 * S + g]};
            int64_t w[3] = {n[g1], n[S + g1], n[2 * S + g1]};
            for (int i = 0; i < 3; i++) s1[3 * (uint64_t)x + i] += v[i];
            for (int p = 0; p < 6; p++) s2[6 * (uint64_t)x + p] += v[pi[p]] * v[pj[p]];
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) snb[9 * (uint64_t)x + 3 * i + j] += v[i] * w[j];
        }
    }
    *count += R;
}

/* Exact (co)variance from the int64 sums: (M s_ij - s_i s_j) / M^2, the
 * numerator in 128-bit integers, one FP64 division at the end. */
double orc_exact_cov(int64_t sij, int64_t si, int64_t sj, uint64_t M)
{
    __int128 num = (__int128)M * sij - (__int128)si * sj;
    long double d = (long double)M * (long double)M;
    return (double)((long double)num / d);
}

/* ------------------------------------------------------------------------ */
/* Slice sampler: the C sub-collisions of one node drawn at once.            */
/*                                                                          */
/* Mass N and momentum J are fixed by the collisions, so a node moves on the */
/* (N, J) slice, indexed by its rest count b (a = (N-J-b)/2, c = (N+J-b)/2). */
/* One sub-collision moves b to b+2 with probability T1(b)/D, to b-2 with    */
/* T_up(b)/D, else keeps it (thresholds of the sequential sampler above).    */
/* The law after C sub-collisions is the C-th power of that matrix: integer  */
/* numerators over D^C, computed here by plain dynamic programming in big    */
/* integers.  The node then takes b' = b + 2 d with d the first offset whose */
/* cumulative probability CDF[d] exceeds a uniform U.                        */
/*                                                                          */
/* Contract: U's first 64 bits are Q = h 2^48 + (w1 mod 2^16) 2^32 + w0:    */
/* h, the top 16 bits, is bits [16 (x mod 2), 16 (x mod 2) + 16) of word     */
/* (x/2) mod 4 of Philox block (x/8, r, t, PURPOSE_SLICE_TOP << 28), so      */
/* eight consecutive nodes share one block; (w0, w1) are words (0, 1) of     */
/* block (x/2, r, t, PURPOSE_SLICE << 28) for even x and words (2, 3) for    */
/* odd x; F[d] = min(floor(CDF[d] 2^64), 2^64 - 1); for d in                 */
/* [dmin, dmax) (the reachable range, CDF[dmax] = 1) U >= CDF[d] when         */
/* Q > F[d], U < CDF[d] when Q < F[d]; Q == F[d] is reported as              */
/* ORC_ERR_SAMPLER (probability below 2^-59 per node-step).  C <= 10.        */
/*                                                                          */
/* Range: the laws are tabulated for masses N <= n_max only; a node with     */
/* N > n_max takes the sequential sampler's C decisions instead (the same    */
/* counters and bits as orc_step gives that node).  Both are exact samplers  */
/* of the node's C sub-collisions, so the dynamics stay exact; the bits      */
/* depend on n_max as they depend on the seed.                              */
/* ------------------------------------------------------------------------ */
#define PURPOSE_SLICE 4u
#define PURPOSE_SLICE_TOP 6u
#define SLICE_MAX_C 10
#define BN_LIMBS 20 /* 640-bit unsigned integers in 32-bit limbs */

typedef struct {
    uint32_t w[BN_LIMBS]; /* least significant limb first */
} bignum;

static void bn_set(bignum *a, uint64_t v)
{
    memset(a->w, 0, sizeof(a->w));
    a->w[0] = (uint32_t)v;
    a->w[1] = (uint32_t)(v >> 32);
}

static void bn_add(bignum *r, const bignum *a)
{
    uint64_t carry = 0;
    for (int i = 0; i < BN_LIMBS; i++) {
        uint64_t s = (uint64_t)r->w[i] + a->w[i] + carry;
        r->w[i] = (uint32_t)s;
        carry = s >> 32;
    }
}

static void bn_sub(bignum *r, const bignum *a) /* r >= a */
{
    int64_t borrow = 0;
    for (int i = 0; i < BN_LIMBS; i++) {
        int64_t d = (int64_t)r->w[i] - a->w[i] - borrow;
        borrow = d < 0;
        r->w[i] = (uint32_t)(d + (borrow ? ((int64_t)1 << 32) : 0));
    }
}

static void bn_mul_small(bignum *r, uint64_t m)
{
    unsigned __int128 carry = 0;
    for (int i = 0; i < BN_LIMBS; i++) {
        unsigned __int128 p = (unsigned __int128)r->w[i] * m + carry;
        r->w[i] = (uint32_t)p;
        carry = p >> 32;
    }
}

static int bn_cmp(const bignum *a, const bignum *b)
{
    for (int i = BN_LIMBS - 1; i >= 0; i--) {
        if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
    }
    return 0;
}

static void bn_shl(bignum *a, int bits) /* 0 <= bits < 32 * BN_LIMBS */
{
    bignum r;
    memset(r.w, 0, sizeof(r.w));
    int limbs = bits / 32, sh = bits % 32;
    for (int i = BN_LIMBS - 1; i >= limbs; i--) {
        uint64_t v = (uint64_t)a->w[i - limbs] << sh;
        if (sh && i - limbs - 1 >= 0) v |= (uint64_t)a->w[i - limbs - 1] >> (32 - sh);
        r.w[i] = (uint32_t)v;
    }
    *a = r;
}

/* floor(num 2^64 / den) for num <= den, by binary long division. */
static uint64_t bn_frac64(const bignum *num, const bignum *den)
{
    bignum rem = *num;
    uint64_t q = 0;
    for (int i = 63; i >= 0; i--) {
        bn_shl(&rem, 1); /* rem = 2 rem: one more bit of the quotient */
        q <<= 1;
        if (bn_cmp(&rem, den) >= 0) {
            bn_sub(&rem, den);
            q |= 1;
        }
    }
    return q;
}

/* Transition thresholds of state b on the (N, J) slice (0 outside it). */
static void slice_thresholds(int64_t N, int64_t J, int64_t b, uint32_t lam_n, uint64_t *down,
                             uint64_t *up)
{
    int64_t aj = J < 0 ? -J : J;
    *down = 0;
    *up = 0;
    if (b < 0 || b > N - aj || ((N - aj - b) & 1)) return;
    int64_t a = (N - J - b) / 2, c = (N + J - b) / 2;
    *down = 16 * (uint64_t)a * (uint64_t)c * lam_n;
    *up = (b > 0 ? (uint64_t)b * (uint64_t)(b - 1) : 0) * lam_n;
}

/* F[d + C] = floor(CDF[d] 2^64) for d in [-C, C] and the reachable offsets
 * [*dmin, *dmax].  Returns 0, or -1 for C > SLICE_MAX_C. */
static int slice_cdf_compute(uint32_t N, int32_t J, uint32_t b, uint32_t C, uint32_t lam_n,
                             uint32_t lam_d, uint64_t *F, int32_t *dmin, int32_t *dmax)
{
    if (C > SLICE_MAX_C) return -1;
    const int W = 2 * SLICE_MAX_C + 1;
    int64_t aj = J < 0 ? -(int64_t)J : J;
    int64_t bmin = (N - aj) & 1;
    *dmin = (int32_t)(-(int64_t)C > (bmin - (int64_t)b) / 2 ? -(int64_t)C : (bmin - (int64_t)b) / 2);
    *dmax = (int32_t)((int64_t)C < ((int64_t)N - aj - b) / 2 ? (int64_t)C : ((int64_t)N - aj - b) / 2);
    if (N < 2) { /* no pair to collide: the law stays at offset 0 */
        for (int d = -(int)C; d <= (int)C; d++) F[d + (int)C] = d < 0 ? 0 : UINT64_MAX;
        return 0;
    }
    uint64_t D = 8 * (uint64_t)N * N * lam_d;
    bignum v[2 * SLICE_MAX_C + 1], nv[2 * SLICE_MAX_C + 1], den;
    for (int i = 0; i < W; i++) bn_set(&v[i], 0);
    bn_set(&v[SLICE_MAX_C], 1); /* all mass at offset 0 */
    bn_set(&den, 1);
    for (uint32_t step = 0; step < C; step++) {
        for (int i = 0; i < W; i++) {
            int d = i - SLICE_MAX_C;
            uint64_t down, up;
            slice_thresholds(N, J, (int64_t)b + 2 * d, lam_n, &down, &up);
            bignum stay = v[i];
            bn_mul_small(&stay, D - down - up);
            nv[i] = stay;
            if (i > 0) { /* from b + 2(d-1) by a down move (b grows by 2) */
                uint64_t dn, upx;
                slice_thresholds(N, J, (int64_t)b + 2 * (d - 1), lam_n, &dn, &upx);
                bignum t = v[i - 1];
                bn_mul_small(&t, dn);
                bn_add(&nv[i], &t);
            }
            if (i < W - 1) { /* from b + 2(d+1) by an up move (b shrinks by 2) */
                uint64_t dn, upx;
                slice_thresholds(N, J, (int64_t)b + 2 * (d + 1), lam_n, &dn, &upx);
                bignum t = v[i + 1];
                bn_mul_small(&t, upx);
                bn_add(&nv[i], &t);
            }
        }
        for (int i = 0; i < W; i++) v[i] = nv[i];
        bn_mul_small(&den, D);
    }
    bignum cum;
    bn_set(&cum, 0);
    for (int i = 0; i < W; i++) {
        int d = i - SLICE_MAX_C;
        bn_add(&cum, &v[i]);
        if (d < -(int)C || d > (int)C) continue;
        F[d + (int)C] = bn_cmp(&cum, &den) >= 0 ? UINT64_MAX : bn_frac64(&cum, &den);
    }
    return 0;
}

/* Remembered laws: an open-addressing table keyed by every argument of the
 * law, filled under a lock, read without one (a slot's key and values are
 * written before its state is published, and never change afterwards).  A
 * reader that meets an empty slot computes the law itself; when the table is
 * 3/4 full, new laws are computed but no longer remembered. */
#define CDF_SLOTS (1u << 19)
typedef struct {
    uint32_t ready; /* 0 empty, 1 published (atomic, release/acquire) */
    uint32_t N, b, C, lam_n, lam_d;
    int32_t J, dmin, dmax;
    uint64_t F[2 * SLICE_MAX_C + 1];
} cdf_slot;
static cdf_slot *cdf_table = NULL;
static uint32_t cdf_used = 0;

static uint32_t cdf_hash(uint32_t N, int32_t J, uint32_t b, uint32_t C, uint32_t lam_n,
                         uint32_t lam_d)
{
    uint64_t h = 1469598103934665603ull; /* FNV-1a over the six arguments */
    uint32_t k[6] = {N, (uint32_t)J, b, C, lam_n, lam_d};
    for (int i = 0; i < 6; i++) {
        h ^= k[i];
        h *= 1099511628211ull;
    }
    return (uint32_t)(h ^ (h >> 32)) & (CDF_SLOTS - 1);
}

static int cdf_match(const cdf_slot *e, uint32_t N, int32_t J, uint32_t b, uint32_t C,
                     uint32_t lam_n, uint32_t lam_d)
{
    return e->N == N && e->J == J && e->b == b && e->C == C && e->lam_n == lam_n &&
           e->lam_d == lam_d;
}

int orc_slice_cdf(uint32_t N, int32_t J, uint32_t b, uint32_t C, uint32_t lam_n, uint32_t lam_d,
                  uint64_t *F, int32_t *dmin, int32_t *dmax)
{
    if (C > SLICE_MAX_C) return -1;
    cdf_slot *table = __atomic_load_n(&cdf_table, __ATOMIC_ACQUIRE);
    uint32_t h = cdf_hash(N, J, b, C, lam_n, lam_d);
    if (table) {
        for (uint32_t i = h;; i = (i + 1) & (CDF_SLOTS - 1)) {
            const cdf_slot *e = &table[i];
            if (!__atomic_load_n(&e->ready, __ATOMIC_ACQUIRE)) break;
            if (cdf_match(e, N, J, b, C, lam_n, lam_d)) {
                memcpy(F, e->F, (2 * C + 1) * sizeof(uint64_t));
                *dmin = e->dmin;
                *dmax = e->dmax;
                return 0;
            }
        }
    }
    int rc = slice_cdf_compute(N, J, b, C, lam_n, lam_d, F, dmin, dmax);
#pragma omp critical(orc_cdf_table)
    {
        if (!cdf_table) __atomic_store_n(&cdf_table, (cdf_slot *)calloc(CDF_SLOTS, sizeof(cdf_slot)),
                                         __ATOMIC_RELEASE);
        if (cdf_table && cdf_used < CDF_SLOTS / 4 * 3) {
            uint32_t i = h;
            while (cdf_table[i].ready && !cdf_match(&cdf_table[i], N, J, b, C, lam_n, lam_d))
                i = (i + 1) & (CDF_SLOTS - 1);
            cdf_slot *e = &cdf_table[i];
            if (!e->ready) {
                e->N = N; e->J = J; e->b = b; e->C = C; e->lam_n = lam_n; e->lam_d = lam_d;
                e->dmin = *dmin;
                e->dmax = *dmax;
                memcpy(e->F, F, (2 * C + 1) * sizeof(uint64_t));
                __atomic_store_n(&e->ready, 1u, __ATOMIC_RELEASE);
                cdf_used++;
            }
        }
    }
    return rc;
}

/* The 64-bit uniform prefix Q of node x of replica r at time t (the
 * contract above). */
uint64_t orc_slice_q(uint32_t x, uint32_t r, uint32_t t, const uint32_t key[2])
{
    uint32_t top_ctr[4] = {x / 8, r, t, PURPOSE_SLICE_TOP << 28}, top[4];
    orc_philox(top_ctr, key, top);
    uint64_t h = (top[(x / 2) % 4] >> (16 * (x % 2))) & 0xFFFFu;
    uint32_t ctr[4] = {x / 2, r, t, PURPOSE_SLICE << 28}, w[4];
    orc_philox(ctr, key, w);
    uint32_t lo = (x % 2 == 0) ? w[0] : w[2];
    uint32_t mid = ((x % 2 == 0) ? w[1] : w[3]) & 0xFFFFu;
    return (h << 48) | ((uint64_t)mid << 32) | lo;
}

/* The new rest count of one node, or -1 for an undecided prefix. */
int64_t orc_slice_draw(uint32_t N, int32_t J, uint32_t b, uint64_t Q, uint32_t C,
                          uint32_t lam_n, uint32_t lam_d)
{
    uint64_t F[2 * SLICE_MAX_C + 1];
    int32_t dmin, dmax;
    orc_slice_cdf(N, J, b, C, lam_n, lam_d, F, &dmin, &dmax);
    int32_t d = dmin;
    for (int32_t k = dmin; k < dmax; k++) {
        if (Q == F[k + (int32_t)C]) return -1;
        if (Q > F[k + (int32_t)C]) d = k + 1;
    }
    return (int64_t)b + 2 * d;
}

int orc_slice_step(const uint32_t *L, uint32_t R, uint64_t seed, uint32_t C, uint32_t lam_n,
                   uint32_t lam_d, uint32_t flags, uint16_t *n, uint64_t t0, uint64_t n_steps,
                   uint32_t r0, uint32_t n_max)
{
    if (C > SLICE_MAX_C) return 8;
    uint32_t key[2];
    seed_key(seed, key);
    uint64_t S = 0;
    for (uint32_t r = 0; r < R; r++) S += L[r];
    uint16_t *post = (uint16_t *)malloc(3 * S * sizeof(uint16_t) + 1);
    if (!post) return 16;
    int err = 0;
    for (uint64_t s = 0; s < n_steps; s++) {
        uint32_t t = (uint32_t)(t0 + s);
#pragma omp parallel reduction(| : err)
        {
        uint64_t off = 0;
        for (uint32_t r = 0; r < R; r++) {
#pragma omp for schedule(static) nowait
            for (uint32_t x = 0; x < L[r]; x++) {
                uint32_t a = n[off + x], b = n[S + off + x], c = n[2 * S + off + x];
                uint32_t N = a + b + c;
                int32_t J = (int32_t)c - (int32_t)a;
                uint32_t ln, ld;
                node_lambda(flags, N, J, lam_n, lam_d, &ln, &ld);
                if (N > n_max) {
                    uint16_t st[3] = {(uint16_t)a, (uint16_t)b, (uint16_t)c};
                    err |= collide_node(st, x, r0 + r, t, C, ln, ld, key);
                    a = st[0];
                    b = st[1];
                    c = st[2];
                } else if (N >= 2) {
                    uint64_t Q = orc_slice_q(x, r0 + r, t, key);
                    int64_t nb = orc_slice_draw(N, J, b, Q, C, ln, ld);
                    if (nb < 0) {
                        err |= ORC_ERR_SAMPLER;
                    } else {
                        b = (uint32_t)nb;
                        a = (uint32_t)(((int64_t)N - J - nb) / 2);
                        c = (uint32_t)(((int64_t)N + J - nb) / 2);
                        if (a > 65535 || b > 65535 || c > 65535) err |= ORC_ERR_OVERFLOW;
                    }
                }
                post[off + x] = (uint16_t)a;
                post[S + off + x] = (uint16_t)b;
                post[2 * S + off + x] = (uint16_t)c;
            }
            off += L[r];
        }
        }
        if (flags & ORC_FLAG_NO_STREAM)
            memcpy(n, post, 3 * S * sizeof(uint16_t));
        else
            stream(L, R, S, post, n);
    }
    free(post);
    return err;
}

/* ------------------------------------------------------------------------ */
/* One block of a larger periodic lattice (domain decomposition of a single  */
/* lattice over several ranks).  The evolution equation of Sec. III moves    */
/* one particle population per link and step: across the cut on each side of */
/* a block, one value leaves and one arrives per step.                       */
/*                                                                          */
/* The block holds global nodes [x0, x0 + Lb) of a lattice whose random      */
/* numbers are keyed by the global node index (replica index r).  A step is  */
/* split in two at the exchange:                                             */
/*   orc_block_collide  the C sub-collisions of every node of the block at    */
/*                      time t (sampler 0 sequential, 1 slice with n_max),   */
/*                      giving the post-collision field; out[0] = the v = -1 */
/*                      value of the first node (it leaves to the left),     */
/*                      out[1] = the v = +1 value of the last node (it       */
/*                      leaves to the right);                                */
/*   orc_block_stream   streaming inside the block; the first node's v = +1  */
/*                      value is in[0] (from the left neighbour's out[1]),   */
/*                      the last node's v = -1 value is in[1] (from the      */
/*                      right neighbour's out[0]).                           */
/* With one block covering the lattice and in = (out[1], out[0]) this is     */
/* exactly orc_step / orc_slice_step.                                        */
/* ------------------------------------------------------------------------ */
int orc_block_collide(uint32_t Lb, uint32_t x0, uint32_t r, uint64_t seed, uint32_t C,
                      uint32_t lam_n, uint32_t lam_d, uint32_t flags, uint32_t sampler,
                      uint32_t n_max, const uint16_t *n, uint16_t *post, uint32_t t,
                      uint16_t out[2])
{
    if (sampler == 1 && C > SLICE_MAX_C) return 8;
    uint32_t key[2];
    seed_key(seed, key);
    int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (uint32_t y = 0; y < Lb; y++) {
        uint32_t x = x0 + y; /* global node index: the random numbers' counter */
        uint32_t a = n[y], b = n[Lb + y], c = n[2 * (uint64_t)Lb + y];
        uint32_t N = a + b + c;
        int32_t J = (int32_t)c - (int32_t)a;
        uint32_t ln, ld;
        node_lambda(flags, N, J, lam_n, lam_d, &ln, &ld);
        if (sampler == 0 || N > n_max) {
            uint16_t st[3] = {(uint16_t)a, (uint16_t)b, (uint16_t)c};
            err |= collide_node(st, x, r, t, C, ln, ld, key);
            a = st[0];
            b = st[1];
            c = st[2];
        } else if (N >= 2) {
            int64_t nb = orc_slice_draw(N, J, b, orc_slice_q(x, r, t, key), C, ln, ld);
            if (nb < 0) {
                err |= ORC_ERR_SAMPLER;
            } else {
                b = (uint32_t)nb;
                a = (uint32_t)(((int64_t)N - J - nb) / 2);
                c = (uint32_t)(((int64_t)N + J - nb) / 2);
            }
        }
        post[y] = (uint16_t)a;
        post[Lb + y] = (uint16_t)b;
        post[2 * (uint64_t)Lb + y] = (uint16_t)c;
    }
    out[0] = post[0];
    out[1] = post[2 * (uint64_t)Lb + Lb - 1];
    return err;
}

void orc_block_stream(uint32_t Lb, const uint16_t *post, const uint16_t in[2], uint16_t *n)
{
    for (uint32_t y = 0; y < Lb; y++) {
        n[y] = y + 1 < Lb ? post[y + 1] : in[1];                          /* v = -1 from the right */
        n[Lb + y] = post[Lb + y];                                         /* v = 0 stays */
        n[2 * (uint64_t)Lb + y] = y > 0 ? post[2 * (uint64_t)Lb + y - 1] : in[0]; /* v = +1 from the left */
    }
}

/* ======================================================================== */
/* D2Q9 (Sec. II.B, III.B, IV.B): velocities v = (vx, vy), vx, vy in        */
/* {-1, 0, 1}, numbered 0 = (0,0), 1 = (1,0), 2 = (0,1), 3 = (-1,0),        */
/* 4 = (0,-1), 5 = (1,1), 6 = (-1,1), 7 = (-1,-1), 8 = (1,-1); weights       */
/* w = 4/9, 1/9 (1-4), 1/36 (5-8), products of the D1Q3 weights.            */
/*                                                                          */
/* Binary collisions: every pair of unordered velocity pairs {A, B} with the */
/* same total momentum, grouped into the nine equivalence classes of Sec.   */
/* III.B under the rotations and reflections of the square.  Numbering is   */
/* the one of the relaxation coefficients in Eq. D2Q9MOmega (the rates      */
/* lambda_1 .. lambda_9 of the simulations): class 1 {0,5}<->{1,2}, 2       */
/* {0,0}<->{1,3}, 3 {0,0}<->{5,7}, 4 {1,3}<->{5,7}, 5 {1,3}<->{2,4}, 6      */
/* {5,7}<->{6,8}, 7 {0,1}<->{2,8}, 8 {1,6}<->{3,5}, 9 {1,1}<->{5,8}.        */
/* Probabilities, as for D1Q3 (Sec. III.A): from the pair whose ordered     */
/* picks are less likely at equilibrium (smaller m w_i w_j, m = 2 for two   */
/* different velocities, 1 for equal ones) to the other pair lambda_c; back  */
/* lambda_c times the ratio of the two m w w products (detailed balance).   */
/* ======================================================================== */
static const int V2X[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int V2Y[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

static int vel2(int vx, int vy)
{
    for (int i = 0; i < 9; i++)
        if (V2X[i] == vx && V2Y[i] == vy) return i;
    return -1;
}

/* m w_i w_j for the unordered pair {i, j}, in units of 1/1296 (w = 36/81,
 * 9/81... written as 16/36^2 etc.): w_i * 36 is 16, 4 or 1. */
static uint32_t mww(int i, int j)
{
    static const uint32_t w36[9] = {16, 4, 4, 4, 4, 1, 1, 1, 1};
    return (i == j ? 1u : 2u) * w36[i] * w36[j];
}

typedef struct {
    int a0, a1, b0, b1; /* the two unordered pairs (a0 <= a1, b0 <= b1) */
    int cls;            /* 1 .. 9 */
} coll2;

static coll2 orc2_colls[64];
static int orc2_ncolls = 0;

static void orc2_add(int cls, int i, int j, int k, int l)
{
    int a0 = i < j ? i : j, a1 = i < j ? j : i, b0 = k < l ? k : l, b1 = k < l ? l : k;
    if (a0 > b0 || (a0 == b0 && a1 > b1)) { /* store the smaller pair first */
        int t0 = a0, t1 = a1;
        a0 = b0; a1 = b1; b0 = t0; b1 = t1;
    }
    for (int c = 0; c < orc2_ncolls; c++)
        if (orc2_colls[c].a0 == a0 && orc2_colls[c].a1 == a1 && orc2_colls[c].b0 == b0 &&
            orc2_colls[c].b1 == b1)
            return;
    coll2 e = {a0, a1, b0, b1, cls};
    orc2_colls[orc2_ncolls++] = e;
}

/* The 30 collisions: each class representative under the 8 symmetries
 * (x, y) -> (sx * (swap ? y : x), sy * (swap ? x : y)). */
static void orc2_build_collisions(void)
{
    if (orc2_ncolls) return;
    static const int rep[9][4] = {{0, 5, 1, 2}, {0, 0, 1, 3}, {0, 0, 5, 7}, {1, 3, 5, 7},
                                  {1, 3, 2, 4}, {5, 7, 6, 8}, {0, 1, 2, 8}, {1, 6, 3, 5},
                                  {1, 1, 5, 8}};
    for (int c = 0; c < 9; c++)
        for (int sw = 0; sw < 2; sw++)
            for (int sx = -1; sx <= 1; sx += 2)
                for (int sy = -1; sy <= 1; sy += 2) {
                    int img[4];
                    for (int q = 0; q < 4; q++) {
                        int x = V2X[rep[c][q]], y = V2Y[rep[c][q]];
                        int nx = sx * (sw ? y : x), ny = sy * (sw ? x : y);
                        img[q] = vel2(nx, ny);
                    }
                    orc2_add(c + 1, img[0], img[1], img[2], img[3]);
                }
}

int orc2_collision_count(void)
{
    orc2_build_collisions();
    return orc2_ncolls;
}

/* Collision k: its two pairs and class (for checking the table). */
void orc2_collision(int k, int out[5])
{
    orc2_build_collisions();
    out[0] = orc2_colls[k].a0; out[1] = orc2_colls[k].a1;
    out[2] = orc2_colls[k].b0; out[3] = orc2_colls[k].b1;
    out[4] = orc2_colls[k].cls;
}

/* Outcomes of an ordered pick of velocities (s1, s2) of two different
 * particles: the pairs B it may turn into, in increasing order of (b0, b1),
 * with integer numerators over D = 128 * lam_den: P = lam_num[c] / lam_den
 * times the ratio mww(lower) / mww(upper) (a power of 2 down to 1/128) when
 * the pick is the more likely pair.  Returns the number of outcomes. */
int orc2_outcomes(int s1, int s2, const uint32_t lam_num[9], uint32_t lam_den, int targets[8],
                  uint64_t nums[4])
{
    orc2_build_collisions();
    int a0 = s1 < s2 ? s1 : s2, a1 = s1 < s2 ? s2 : s1;
    int n = 0;
    for (int c = 0; c < orc2_ncolls; c++) {
        const coll2 *e = &orc2_colls[c];
        int b0, b1;
        if (e->a0 == a0 && e->a1 == a1) { b0 = e->b0; b1 = e->b1; }
        else if (e->b0 == a0 && e->b1 == a1) { b0 = e->a0; b1 = e->a1; }
        else continue;
        uint32_t from = mww(a0, a1), to = mww(b0, b1);
        /* lambda from the smaller m w w product; the other way scaled by the ratio */
        uint64_t num = (uint64_t)lam_num[e->cls - 1] * 128u;
        if (from > to) num = num * to / from; /* to / from = 2^-k with k <= 7: exact */
        /* insert in increasing (b0, b1) */
        int pos = n;
        while (pos > 0 && (targets[2 * (pos - 1)] > b0 ||
                           (targets[2 * (pos - 1)] == b0 && targets[2 * (pos - 1) + 1] > b1))) {
            targets[2 * pos] = targets[2 * (pos - 1)];
            targets[2 * pos + 1] = targets[2 * (pos - 1) + 1];
            nums[pos] = nums[pos - 1];
            pos--;
        }
        targets[2 * pos] = b0;
        targets[2 * pos + 1] = b1;
        nums[pos] = num;
        n++;
    }
    (void)lam_den;
    return n;
}

/* Entropic D2Q9 equilibrium, Eq. D2Q9eqdist: the product over x and y of the
 * D1Q3 factors w_{v_a} [1 + 3 v_a u_a + (3 v_a^2 - 1)(sqrt(1 + 3 u_a^2) - 1)]. */
void orc2_feq(double rho, double ux, double uy, double f[9])
{
    const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0}; /* v = -1, 0, +1 */
    double sx = sqrt(1.0 + 3.0 * ux * ux) - 1.0, sy = sqrt(1.0 + 3.0 * uy * uy) - 1.0;
    for (int i = 0; i < 9; i++) {
        double vx = V2X[i], vy = V2Y[i];
        double gx = w1[V2X[i] + 1] * (1.0 + 3.0 * vx * ux + (3.0 * vx * vx - 1.0) * sx);
        double gy = w1[V2Y[i] + 1] * (1.0 + 3.0 * vy * uy + (3.0 * vy * vy - 1.0) * sy);
        f[i] = rho * gx * gy;
    }
}

/* n_i(x, y, 0) ~ Poisson(f_i^eq(rho, ux, uy)) per node (Eq. poisson), split into
 * parts of mean <= 32 like orc_init; part p of velocity i at node g = y Lx + x
 * of replica r takes U from Philox block (g, r, p/2, PURPOSE_INIT << 28 | i),
 * words (0, 1) for even p and (2, 3) for odd p.  n is [9][R Lx Ly]. */
int orc2_init(uint32_t Lx, uint32_t Ly, uint32_t R, uint64_t seed, const double *rho,
              const double *ux, const double *uy, uint16_t *n, uint32_t r0)
{
    uint32_t key[2];
    seed_key(seed, key);
    const uint64_t G = (uint64_t)Lx * Ly, S = G * R;
    int err = 0;
    for (uint32_t r = 0; r < R; r++) {
#pragma omp parallel for schedule(static) reduction(| : err)
        for (uint64_t g = 0; g < G; g++) {
            uint64_t o = (uint64_t)r * G + g;
            double rh = rho[o], u1 = ux[o], u2 = uy[o];
            if (!(rh >= 0.0) || !isfinite(rh) || !(fabs(u1) <= 1.0) || !(fabs(u2) <= 1.0)) {
                err |= 8;
                continue;
            }
            double f[9];
            orc2_feq(rh, u1, u2, f);
            for (uint32_t i = 0; i < 9; i++) {
                double mu = f[i] > 0.0 ? f[i] : 0.0;
                uint32_t parts = (uint32_t)ceil(mu / 32.0);
                if (parts < 1) parts = 1;
                double mup = mu / (double)parts;
                uint64_t total = 0;
                for (uint32_t p = 0; p < parts; p++) {
                    uint32_t ctr[4] = {(uint32_t)g, r0 + r, p / 2, (PURPOSE_INIT << 28) | i}, w[4];
                    orc_philox(ctr, key, w);
                    uint32_t lo = (p % 2 == 0) ? w[0] : w[2];
                    uint32_t hi = (p % 2 == 0) ? w[1] : w[3];
                    uint64_t m = (((uint64_t)hi << 32) | lo) >> 11;
                    total += orc_poisson_inv(mup, (double)m * (1.0 / 9007199254740992.0));
                }
                if (total > 65535) {
                    err |= ORC_ERR_OVERFLOW;
                    total = 65535;
                }
                n[i * S + o] = (uint16_t)total;
            }
        }
    }
    return (err & 8) ? 8 : err;
}

/* The stream of 32-bit random words of one node-step: word k is word k % 4 of
 * Philox block (g, r, t, PURPOSE_D2Q9 << 28 | k / 4). */
#define PURPOSE_D2Q9 5u

/* Words of a node-step: at most 16 C + 64 (a sub-collision takes 2 or 3 plus
 * the rare rejections; running out is reported as a sampler error). */
typedef struct {
    uint32_t g, r, t, k, cap;
    uint32_t w[4];
    const uint32_t *key;
} word2_stream;

static int next_word2(word2_stream *s, uint32_t *out)
{
    if (s->k >= s->cap) return 0;
    if (s->k % 4 == 0) {
        uint32_t ctr[4] = {s->g, s->r, s->t, (PURPOSE_D2Q9 << 28) | (s->k / 4)};
        orc_philox(ctr, s->key, s->w);
    }
    *out = s->w[s->k % 4];
    s->k++;
    return 1;
}

/* A uniform integer in [0, m), 1 <= m < 2^32, exactly: the multiply-shift
 * method with rejection of Lemire (2019, "Fast random integer generation in an
 * interval"): x m = hi 2^32 + lo with x a uniform word; lo < (2^32 - m) mod m
 * is rejected and a new word drawn.  Returns 0 when the words run out. */
static int uniform_below2(word2_stream *s, uint32_t m, uint32_t *out)
{
    uint32_t x;
    if (!next_word2(s, &x)) return 0;
    uint64_t prod = (uint64_t)x * m;
    uint32_t lo = (uint32_t)prod;
    if (lo < m) {
        uint32_t thr = (uint32_t)(-m) % m; /* (2^32 - m) mod m */
        while (lo < thr) {
            if (!next_word2(s, &x)) return 0;
            prod = (uint64_t)x * m;
            lo = (uint32_t)prod;
        }
    }
    *out = (uint32_t)(prod >> 32);
    return 1;
}

/* The velocity of particle index q in [0, N): the smallest s with
 * q < n_0 + ... + n_s (Eq. select, velocities in the numbering above). */
static int velocity_of2(const uint32_t n[9], uint32_t q)
{
    uint32_t cum = 0;
    for (int s = 0; s < 9; s++) {
        cum += n[s];
        if (q < cum) return s;
    }
    return 8;
}

/* C sub-collisions at one D2Q9 node (Sec. III's algorithm: two uniform
 * particle picks; the same particle twice collides nothing; otherwise the
 * pair's outcomes by one uniform integer below D = 128 lam_den against the
 * cumulative numerators, none if it lies beyond them).  N < 2: nothing, no
 * words. */
static int collide2(uint32_t st[9], uint32_t g, uint32_t r, uint32_t t, uint32_t C,
                    const uint32_t lam_num[9], uint32_t lam_den, const uint32_t key[2])
{
    uint32_t N = 0;
    for (int i = 0; i < 9; i++) N += st[i];
    if (N < 2) return 0;
    word2_stream ws = {g, r, t, 0, 16u * C + 64u, {0, 0, 0, 0}, key};
    const uint32_t D = 128u * lam_den;
    for (uint32_t k = 0; k < C; k++) {
        uint32_t q1, q2;
        if (!uniform_below2(&ws, N, &q1) || !uniform_below2(&ws, N, &q2)) return ORC_ERR_SAMPLER;
        if (q1 == q2) continue;
        int s1 = velocity_of2(st, q1), s2 = velocity_of2(st, q2);
        int targets[8];
        uint64_t nums[4];
        int no = orc2_outcomes(s1, s2, lam_num, lam_den, targets, nums);
        if (no == 0) continue;
        uint32_t u;
        if (!uniform_below2(&ws, D, &u)) return ORC_ERR_SAMPLER;
        uint64_t cum = 0;
        for (int o = 0; o < no; o++) {
            cum += nums[o];
            if (u < cum) {
                int b0 = targets[2 * o], b1 = targets[2 * o + 1];
                st[s1]--; st[s2]--;
                st[b0]++; st[b1]++;
                if (st[b0] > 65535 || st[b1] > 65535) return ORC_ERR_OVERFLOW;
                break;
            }
        }
    }
    return 0;
}

/* n_steps time steps of R periodic Lx x Ly lattices, n[9][R Lx Ly] with node
 * g = y Lx + x of replica r at r Lx Ly + g; streaming n_i(x + v_i, t + 1) =
 * post_i(x, t) (Sec. III's evolution equation in two dimensions). */
int orc2_step(uint32_t Lx, uint32_t Ly, uint32_t R, uint64_t seed, uint32_t C,
              const uint32_t lam_num[9], uint32_t lam_den, uint32_t flags, uint16_t *n,
              uint64_t t0, uint64_t n_steps, uint32_t r0)
{
    uint32_t key[2];
    seed_key(seed, key);
    orc2_build_collisions();
    const uint64_t G = (uint64_t)Lx * Ly, S = G * R;
    uint16_t *post = (uint16_t *)malloc(9 * S * sizeof(uint16_t) + 1);
    if (!post) return 16;
    int err = 0;
    for (uint64_t s = 0; s < n_steps; s++) {
        uint32_t t = (uint32_t)(t0 + s);
        for (uint32_t r = 0; r < R; r++) {
#pragma omp parallel for schedule(static) reduction(| : err)
            for (uint64_t g = 0; g < G; g++) {
                uint64_t o = (uint64_t)r * G + g;
                uint32_t st[9];
                for (int i = 0; i < 9; i++) st[i] = n[i * S + o];
                err |= collide2(st, (uint32_t)g, r0 + r, t, C, lam_num, lam_den, key);
                for (int i = 0; i < 9; i++) post[i * S + o] = (uint16_t)st[i];
            }
        }
        if (flags & ORC_FLAG_NO_STREAM) {
            memcpy(n, post, 9 * S * sizeof(uint16_t));
            continue;
        }
        for (uint32_t r = 0; r < R; r++)
            for (uint32_t y = 0; y < Ly; y++)
                for (uint32_t x = 0; x < Lx; x++)
                    for (int i = 0; i < 9; i++) {
                        uint32_t xd = (x + Lx + V2X[i]) % Lx, yd = (y + Ly + V2Y[i]) % Ly;
                        n[i * S + (uint64_t)r * G + (uint64_t)yd * Lx + xd] =
                            post[i * S + (uint64_t)r * G + (uint64_t)y * Lx + x];
                    }
    }
    free(post);
    return err;
}

/* Density and momentum per node (Eq. MomD2Q9's first three moments without
 * the sqrt(3) of the normalisation): rho = sum n_i, j = sum n_i v_i. */
void orc2_moments(uint64_t S, const uint16_t *n, int32_t *rho, int32_t *jx, int32_t *jy,
                  int64_t totals[3])
{
    totals[0] = totals[1] = totals[2] = 0;
    for (uint64_t o = 0; o < S; o++) {
        int32_t a = 0, bx = 0, by = 0;
        for (int i = 0; i < 9; i++) {
            int32_t v = n[i * S + o];
            a += v;
            bx += v * V2X[i];
            by += v * V2Y[i];
        }
        rho[o] = a; jx[o] = bx; jy[o] = by;
        totals[0] += a; totals[1] += bx; totals[2] += by;
    }
}
