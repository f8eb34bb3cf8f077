/*
 * mclg.h - C ABI of the GB300 (sm_103a) D1Q3 Monte Carlo Lattice Gas library.
 *
 * The method (Blommel & Wagner, arXiv:1706.01094): integer occupation numbers
 * n_i(x, t), i <-> v_i in {-1, 0, +1}, on periodic 1D lattices evolve by
 *     n_i(x + v_i, t + 1) = n_i(x, t) + Xi_i                      (Sec. III)
 * where Xi is the sum of C random binary sub-collisions at each node, each
 * acting on the state left by the previous one.  A sub-collision picks two
 * particles uniformly (Eq. select) and applies the D1Q3 table of Sec. III.A:
 * {-1, +1} -> {0, 0} with probability lambda, {0, 0} -> {-1, +1} with
 * probability lambda/8 (two orderings of lambda/16).  Mass N = sum n_i and
 * momentum J = n_+1 - n_-1 are conserved exactly at every node.
 *
 * Exact sampling contract (identical on every execution path, so results do
 * not depend on the kernel, tile shape or batch composition):
 *   - Random bits: Philox4x32-10, key (seed & 0xffffffff, seed >> 32),
 *     counter (x, r, t, purpose << 28 | block) with x the replica-local node,
 *     r the replica index (plus mclg_params.first_replica), t the time step
 *     (t < 2^32).
 *   - Sub-collision k at node (x, r) and time t draws a uniform real U whose
 *     first 12 bits are bits [12m, 12m+12) (m = k % 10) of the 128-bit block
 *     (x, r, t, k / 10) (word 0 least significant); while U's region is still
 *     undecided, the next bits come as 16-bit chunks, in order, from blocks
 *     (x, r, t, 1 << 28 | j) (chunk s = bits [16(s%8), 16(s%8)+16) of block
 *     j = s / 8), counted across the node's whole time step.
 *   - With (a, b, c) = (n_-1, n_0, n_+1), N = a + b + c, lambda = ln / ld:
 *     T1 = 16 a c ln, T2 = T1 + b (b - 1) ln, D = 8 N^2 ld.
 *     U < T1/D: (a-1, b+2, c-1); T1/D <= U < T2/D: (a+1, b-2, c+1); else no
 *     change.  Nodes with N < 2 are left as they are.
 *   - Initial occupations (mclg_init): n_i ~ Poisson(f_i^eq(rho, u)) with the
 *     entropic equilibrium of Eq. D1Q3equil, sampled on the host in FP64 by
 *     CDF inversion over parts of mean <= 32 (purpose 2).
 *
 * Layout of every state array crossing this ABI: uint16 n[3][S], S = sum of
 * the replica lengths, plane i = 0, 1, 2 for v = -1, 0, +1, replica r at
 * nodes [L[0] + ... + L[r-1], ... + L[r]).  Arrays may be host or device
 * pointers (detected with cudaPointerGetAttributes).
 *
 * Ownership: the library owns every device buffer it allocates; the caller
 * owns every array it passes and may free it when the call returns.
 * Errors: every call returns an mclg_status; nothing is thrown across the
 * ABI.  Device-side errors (overflow, sampler cap) are sticky: they are
 * reported by mclg_sync and by every later call until mclg_init or
 * mclg_set_state replaces the state.  A handle is not thread-safe; all its
 * work is ordered on its CUDA stream.
 */
#ifndef MCLG_H
#define MCLG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mclg_ctx *mclg_handle;

typedef enum {
    MCLG_OK = 0,
    MCLG_ERR_ARG = 1,      /* invalid argument */
    MCLG_ERR_NOMEM = 2,    /* device or host allocation failed */
    MCLG_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    MCLG_ERR_OVERFLOW = 4, /* an occupation would leave [0, 65535]; state unspecified */
    MCLG_ERR_TIMEOUT = 5,  /* a bounded device-side wait gave up (the warp-specialised
                              slice kernel's pipeline waits, about 2 s each); state unspecified */
    MCLG_ERR_STATE = 6,    /* no state yet (call mclg_init or mclg_set_state) */
    MCLG_ERR_SAMPLER = 7   /* a decision stayed open (sequential: after 4 refinement chunks,
                              p < 2^-70; slice: the 64-bit prefix hit a table value, p < 2^-59) */
} mclg_status;

/* flags */
#define MCLG_NO_STREAM 1u /* collide only, no streaming (the "without streaming" runs of Fig. decay) */
#define MCLG_STATS 2u     /* accumulate ensemble statistics after every step (Sec. V) */
#define MCLG_GALILEAN 4u  /* Galilean-invariant collision rate (end of Sec. IV.A): each node
                             collides with lambda(N, J) = q / 256, q the largest integer with
                             q / 256 <= lambda / sqrt(1 + 3 u^2), u = J / N, lambda the
                             handle's lambda_num / lambda_den; both samplers */
#define MCLG_HALO 8u      /* the handle's one replica is a block of a larger periodic lattice
                             (domain decomposition over ranks): its node x is the lattice's
                             node node_offset + x for every random number, and its two edges
                             exchange one value each per step with the neighbouring blocks
                             (mclg_halo_get / mclg_halo_put).  One replica, no MCLG_STATS, not
                             MCLG_MODE_PERSISTENT; with the SLICE sampler node_offset is a
                             multiple of 8 (eight consecutive nodes share the Philox block of
                             their uniforms' top bits). */

/* samplers: two exact ways to draw the C sub-collisions of a node, with
 * different uses of the random bits (each is bit-exact to its own oracle):
 *   SEQUENTIAL  the paper's order (Sec. III): C decisions one after another,
 *               each an exact uniform against the thresholds T1/D, T2/D.
 *   SLICE       all C at once: the rest count b moves to b + 2d with the exact
 *               C-step law on the node's (N, J) slice (the C-th power of the
 *               one-sub-collision matrix), inverted with one 64-bit uniform
 *               prefix Q = h 2^48 + (w1 mod 2^16) 2^32 + w0: h is bits
 *               [16 (x mod 2), 16 (x mod 2) + 16) of word (x/2) mod 4 of
 *               Philox block (x/8, r, t, 6 << 28), (w0, w1) words (0, 1) of
 *               block (x/2, r, t, 4 << 28) for even x, words (2, 3) for odd x;
 *               d = dmin + #{d' in [dmin, dmax) : Q > F[d']} with
 *               F[d'] = min(floor(CDF[d'] 2^64), 2^64 - 1) over the reachable
 *               offsets, Q == F[d'] reported as MCLG_ERR_SAMPLER.  Tables of F
 *               are built exactly (big integers) on the host for masses up to
 *               slice_n_max; heavier nodes take the SEQUENTIAL decisions.
 *               Requires C <= 10; runs in every mode (AUTO takes the
 *               per-step kernel, MCLG_MODE_PERSISTENT the persistent one). */
#define MCLG_SAMPLER_SEQUENTIAL 0u
#define MCLG_SAMPLER_SLICE 1u

/* execution modes; every mode gives bit-identical results */
#define MCLG_MODE_AUTO 0u       /* persistent batch where it pays, plain otherwise */
#define MCLG_MODE_PLAIN 1u      /* one plain-kernel launch per replica and step */
#define MCLG_MODE_PERSISTENT 2u /* replicas resident on chip for many steps, one launch */
#define MCLG_MODE_BATCHED 3u    /* one plain-kernel launch per step over all replicas */

typedef struct {
    uint32_t C;          /* sub-collisions per node and step (paper: C = 10, Sec. III.A, IV.A) */
    uint32_t lambda_num; /* lambda = lambda_num / lambda_den, 0 <= lambda <= 1 (Sec. III.A) */
    uint32_t lambda_den; /* 1 <= lambda_den <= 256 */
    uint32_t flags;      /* MCLG_NO_STREAM | MCLG_STATS */
    uint32_t mode;       /* MCLG_MODE_* */
    uint32_t first_replica; /* random-stream index of replica 0: replica r draws with index
                               first_replica + r, so a batch split over several handles or
                               GPUs, each given the index of its first replica, reproduces
                               the unsplit batch bit for bit */
    uint32_t sampler;       /* MCLG_SAMPLER_* */
    uint32_t slice_n_max;   /* SLICE: the tables cover node masses N <= slice_n_max (1 ..
                               1024; 0 = 256; larger values return MCLG_ERR_ARG); a node
                               with a larger mass takes the SEQUENTIAL sampler's C
                               decisions (the same bits that sampler gives it).  The bits
                               depend on slice_n_max like on the seed.  Tables take about
                               21 n^3 bytes of device memory and as much host memory
                               while they are built (0.37 GB at 256, 2.9 GB at 512,
                               23 GB at 1024, where the 32-bit record index still
                               holds); built once, at the first mclg_step, on the host
                               cores. */
    uint32_t kernel_variant; /* 0 = autotune the per-step kernel's launch variant at the first
                                mclg_step; v + 1 = use variant v (SEQUENTIAL: 0 <= v < 6, nodes
                                per thread and register bound; SLICE: 0 <= v < 20, 0-5 likewise,
                                6-9 the warp-specialised form with bulk-copy staging, 10-13 a
                                grid-stride form that loads each warp's next tile while it
                                draws the current one, 14-19 a temporally blocked form that
                                advances a window of nodes several steps per launch in
                                registers; 6-19 apply to single-replica launches; reported by
                                mclg_tuning).  With MCLG_STATS and the SLICE sampler, v + 1
                                = use the statistics form's configuration v (0 <= v < 4,
                                cfg[5] of mclg_tuning).
                                Every variant gives the same bits; this only fixes the launch
                                shape. */
    uint32_t node_offset;    /* MCLG_HALO: index of the block's first node in the whole lattice
                                (node_offset + L[0] <= 2^32); must be 0 without MCLG_HALO */
} mclg_params;

/* Defaults: C = 10, lambda = 1, flags 0, mode AUTO, first_replica 0,
 * SEQUENTIAL sampler (the paper's D1Q3 runs), slice_n_max 0, kernel_variant 0,
 * node_offset 0. */
void mclg_default_params(mclg_params *p);

/* Create a handle for `replicas` independent periodic lattices of lengths
 * L[0..replicas-1] (1 <= L[r] <= 2^31, sum L < 2^40), Philox seed `seed`.
 * p = NULL selects the defaults; cuda_stream = NULL uses the legacy default
 * stream.  Allocates the device state; no state is set yet.
 * MCLG_STATS requires all replicas to have the same length. */
mclg_status mclg_create(const uint32_t *L, uint32_t replicas, uint64_t seed, const mclg_params *p,
                        void *cuda_stream, mclg_handle *out);

/* n_i(x, 0) ~ Poisson(f_i^eq(rho(x), u(x))) with f^eq of Eq. D1Q3equil; rho, u
 * are host arrays of S doubles (rho >= 0, |u| <= 1).  Sets t = 0 and clears the
 * sticky error.  MCLG_ERR_OVERFLOW if a sampled count exceeds 65535. */
mclg_status mclg_init(mclg_handle h, const double *rho, const double *u);

/* Replace the state by the pre-collision field n(x, t) (layout above, host or
 * device pointer) at time t (t < 2^32).  Clears the sticky error. */
mclg_status mclg_set_state(mclg_handle h, const uint16_t *n, uint64_t t);

/* Copy the pre-collision field n(x, t) of the current time t into n (host or
 * device) and t into *t (may be NULL).  Synchronises the handle's stream. */
mclg_status mclg_get_state(mclg_handle h, uint16_t *n, uint64_t *t);

/* Advance n_steps time steps (stream + C sub-collisions per node, Sec. III).
 * Asynchronous: returns once the work is enqueued.  Returns the sticky error
 * of earlier work if one is known. */
mclg_status mclg_step(mclg_handle h, uint64_t n_steps);

/* Node moments of the current state: N(x) = sum_i n_i and J(x) = n_+1 - n_-1
 * (int32, S entries each, host or device, either may be NULL) and the exact
 * totals (sum N, sum J) into totals[2] (host, may be NULL).  Synchronises. */
mclg_status mclg_moments(mclg_handle h, int32_t *N, int32_t *J, int64_t *totals);

/* Statistics (MCLG_STATS): after every step the new field n(x, t+1) is added,
 * per replica-local position x and pooled over the replicas, as exact int64
 * sums s1[x][i] = sum n_i, s2[x][p] = sum n_i n_j for p over (i,j) =
 * 00 01 02 11 12 22, snb[x][3i+j] = sum n_i(x) n_j(x+1), and as FP32
 * compensated running means and (co)variances.  Eqs. poisson, Poisson2, corr. */
mclg_status mclg_stats_reset(mclg_handle h);

/* Read the statistics into host arrays (any may be NULL): s1[L*3], s2[L*6],
 * snb[L*9] int64; cov32[L*6] the FP32-path covariances of n_i, n_j at x;
 * cov64[L*6] the same from the exact int64 sums (FP64 only in this final
 * normalisation); *count = number of samples per position.  Synchronises. */
mclg_status mclg_stats_read(mclg_handle h, int64_t *s1, int64_t *s2, int64_t *snb, float *cov32,
                            double *cov64, uint64_t *count);

/* Wait for all enqueued work; returns the sticky device error, if any. */
mclg_status mclg_sync(mclg_handle h);

/* Current time step of the handle (host-side counter, no synchronisation). */
uint64_t mclg_time(mclg_handle h);

/* The autotuned launch configuration of the handle (zeros before the first
 * mclg_step): cfg[0] = 100 * nodes per thread of the per-step kernel (the
 * plain kernel, or the slice kernel with the slice sampler) + its variant
 * index (register bound), cfg[1] = threads per persistent CTA,
 * cfg[2] = nodes per persistent work unit, cfg[3] = number of persistent work
 * units, cfg[4] = persistent register-bound variant (0, 1, 2 = 1, 2, 3 CTAs of
 * 512 threads per SM), cfg[5] = the launch configuration of the slice
 * sampler's statistics form (MCLG_STATS with MCLG_SAMPLER_SLICE: 0-3 for 4 or
 * 8 replicas per warp, shared-memory counters updated by load-add-store or by
 * reductions), else 0. */
mclg_status mclg_tuning(mclg_handle h, uint32_t cfg[6]);

/* Domain decomposition of one periodic lattice (MCLG_HALO handles).  The
 * evolution equation (Sec. III) moves one population per link and step, so
 * across each cut one value leaves and one arrives per step.  A rank owning
 * global nodes [node_offset, node_offset + L) steps with
 *     mclg_step(h, 1); mclg_halo_get(h, out);
 *     send out[0] to the left neighbour and out[1] to the right neighbour,
 *     receive in[0] from the left neighbour (its out[1]) and in[1] from the
 *     right neighbour (its out[0]);
 *     mclg_halo_put(h, in);
 * and the blocks together reproduce the undecomposed lattice bit for bit (the
 * random numbers are keyed by the global node index).  One block whose out is
 * put back crossed over, in = (out[1], out[0]), is the periodic lattice.
 *
 * mclg_halo_get: out[0] = the post-collision v = -1 occupation of the block's
 * first node, out[1] = the post-collision v = +1 occupation of its last node,
 * from the last mclg_step (2 uint16, host or device; a host destination
 * synchronises).  MCLG_ERR_STATE before the first step.
 * mclg_halo_put: the arriving values in[0] (v = +1, into the first node) and
 * in[1] (v = -1, into the last node) complete the field n(x, t); required
 * after every mclg_step before the next mclg_step, mclg_get_state or
 * mclg_moments (MCLG_ERR_STATE otherwise).  mclg_init and mclg_set_state
 * take the edge values from the given field.  mclg_step advances one step per
 * call on such a handle (n_steps > 1 returns MCLG_ERR_ARG).  Both calls are
 * asynchronous for device pointers (ordered on the handle's stream). */
mclg_status mclg_halo_get(mclg_handle h, uint16_t *out);
mclg_status mclg_halo_put(mclg_handle h, const uint16_t *in);

/* Release every resource of the handle.  NULL-safe. */
void mclg_destroy(mclg_handle h);

/* ------------------------------------------------------------------------
 * D2Q9 (Sec. II.B, III.B, IV.B): R periodic Lx x Ly lattices of the nine
 * velocities v = (vx, vy), vx, vy in {-1, 0, 1}, numbered 0 = (0,0),
 * 1 = (1,0), 2 = (0,1), 3 = (-1,0), 4 = (0,-1), 5 = (1,1), 6 = (-1,1),
 * 7 = (-1,-1), 8 = (1,-1); state uint16 n[9][S], S = R Lx Ly, node
 * g = y Lx + x of replica r at r Lx Ly + g.
 *
 * Sampling contract (identical on every path):
 *   - Random words of node g of replica r at time t: word k of the node-step
 *     is word k % 4 of Philox4x32-10 block (g, r, t, 5 << 28 | k / 4), key as
 *     for D1Q3; at most 16 C + 64 words (MCLG_ERR_SAMPLER beyond).
 *   - Uniform integer below m: Lemire's multiply-shift x m = hi 2^32 + lo of a
 *     word x, rejecting lo < (2^32 - m) mod m with a new word; the value is hi.
 *   - A node with N < 2 is left alone.  Each of the C sub-collisions (Sec. III):
 *     q1, q2 uniform below N; q1 == q2: nothing; else s = the smallest
 *     velocity with q < n_0 + ... + n_s for each pick; the pick (s1, s2) has
 *     the outcome list of mclg2d_pair_outcomes (target pairs in increasing
 *     order, numerators over D = 128 lambda_den); then u uniform below D picks
 *     the first outcome whose cumulative numerator exceeds u, or nothing.
 *   - Collision classes (Sec. III.B, numbered as the rates in Eq. D2Q9MOmega):
 *     1 {0,5}<->{1,2}, 2 {0,0}<->{1,3}, 3 {0,0}<->{5,7}, 4 {1,3}<->{5,7},
 *     5 {1,3}<->{2,4}, 6 {5,7}<->{6,8}, 7 {0,1}<->{2,8}, 8 {1,6}<->{3,5},
 *     9 {1,1}<->{5,8}, each with its images under the rotations and
 *     reflections of the square.  From the pair with the smaller equilibrium
 *     pick weight (2 w_i w_j for different velocities, w_i^2 for equal ones) to
 *     the other: lambda_c; the other way: lambda_c times the ratio of the two
 *     weights (detailed balance; a power of 2 down to 1/128).
 *   - Streaming: n_i(x + v_i, t + 1) = post-collision n_i(x, t), periodic.
 *   - mclg2d_init: n_i ~ Poisson(f_i^eq(rho, u)) of Eq. D2Q9eqdist, by the
 *     D1Q3 initialisation contract with counters (g, r, p/2, 2 << 28 | i).
 * ------------------------------------------------------------------------ */
typedef struct mclg2d_ctx *mclg2d_handle;

typedef struct {
    uint32_t C;               /* sub-collisions per node and step (<= 2^24) */
    uint32_t lambda_num[9];   /* class rates lambda_c = lambda_num[c-1] / lambda_den */
    uint32_t lambda_den;      /* 1 .. 65536; every pick's outcomes must add up to <= 1 */
    uint32_t flags;           /* MCLG_NO_STREAM */
    uint32_t first_replica;   /* random-stream index of replica 0 */
} mclg2d_params;

/* Defaults: C = 10 and the rates of the paper's D2Q9 runs (Sec. IV.B):
 * lambda_1 = 15/128, lambda_2..7 = 1/4, lambda_8 = 1/8, lambda_9 = 18/144. */
void mclg2d_default_params(mclg2d_params *p);

/* R replicas of an Lx x Ly periodic lattice (Lx Ly < 2^32); p = NULL: defaults.
 * MCLG_ERR_ARG for invalid sizes or rates (including outcome probabilities of a
 * pick that add up to more than 1). */
mclg_status mclg2d_create(uint32_t Lx, uint32_t Ly, uint32_t replicas, uint64_t seed,
                          const mclg2d_params *p, void *cuda_stream, mclg2d_handle *out);

/* n_i ~ Poisson(f_i^eq(rho, ux, uy)) (Eq. D2Q9eqdist, Eq. poisson); host arrays
 * of S doubles (rho >= 0, |u| <= 1).  Sets t = 0. */
mclg_status mclg2d_init(mclg2d_handle h, const double *rho, const double *ux, const double *uy);

/* Replace / read the state n[9][S] (host or device) at time t (< 2^32); reading
 * synchronises and returns the sticky device error, if any. */
mclg_status mclg2d_set_state(mclg2d_handle h, const uint16_t *n, uint64_t t);
mclg_status mclg2d_get_state(mclg2d_handle h, uint16_t *n, uint64_t *t);

/* Advance n_steps time steps (asynchronous). */
mclg_status mclg2d_step(mclg2d_handle h, uint64_t n_steps);

/* Density and momentum per node (device int32 arrays of S entries, or NULL)
 * and the exact totals (sum rho, sum j_x, sum j_y) into totals[3] (host, or
 * NULL).  Synchronises. */
mclg_status mclg2d_moments(mclg2d_handle h, int32_t *rho, int32_t *jx, int32_t *jy,
                           int64_t *totals);

mclg_status mclg2d_sync(mclg2d_handle h);
uint64_t mclg2d_time(mclg2d_handle h);
void mclg2d_destroy(mclg2d_handle h);

/* The outcome list of a pick of velocities (s1, s2) under the rates of p (host
 * computation, no GPU): *count outcomes, target pairs targets[2k], targets[2k+1]
 * (increasing), numerators nums[k] over 128 lambda_den (arrays of 4 entries,
 * targets of 8; either may be NULL).  For checking the table independently. */
mclg_status mclg2d_pair_outcomes(uint32_t s1, uint32_t s2, const mclg2d_params *p,
                                 uint32_t *count, uint32_t *targets, uint64_t *nums);

/* Static description of a status code. */
const char *mclg_status_str(mclg_status s);

/* Allocation-free variant of the totals and node moments of mclg_moments,
 * for callers that cannot allocate device memory: code whose GPU memory is
 * owned by another pool (a framework's caching allocator may hold nearly all
 * of it) and loops that cannot accept the device-wide synchronisation that
 * cudaMalloc/cudaFree may imply.  The paper has no counterpart; this is a
 * library convenience.
 *   n       device array on the current device, the canonical field n[3][S]
 *           (as mclg_get_state writes it)
 *   S       nodes, 1 <= S <= 2^26 (67,108,864); larger S returns MCLG_ERR_ARG
 *   N, J    int32 arrays of S entries on the current device, or NULL
 *   totals  (sum N, sum J) as two int64, host or on the current device, or
 *           NULL; a host destination synchronises cuda_stream before returning
 * A buffer on another device (or a host n, N or J) returns MCLG_ERR_ARG before
 * any launch.  A CUDA error already pending on the calling thread is left in
 * place and reported as MCLG_ERR_CUDA, with nothing launched.
 * Allocates nothing: its only scratch is a fixed 512 KiB device array that
 * every GPU loading this library holds until the process exits.  The first
 * call on a device looks up that array's device address (with the device
 * current); make that first call before any stream capture.  All calls share
 * the one array, so calls that overlap on the GPU (other streams, other host
 * threads on the same device) race: order them on one stream. */
mclg_status mclg_moments_noalloc(const uint16_t *n, uint64_t S, int32_t *N, int32_t *J,
                                 int64_t *totals, void *cuda_stream);

/* The slice sampler's table row for the state (N, J, b) (host computation, no
 * GPU): F[k] = min(floor(CDF[dmin + k] 2^64), 2^64 - 1) for k < dmax - dmin,
 * the exact cumulative C-step law of the rest count (F holds 2C entries);
 * *dmin, *dmax the reachable offsets.  record (8 uint16, or NULL) receives
 * the state's record as the device reads it: lane j = F[c0 - 4 + j] >> 49
 * with c0 = -dmin (0 where c0 - 4 + j < 0, 0x7FFF where it is >= dmax -
 * dmin).  If q = Q >> 49 equals no lane and lies above lane 0 and below lane
 * 7, the draw is d = #{lanes below q} - 4; otherwise the kernel compares Q
 * with the u64 values.
 * For checking the tables against an independent computation.  MCLG_ERR_ARG
 * for C > 10, an invalid state, or D = 8 N^2 lambda_den >= 2^44 (the exact
 * numerators over D^C would not fit the builder's 512-bit integers; with
 * lambda_den = 1 every N <= 2^20 is accepted, with 256 every N <= 92681). */
mclg_status mclg_slice_row(uint32_t N, int32_t J, uint32_t b, uint32_t C, uint32_t lambda_num,
                           uint32_t lambda_den, uint64_t *F, int32_t *dmin, int32_t *dmax,
                           uint16_t *record);

/* Philox4x32-10 of the library's device generator on n counters: ctr and out
 * are device arrays of n uint4 (x, y, z, w); key = (seed lo, seed hi).  For
 * checking the generator against an independent implementation. */
mclg_status mclg_philox(const uint32_t *ctr, uint64_t n, uint64_t seed, uint32_t *out,
                        void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MCLG_H */
