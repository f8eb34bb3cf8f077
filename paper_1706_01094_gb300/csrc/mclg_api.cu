// Host side of the C ABI declared in include/mclg.h: handle, layout, modes,
// autotuner, host Poisson initialisation and the conversions between the ABI
// field and the device form.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "../../include/mclg.h"
#include "mclg_device.cuh"
#include "mclg_internal.h"

using namespace mclg;

struct mclg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr;  // second stream: plain steps of large replicas beside the persistent kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    mclg_params prm{};
    uint64_t seed = 0;
    uint32_t R = 0;
    std::vector<uint32_t> L;          // ABI order
    std::vector<uint64_t> abi_off;    // ABI order
    uint64_t S = 0;                   // sum of L
    // internal order
    std::vector<uint32_t> order;      // internal k -> replica id
    std::vector<uint64_t> rep_off;    // internal k -> node offset
    std::vector<uint32_t> rep_L;      // internal k -> length
    uint32_t n_small = 0;             // internal replicas [0, n_small) fit a persistent CTA
    uint64_t small_chunks = 0;        // chunks of the small replicas (they come first)
    Layout lay;
    uint16_t *d_B[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t *d_err = nullptr;
    unsigned long long *d_totals = nullptr;
    uint16_t *d_stage = nullptr;      // ABI-layout staging for host transfers
    int32_t *d_stageNJ = nullptr;
    uint64_t t = 0;
    bool has_state = false;
    uint32_t sticky = 0;              // device error bits seen so far
    // persistent configuration (autotuned)
    bool tuned = false;
    uint32_t p_threads = 256, p_cap = 0, p_variant = 1;
    bool plain_tuned = false;
    uint32_t plain_variant = 0;       // plain-kernel variant (autotuned)
    std::vector<Unit> units;
    Unit *d_units = nullptr;
    uint32_t *d_unit_counter = nullptr;  // work queue of the persistent kernel
    // statistics
    StatsBuffers st{};
    unsigned long long *d_stat_partials = nullptr;  // the step's batch sums (cleared by the merge)
    // CUDA graphs of kGraphSteps per-step launch sequences, one per starting
    // buffer parity, for the plain and batched modes and for the long replicas
    uint32_t *d_t = nullptr;          // time step read by graph-replayed launches
    cudaStream_t cap = nullptr;       // private stream for graph capture
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    uint32_t graph_kb = 0, graph_ke = 0;  // replica range the graphs step
    // slice sampler: exact cumulative C-step laws for masses up to slice.n_max
    SliceTables slice{};
    uint32_t *d_rowstart = nullptr;
    unsigned long long *d_heavy_pos = nullptr;  // slice sampler: nodes beyond the tables
    uint32_t *d_heavy_ctl = nullptr;
    uint4 *d_slice_record = nullptr;
    unsigned long long *d_slice_secondary = nullptr;
    uint64_t stats_count = 0;
    // a block of a larger lattice (MCLG_HALO): the two arriving edge values
    bool halo = false;
    bool halo_ready = false;          // the arriving values of the current time are in d_halo
    bool stepped = false;             // a step has run since the state was set
    uint16_t *d_halo = nullptr;       // [2]: v = +1 into node 0, v = -1 into node L - 1
    uint32_t *d_stats_from = nullptr; // statistics form of the slice step: first time step
                                      // whose input field is a sample
    uint32_t stats_config = 0;        // statistics form: autotuned launch configuration
};

namespace {

constexpr uint64_t kMaxT = uint64_t(1) << 32;
constexpr uint32_t kGraphSteps = 32;  // steps per captured graph (even: parity preserved)

mclg_status cuda_fail(cudaError_t e) { return e == cudaSuccess ? MCLG_OK : MCLG_ERR_CUDA; }

#define MCLG_CK(expr)                                   \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return cuda_fail(_e);    \
    } while (0)

uint64_t pad8(uint64_t v) { return (v + 7u) & ~uint64_t(7); }

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mclg_status status_from_bits(uint32_t bits)
{
    if (bits & kErrOverflow) return MCLG_ERR_OVERFLOW;
    if (bits & kErrSampler) return MCLG_ERR_SAMPLER;
    if (bits & kErrTimeout) return MCLG_ERR_TIMEOUT;
    return MCLG_OK;
}

// Read the device error word after the stream is idle, fold it into the sticky bits.
mclg_status collect_errors(mclg_ctx *h)
{
    MCLG_CK(cudaStreamSynchronize(h->stream));
    uint32_t bits = 0;
    MCLG_CK(cudaMemcpy(&bits, h->d_err, sizeof(bits), cudaMemcpyDeviceToHost));
    h->sticky |= bits;
    return status_from_bits(h->sticky);
}

std::vector<Unit> build_units(const mclg_ctx *h, uint32_t cap)
{
    std::vector<Unit> out;
    uint32_t k = 0;
    while (k < h->n_small) {
        Unit u{};
        u.node_begin = h->rep_off[k];
        u.rep_begin = k;
        u.rep_end = k;
        uint64_t nodes = 0;
        while (k < h->n_small && u.rep_end - u.rep_begin < kMaxUnitReplicas) {
            const uint64_t need = pad8(h->rep_L[k]);
            if (nodes + need > cap && nodes > 0) break;
            nodes += need;
            ++k;
            u.rep_end = k;
        }
        u.nodes = uint32_t(nodes);
        out.push_back(u);
    }
    // largest units first: the CTAs pull them from a queue, so the tail is short
    std::stable_sort(out.begin(), out.end(),
                     [](const Unit &x, const Unit &y) { return x.nodes > y.nodes; });
    return out;
}

PlainArgs plain_args(const mclg_ctx *h, const uint16_t *in, uint16_t *out, uint64_t t)
{
    PlainArgs a{};
    a.in = in;
    a.out = out;
    a.P = h->lay.P;
    a.chunk_rep = h->lay.d_chunk_rep;
    a.rep_off = h->lay.d_rep_off;
    a.rep_L = h->lay.d_rep_L;
    a.rep_id = h->lay.d_rep_id;
    a.t = uint32_t(t);
    a.C = h->prm.C;
    a.lam_n = h->prm.lambda_num;
    a.lam_d = h->prm.lambda_den;
    a.k0 = uint32_t(h->seed);
    a.k1 = uint32_t(h->seed >> 32);
    a.err = h->d_err;
    a.variant = h->plain_variant;
    a.stream = (h->prm.flags & MCLG_NO_STREAM) ? 0u : 1u;
    a.galilean = (h->prm.flags & MCLG_GALILEAN) ? 1u : 0u;
    a.r0 = h->prm.first_replica;
    a.t_dev = nullptr;
    a.halo_in = h->halo ? h->d_halo : nullptr;
    a.x_base = h->prm.node_offset;
    a.rk = make_round_keys(h->seed);
    return a;
}

bool streaming(const mclg_ctx *h) { return !(h->prm.flags & MCLG_NO_STREAM); }

// Steps that one launch of the plain path over [kb, ke) covers: the
// temporally blocked slice variants advance a handle's single replica several
// steps per launch; everything else one (the persistent mode's long replicas
// must end in the buffer that the step count's parity gives).
uint32_t launch_span(const mclg_ctx *h, uint32_t kb, uint32_t ke)
{
    if (h->prm.sampler != MCLG_SAMPLER_SLICE || kb != 0u || ke != 1u || h->R != 1u || h->halo ||
        (h->prm.flags & MCLG_STATS) || h->plain_variant < kSliceTbFirst)
        return 1u;
    return slice_tb_steps(h->plain_variant - kSliceTbFirst);
}

// `steps` steps (1, or up to launch_span) over internal replicas
// [k_begin, k_end) with a single plain launch.
cudaError_t plain_batch_step(mclg_ctx *h, const uint16_t *in, uint16_t *out, uint64_t t,
                             uint32_t k_begin, uint32_t k_end, cudaStream_t s,
                             const uint32_t *t_dev = nullptr, uint32_t steps = 1)
{
    if (k_begin >= k_end) return cudaSuccess;
    PlainArgs a = plain_args(h, in, out, t);
    a.t_dev = t_dev;
    a.g_begin = h->rep_off[k_begin] / 8u;
    a.g_end = (h->rep_off[k_end - 1] + pad8(h->rep_L[k_end - 1])) / 8u;
    const bool one = k_end - k_begin == 1;
    if (one) {
        a.one_off = h->rep_off[k_begin];
        a.one_L = h->rep_L[k_begin];
        a.one_rid = h->order[k_begin];
    }
    if (steps > 1u) {
        if (steps > launch_span(h, k_begin, k_end)) return cudaErrorInvalidValue;
        return launch_slice_tb(a, h->slice, steps, h->plain_variant - kSliceTbFirst, s);
    }
    if (h->prm.sampler == MCLG_SAMPLER_SLICE) return launch_slice(a, one, h->slice, s);
    return launch_plain(a, one, s);
}

// One step with one plain launch per replica (the per-replica baseline).
cudaError_t plain_per_replica_step(mclg_ctx *h, const uint16_t *in, uint16_t *out, uint64_t t,
                                   cudaStream_t s)
{
    for (uint32_t k = 0; k < h->R; ++k) {
        cudaError_t e = plain_batch_step(h, in, out, t, k, k + 1, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

PersistentArgs persistent_args(const mclg_ctx *h, const uint16_t *in, uint16_t *out, uint64_t t0,
                               uint32_t n_steps, const Unit *d_units, uint32_t cap)
{
    PersistentArgs a{};
    a.in = in;
    a.out = out;
    a.P = h->lay.P;
    a.units = d_units;
    a.rep_off = h->lay.d_rep_off;
    a.rep_L = h->lay.d_rep_L;
    a.rep_id = h->lay.d_rep_id;
    a.cap = cap;
    a.t0 = uint32_t(t0);
    a.n_steps = n_steps;
    a.C = h->prm.C;
    a.lam_n = h->prm.lambda_num;
    a.lam_d = h->prm.lambda_den;
    a.k0 = uint32_t(h->seed);
    a.k1 = uint32_t(h->seed >> 32);
    a.err = h->d_err;
    a.stream = (h->prm.flags & MCLG_NO_STREAM) ? 0u : 1u;
    a.galilean = (h->prm.flags & MCLG_GALILEAN) ? 1u : 0u;
    a.r0 = h->prm.first_replica;
    a.rk = make_round_keys(h->seed);
    a.unit_counter = h->d_unit_counter;
    a.variant = h->p_variant;
    a.slice = h->prm.sampler == MCLG_SAMPLER_SLICE ? 1u : 0u;
    a.tab = h->slice;
    return a;
}

// Autotuner: time a few steps of each (threads, capacity) candidate on a
// scratch output buffer (results are identical for every candidate; only the
// speed differs) and keep the fastest.
mclg_status autotune(mclg_ctx *h)
{
    h->tuned = true;
    if (h->n_small == 0) return MCLG_OK;
    uint32_t max_small = 0;
    for (uint32_t k = 0; k < h->n_small; ++k) max_small = std::max<uint32_t>(max_small, uint32_t(pad8(h->rep_L[k])));
    // unit capacities from the longest small replica up to the limit, and CTA
    // sizes up to one thread per node pair of a unit
    std::vector<uint32_t> caps;
    for (uint32_t c = 64; c <= kMaxUnitNodes; c *= 2)
        if (c >= max_small) caps.push_back(c);
    const uint32_t threads_all[] = {32, 64, 128, 256, 512};
    uint16_t *scratch = nullptr;
    MCLG_CK(cudaMalloc(&scratch, 3 * h->lay.P * sizeof(uint16_t)));
    cudaEvent_t e0, e1;
    MCLG_CK(cudaEventCreate(&e0));
    MCLG_CK(cudaEventCreate(&e1));
    float best = 1e30f;
    uint32_t best_threads = 256, best_cap = caps.empty() ? kMaxUnitNodes : caps.back();
    uint32_t best_variant = 1;
    const uint32_t probe_steps = 4;
    for (uint32_t cap : caps) {
        std::vector<Unit> units = build_units(h, cap);
        Unit *d_units = nullptr;
        MCLG_CK(cudaMalloc(&d_units, units.size() * sizeof(Unit)));
        MCLG_CK(cudaMemcpyAsync(d_units, units.data(), units.size() * sizeof(Unit),
                                cudaMemcpyHostToDevice, h->stream));
        for (uint32_t th : threads_all)
        for (uint32_t pv = 0; pv < kPersistentVariants; ++pv) {
            if (th > std::max<uint32_t>(32u, cap / 2u)) continue;
            PersistentArgs a = persistent_args(h, h->d_B[h->cur], scratch, h->t, probe_steps,
                                               d_units, cap);
            a.variant = pv;
            // warm-up, then timed
            MCLG_CK(launch_persistent(a, uint32_t(units.size()), th, h->stream));
            MCLG_CK(cudaEventRecord(e0, h->stream));
            MCLG_CK(launch_persistent(a, uint32_t(units.size()), th, h->stream));
            MCLG_CK(cudaEventRecord(e1, h->stream));
            MCLG_CK(cudaEventSynchronize(e1));
            float ms = 0;
            MCLG_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                best_threads = th;
                best_cap = cap;
                best_variant = pv;
            }
        }
        MCLG_CK(cudaStreamSynchronize(h->stream));
        cudaFree(d_units);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    // the probes may have flagged errors of the current state; they are the
    // same errors the real steps will flag, so they are not folded in here
    MCLG_CK(cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream));
    h->p_threads = best_threads;
    h->p_cap = best_cap;
    h->p_variant = best_variant;
    h->units = build_units(h, best_cap);
    if (h->d_units) cudaFree(h->d_units);
    MCLG_CK(cudaMalloc(&h->d_units, h->units.size() * sizeof(Unit)));
    MCLG_CK(cudaMemcpyAsync(h->d_units, h->units.data(), h->units.size() * sizeof(Unit),
                            cudaMemcpyHostToDevice, h->stream));
    return MCLG_OK;
}

bool fused_stats(const mclg_ctx *h);
cudaError_t plain_step_seq(mclg_ctx *h, int c, uint64_t t, uint32_t kb, uint32_t ke,
                           cudaStream_t s, const uint32_t *t_dev, uint32_t steps = 1);

// Plain-kernel autotuner: time each vector width on the real input, writing
// into the buffer the next step overwrites anyway (results do not depend on
// the width), and keep the fastest.
mclg_status autotune_plain(mclg_ctx *h, uint32_t mode, uint32_t k_begin, uint32_t k_end)
{
    h->plain_tuned = true;
    cudaEvent_t e0, e1;
    MCLG_CK(cudaEventCreate(&e0));
    MCLG_CK(cudaEventCreate(&e1));
    if (fused_stats(h)) {
        // the statistics form's configurations, timed on steps that count their
        // input field (the configurations differ only in how the sums are
        // gathered) into scratch sums, so the batch's own stay untouched; the
        // buffer written is the one the next step overwrites anyway
        const size_t pb = stats_partials_bytes(h->L[0], h->R);
        unsigned long long *scratch = nullptr;
        MCLG_CK(cudaMalloc(&scratch, pb + 3 * sizeof(unsigned long long)));
        MCLG_CK(cudaMemsetAsync(scratch, 0, pb + 3 * sizeof(unsigned long long), h->stream));
        unsigned long long *const own_partials = h->d_stat_partials, *const own_count = h->st.count;
        h->d_stat_partials = scratch;
        h->st.count = scratch + pb / sizeof(unsigned long long);
        auto probe = [&]() -> mclg_status {
            MCLG_CK(launch_set_time(h->d_stats_from, 0u, h->stream));
            float best = 1e30f;
            for (uint32_t v = 0; v < kStatsConfigs; ++v) {
                h->stats_config = v;
                float ms = 1e30f;
                for (int rep = 0; rep < 8; ++rep) {
                    MCLG_CK(cudaEventRecord(e0, h->stream));
                    MCLG_CK(plain_step_seq(h, h->cur, h->t, 0, h->R, h->stream, nullptr));
                    MCLG_CK(cudaEventRecord(e1, h->stream));
                    MCLG_CK(cudaEventSynchronize(e1));
                    float one = 0;
                    MCLG_CK(cudaEventElapsedTime(&one, e0, e1));
                    if (rep > 0) ms = std::min(ms, one);
                }
                if (ms < best) {
                    best = ms;
                    h->plain_variant = v;  // reported by mclg_tuning
                }
            }
            MCLG_CK(cudaStreamSynchronize(h->stream));
            return MCLG_OK;
        };
        const mclg_status st = probe();
        h->d_stat_partials = own_partials;
        h->st.count = own_count;
        cudaFree(scratch);
        if (st != MCLG_OK) return st;
        h->stats_config = h->plain_variant;
        h->plain_variant = 0;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return MCLG_OK;
    }
    float best = 1e30f;
    uint32_t best_variant = h->plain_variant;
    const uint16_t *in = h->d_B[h->cur];
    uint16_t *outb = h->d_B[h->cur ^ 1];
    const uint32_t variants =
        h->prm.sampler == MCLG_SAMPLER_SLICE ? kSliceVariants : kPlainVariants;
    for (uint32_t v = 0; v < variants; ++v) {
        h->plain_variant = v;
        // per step: a blocked variant is timed over the steps one launch covers
        const bool per_replica = mode == MCLG_MODE_PLAIN && h->R > 1u;
        const uint32_t span = per_replica ? 1u : launch_span(h, k_begin, k_end);
        float ms = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {  // first launch warms up, keep the best of 3
            MCLG_CK(cudaEventRecord(e0, h->stream));
            if (per_replica)
                MCLG_CK(plain_per_replica_step(h, in, outb, h->t, h->stream));
            else
                MCLG_CK(plain_batch_step(h, in, outb, h->t, k_begin, k_end, h->stream, nullptr,
                                         span));
            MCLG_CK(cudaEventRecord(e1, h->stream));
            MCLG_CK(cudaEventSynchronize(e1));
            float one = 0;
            MCLG_CK(cudaEventElapsedTime(&one, e0, e1));
            if (rep > 0) ms = std::min(ms, one / float(span));
        }
        if (ms < best) {
            best = ms;
            best_variant = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->plain_variant = best_variant;
    return MCLG_OK;
}

// Statistics with the slice sampler run in the step kernel's statistics form:
// the kernel of step t adds its input field n(t) (from t = *d_stats_from on).
bool fused_stats(const mclg_ctx *h)
{
    return (h->prm.flags & MCLG_STATS) && h->prm.sampler == MCLG_SAMPLER_SLICE;
}

// The statistics partial pass over the field in buffer c (adds one sample of
// every replica to the batch).
cudaError_t stats_partial(mclg_ctx *h, int c, cudaStream_t s)
{
    return launch_stats_partial(h->d_B[c], h->lay.P, h->L[0], h->R, pad8(h->L[0]),
                                streaming(h) ? 1 : 0, h->d_stat_partials, h->st.count + 2, s);
}

// One launch of the plain path over internal replicas [kb, ke) from buffer c
// to buffer c ^ 1 (`steps` steps, at most launch_span), plus the statistics
// when they are on: of the new field (partial pass after the step), or, in
// the slice sampler's statistics form, of the input field inside the step
// kernel.  With t_dev set the launches read their time step from the device
// (t is then an offset).
cudaError_t plain_step_seq(mclg_ctx *h, int c, uint64_t t, uint32_t kb, uint32_t ke,
                           cudaStream_t s, const uint32_t *t_dev, uint32_t steps)
{
    if (fused_stats(h)) {
        PlainArgs a = plain_args(h, h->d_B[c], h->d_B[c ^ 1], t);
        a.t_dev = t_dev;
        a.g_begin = 0;
        a.g_end = h->lay.P / 8u;
        a.one_L = h->L[0];
        StatsArgs sa{h->R, pad8(h->L[0]), h->d_stats_from, h->d_stat_partials, h->st.count + 2,
                     h->stats_config};
        return launch_slice_stats(a, h->slice, sa, s);
    }
    cudaError_t e = plain_batch_step(h, h->d_B[c], h->d_B[c ^ 1], t, kb, ke, s, t_dev, steps);
    if (e != cudaSuccess) return e;
    if (h->prm.flags & MCLG_STATS) e = stats_partial(h, c ^ 1, s);
    return e;
}

// Fold the batch of samples accumulated so far into the running moments.
cudaError_t stats_merge(mclg_ctx *h, cudaStream_t s)
{
    if (!(h->prm.flags & MCLG_STATS)) return cudaSuccess;
    return launch_stats_merge(h->d_stat_partials, h->L[0], h->st, s);
}

void drop_graphs(mclg_ctx *h)
{
    for (auto &g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Capture kGraphSteps steps starting from buffer c into h->graph[c].
mclg_status capture_graph(mclg_ctx *h, int c, uint32_t kb, uint32_t ke)
{
    if (h->graph_kb != kb || h->graph_ke != ke) {
        drop_graphs(h);
        h->graph_kb = kb;
        h->graph_ke = ke;
    }
    if (h->graph[c]) return MCLG_OK;
    cudaGraph_t g = nullptr;
    MCLG_CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    int cc = c;
    // an even number of launches (each flips the buffer): spans divide kGraphSteps / 2
    const uint32_t span = launch_span(h, kb, ke);
    for (uint32_t j = 0; j < kGraphSteps && e == cudaSuccess; j += span) {
        e = plain_step_seq(h, cc, j, kb, ke, h->cap, h->d_t, span);
        cc ^= 1;
    }
    if (e == cudaSuccess) e = stats_merge(h, h->cap);  // one merge per graph
    if (e == cudaSuccess) e = launch_advance_time(h->d_t, kGraphSteps, h->cap);
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return MCLG_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&h->graph[c], g, 0);
    cudaGraphDestroy(g);
    return cuda_fail(e);
}

// n_steps steps of the plain path over [kb, ke) on stream s: whole groups of
// kGraphSteps replay a captured graph, the rest launch directly.  Returns the
// buffer that holds the result.
mclg_status plain_steps(mclg_ctx *h, int c, uint64_t t, uint64_t n_steps, uint32_t kb, uint32_t ke,
                        cudaStream_t s, int *c_out)
{
    uint64_t done = 0;
    const uint64_t groups = n_steps / kGraphSteps;
    // the statistics form counts the input fields from the second step of the
    // call on: the first one was counted at the end of the previous call (or is
    // the field at a reset)
    if (fused_stats(h)) MCLG_CK(launch_set_time(h->d_stats_from, uint32_t(t + 1), s));
    if (groups > 0) {
        mclg_status st = capture_graph(h, c, kb, ke);
        if (st != MCLG_OK) return st;
        MCLG_CK(launch_set_time(h->d_t, uint32_t(t), s));
        for (uint64_t g = 0; g < groups; ++g) MCLG_CK(cudaGraphLaunch(h->graph[c], s));
        done = groups * kGraphSteps;  // even: the parity of c is unchanged
    }
    const uint32_t span = launch_span(h, kb, ke);
    while (done < n_steps) {
        const uint32_t k = uint32_t(std::min<uint64_t>(span, n_steps - done));
        MCLG_CK(plain_step_seq(h, c, t + done, kb, ke, s, nullptr, k));
        c ^= 1;
        done += k;
    }
    if (fused_stats(h)) MCLG_CK(stats_partial(h, c, s));  // the call's last field
    MCLG_CK(stats_merge(h, s));  // every call leaves the statistics merged
    *c_out = c;
    return MCLG_OK;
}

void free_slice_tables(mclg_ctx *h)
{
    cudaFree(h->d_rowstart);
    cudaFree(h->d_heavy_pos);
    cudaFree(h->d_heavy_ctl);
    h->d_heavy_pos = nullptr;
    h->d_heavy_ctl = nullptr;
    cudaFree(h->d_slice_record);
    cudaFree(h->d_slice_secondary);
    h->d_rowstart = nullptr;
    h->d_slice_record = nullptr;
    h->d_slice_secondary = nullptr;
    h->slice = SliceTables{};
}

// Build the slice tables (exact big-integer laws, host cores) for masses up
// to the handle's n_max, once, and the list of heavier nodes, which take the
// sequential draws in a second pass of each step.
mclg_status ensure_slice_tables(mclg_ctx *h)
{
    if (h->slice.record) return MCLG_OK;
    const uint32_t n_max = h->prm.slice_n_max ? h->prm.slice_n_max : kSliceDefaultN;
    std::vector<uint32_t> rowstart;
    std::vector<uint16_t> record;
    std::vector<uint64_t> secondary;
    try {
        build_slice_tables(n_max, h->prm.C, h->prm.lambda_num, h->prm.lambda_den,
                           (h->prm.flags & MCLG_GALILEAN) != 0u, rowstart, record,
                           secondary);
    } catch (...) {
        return MCLG_ERR_NOMEM;
    }
    MCLG_CK(cudaStreamSynchronize(h->stream));
    free_slice_tables(h);
    if (cudaMalloc(&h->d_rowstart, rowstart.size() * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&h->d_slice_record, record.size() * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc(&h->d_slice_secondary, secondary.size() * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&h->d_heavy_pos, kHeavyCap * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&h->d_heavy_ctl, 3 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        free_slice_tables(h);
        return MCLG_ERR_NOMEM;
    }
    MCLG_CK(cudaMemcpy(h->d_rowstart, rowstart.data(), rowstart.size() * sizeof(uint32_t),
                       cudaMemcpyHostToDevice));
    MCLG_CK(cudaMemcpy(h->d_slice_record, record.data(), record.size() * sizeof(uint16_t),
                       cudaMemcpyHostToDevice));
    MCLG_CK(cudaMemcpy(h->d_slice_secondary, secondary.data(), secondary.size() * sizeof(uint64_t),
                       cudaMemcpyHostToDevice));
    h->slice.n_max = n_max;
    h->slice.rec_hb = n_max / 2 + 1;
    h->slice.rowstart = h->d_rowstart;
    h->slice.record = h->d_slice_record;
    h->slice.secondary = h->d_slice_secondary;
    MCLG_CK(cudaMemset(h->d_heavy_ctl, 0, 3 * sizeof(uint32_t)));
    h->slice.heavy_pos = h->d_heavy_pos;
    h->slice.heavy_ctl = h->d_heavy_ctl;
    h->slice.heavy_cap = kHeavyCap;
    drop_graphs(h);  // captured launches hold the old table pointers
    return MCLG_OK;
}

uint32_t effective_mode(const mclg_ctx *h)
{
    if (h->halo) return MCLG_MODE_PLAIN;       // one block, edges exchanged every step
    if (h->prm.flags & MCLG_STATS) return 3u;  // batched plain: state in HBM after each step
    if (h->prm.sampler == MCLG_SAMPLER_SLICE) {
        // AUTO: the per-step slice kernel (the persistent form only on request)
        if (h->prm.mode == MCLG_MODE_PLAIN || h->R == 1) return MCLG_MODE_PLAIN;
        if (h->prm.mode == MCLG_MODE_PERSISTENT && h->n_small > 0) return MCLG_MODE_PERSISTENT;
        return 3u;
    }
    if (h->prm.mode == MCLG_MODE_PLAIN) return MCLG_MODE_PLAIN;
    if (h->prm.mode == MCLG_MODE_PERSISTENT) return MCLG_MODE_PERSISTENT;
    if (h->prm.mode == 3u) return 3u;
    // AUTO: a single replica or only large replicas -> plain; else persistent
    if (h->n_small == 0) return h->R == 1 ? MCLG_MODE_PLAIN : 3u;
    return MCLG_MODE_PERSISTENT;
}

// ----------------------------------------------------------- host init ---
// Entropic equilibrium of Eq. D1Q3equil and Poisson sampling by inversion,
// evaluated in the operation order fixed by the ABI's initialisation
// contract (FP64, no contraction).
void equilibrium(double rho, double u, double f[3])
{
    static const double w[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    const double s = std::sqrt(1.0 + 3.0 * u * u) - 1.0;
    for (int i = 0; i < 3; ++i) {
        const double v = double(i - 1);
        f[i] = rho * w[i] * (1.0 + 3.0 * v * u + (3.0 * v * v - 1.0) * s);
    }
}

uint32_t poisson_by_inversion(double mu, double U)
{
    double pk = std::exp(-mu);
    double cdf = pk;
    uint32_t k = 0;
    while (U >= cdf && k < 200u) {
        ++k;
        pk = pk * (mu / double(k));
        cdf = cdf + pk;
    }
    return k;
}

int init_range(const mclg_ctx *h, const double *rho, const double *u, uint16_t *n, uint32_t r,
               uint32_t x_begin, uint32_t x_end)
{
    const uint32_t k0 = uint32_t(h->seed), k1 = uint32_t(h->seed >> 32);
    int err = 0;
    const uint64_t a0 = h->abi_off[r];
    for (uint32_t x = x_begin; x < x_end; ++x) {
        const double rh = rho[a0 + x], uu = u[a0 + x];
        if (!(rh >= 0.0) || !std::isfinite(rh) || !(std::fabs(uu) <= 1.0)) return 8;
        double f[3];
        equilibrium(rh, uu, f);
        for (uint32_t i = 0; i < 3; ++i) {
            const double mu = f[i] > 0.0 ? f[i] : 0.0;
            uint32_t parts = uint32_t(std::ceil(mu / 32.0));
            if (parts < 1) parts = 1;
            const double part_mu = mu / double(parts);
            uint64_t total = 0;
            for (uint32_t q = 0; q < parts; ++q) {
                uint32_t w0 = h->prm.node_offset + x, w1 = r + h->prm.first_replica, w2 = q / 2,
                         w3 = (kPurposeInit << 28) | i;
                philox4x32_10(w0, w1, w2, w3, k0, k1);
                const uint32_t lo = (q & 1u) ? w2 : w0, hi = (q & 1u) ? w3 : w1;
                const uint64_t m = ((uint64_t(hi) << 32) | lo) >> 11;
                const double U = double(m) * (1.0 / 9007199254740992.0);
                total += poisson_by_inversion(part_mu, U);
            }
            if (total > 65535u) {
                err |= 1;
                total = 65535u;
            }
            n[i * h->S + a0 + x] = uint16_t(total);
        }
    }
    return err;
}

mclg_status upload_state(mclg_ctx *h, const uint16_t *n, uint64_t t)
{
    const bool dev = is_device_ptr(n);
    const uint16_t *src = n;
    if (!dev) {
        MCLG_CK(cudaMemcpyAsync(h->d_stage, n, 3 * h->S * sizeof(uint16_t), cudaMemcpyHostToDevice,
                                h->stream));
        src = h->d_stage;
    }
    MCLG_CK(launch_to_device_form(src, h->S, h->d_B[h->cur], h->lay, streaming(h) ? 1 : 0,
                                  h->stream));
    if (h->halo) {
        // the edge values that arrived from the neighbouring blocks are part of the
        // given field: v = +1 at node 0 and v = -1 at node L - 1
        MCLG_CK(cudaMemcpyAsync(h->d_halo, src + 2 * h->S, sizeof(uint16_t),
                                cudaMemcpyDeviceToDevice, h->stream));
        MCLG_CK(cudaMemcpyAsync(h->d_halo + 1, src + (h->S - 1), sizeof(uint16_t),
                                cudaMemcpyDeviceToDevice, h->stream));
        h->halo_ready = true;
        h->stepped = false;
    }
    MCLG_CK(cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream));
    if (!dev) MCLG_CK(cudaStreamSynchronize(h->stream));  // the caller may free n on return
    h->t = t;
    h->sticky = 0;
    h->has_state = true;
    return MCLG_OK;
}

}  // namespace

extern "C" {

void mclg_default_params(mclg_params *p)
{
    if (!p) return;
    p->C = 10;
    p->lambda_num = 1;
    p->lambda_den = 1;
    p->flags = 0;
    p->mode = MCLG_MODE_AUTO;
    p->first_replica = 0;
    p->sampler = MCLG_SAMPLER_SEQUENTIAL;
    p->slice_n_max = 0;
    p->kernel_variant = 0;
    p->node_offset = 0;
}

const char *mclg_status_str(mclg_status s)
{
    switch (s) {
    case MCLG_OK: return "ok";
    case MCLG_ERR_ARG: return "invalid argument";
    case MCLG_ERR_NOMEM: return "out of memory";
    case MCLG_ERR_CUDA: return "CUDA runtime error";
    case MCLG_ERR_OVERFLOW: return "occupation overflow (uint16)";
    case MCLG_ERR_TIMEOUT: return "device wait timed out";
    case MCLG_ERR_STATE: return "no state set";
    case MCLG_ERR_SAMPLER: return "sampler could not decide (refinement cap / table tie)";
    }
    return "unknown status";
}

void mclg_destroy(mclg_handle h)
{
    if (!h) return;
    if (h->stream || h->d_err) cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->aux) {
        cudaStreamSynchronize(h->aux);
        cudaStreamDestroy(h->aux);
    }
    drop_graphs(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    cudaFree(h->d_B[0]);
    cudaFree(h->d_B[1]);
    cudaFree(h->d_err);
    cudaFree(h->d_totals);
    cudaFree(h->d_stage);
    cudaFree(h->d_stageNJ);
    cudaFree(h->d_units);
    cudaFree(h->d_unit_counter);
    cudaFree(h->d_t);
    free_slice_tables(h);
    cudaFree(h->lay.d_abi_off);
    cudaFree(h->lay.d_rep_off);
    cudaFree(h->lay.d_rep_L);
    cudaFree(h->lay.d_rep_id);
    cudaFree(h->lay.d_chunk_rep);
    cudaFree(h->st.s1);
    cudaFree(h->st.s2);
    cudaFree(h->st.snb);
    cudaFree(h->st.mean32);
    cudaFree(h->st.mean32c);
    cudaFree(h->st.m2);
    cudaFree(h->st.m2c);
    cudaFree(h->st.count);
    cudaFree(h->d_stat_partials);
    cudaFree(h->d_halo);
    cudaFree(h->d_stats_from);
    delete h;
}

mclg_status mclg_create(const uint32_t *L, uint32_t replicas, uint64_t seed, const mclg_params *p,
                        void *cuda_stream, mclg_handle *out)
{
    if (!out) return MCLG_ERR_ARG;
    *out = nullptr;
    if (!L || replicas == 0) return MCLG_ERR_ARG;
    mclg_params prm;
    mclg_default_params(&prm);
    if (p) prm = *p;
    if (prm.lambda_den < 1 || prm.lambda_den > 256 || prm.lambda_num > prm.lambda_den) return MCLG_ERR_ARG;
    if (prm.mode > MCLG_MODE_BATCHED ||
        (prm.flags & ~(MCLG_NO_STREAM | MCLG_STATS | MCLG_GALILEAN | MCLG_HALO)))
        return MCLG_ERR_ARG;
    if (prm.flags & MCLG_HALO) {
        // one block of a larger periodic lattice: one replica, global node indices < 2^32,
        // node pairs of the slice sampler's random numbers aligned with the lattice's
        if (replicas != 1 || (prm.flags & MCLG_STATS) || prm.mode == MCLG_MODE_PERSISTENT ||
            uint64_t(prm.node_offset) + L[0] > (uint64_t(1) << 32) ||
            (prm.sampler == MCLG_SAMPLER_SLICE && (prm.node_offset & 7u)))
            return MCLG_ERR_ARG;
    } else if (prm.node_offset != 0) {
        return MCLG_ERR_ARG;
    }
    uint64_t S = 0;
    for (uint32_t r = 0; r < replicas; ++r) {
        if (L[r] == 0 || L[r] > (uint32_t(1) << 31)) return MCLG_ERR_ARG;
        S += L[r];
    }
    if (S >= (uint64_t(1) << 40)) return MCLG_ERR_ARG;
    if (uint64_t(prm.first_replica) + replicas > (uint64_t(1) << 32)) return MCLG_ERR_ARG;
    if (prm.sampler > MCLG_SAMPLER_SLICE) return MCLG_ERR_ARG;
    const bool stats_form = (prm.flags & MCLG_STATS) && prm.sampler == MCLG_SAMPLER_SLICE;
    if (prm.kernel_variant > (stats_form ? kStatsConfigs
                              : prm.sampler == MCLG_SAMPLER_SLICE ? kSliceVariants : kPlainVariants))
        return MCLG_ERR_ARG;
    if (prm.sampler == MCLG_SAMPLER_SLICE &&
        (prm.C > uint32_t(kSliceMaxC) || prm.slice_n_max > kSliceMaxN))
        return MCLG_ERR_ARG;
    if (prm.flags & MCLG_STATS)
        for (uint32_t r = 1; r < replicas; ++r)
            if (L[r] != L[0]) return MCLG_ERR_ARG;

    mclg_ctx *h = new (std::nothrow) mclg_ctx();
    if (!h) return MCLG_ERR_NOMEM;
    h->prm = prm;
    if (prm.kernel_variant) {  // a fixed launch variant: no autotuning
        if (stats_form) h->stats_config = prm.kernel_variant - 1u;
        else h->plain_variant = prm.kernel_variant - 1u;
        h->plain_tuned = true;
    }
    h->seed = seed;
    h->R = replicas;
    h->L.assign(L, L + replicas);
    h->S = S;
    h->abi_off.resize(replicas);
    uint64_t acc = 0;
    for (uint32_t r = 0; r < replicas; ++r) {
        h->abi_off[r] = acc;
        acc += L[r];
    }
    // internal order: replicas that fit a persistent CTA first (ABI order
    // within each group); with statistics the ABI order is kept so that the
    // pooled positions line up with a fixed stride
    const bool keep_order = (prm.flags & MCLG_STATS) != 0;
    for (uint32_t r = 0; r < replicas; ++r)
        if (keep_order || pad8(L[r]) <= kMaxUnitNodes) h->order.push_back(r);
    h->n_small = 0;
    for (uint32_t r : h->order)
        if (pad8(L[r]) <= kMaxUnitNodes) ++h->n_small;
    if (keep_order) h->n_small = 0;
    if (!keep_order)
        for (uint32_t r = 0; r < replicas; ++r)
            if (pad8(L[r]) > kMaxUnitNodes) h->order.push_back(r);
    h->rep_off.resize(replicas);
    h->rep_L.resize(replicas);
    uint64_t off = 0;
    for (uint32_t k = 0; k < replicas; ++k) {
        h->rep_off[k] = off;
        h->rep_L[k] = L[h->order[k]];
        off += pad8(h->rep_L[k]);
    }
    h->lay.P = off;
    h->small_chunks = h->n_small ? (h->rep_off[h->n_small - 1] + pad8(h->rep_L[h->n_small - 1])) / 8 : 0;
    std::vector<uint32_t> chunk_rep(off / 8);
    for (uint32_t k = 0; k < replicas; ++k)
        for (uint64_t g = h->rep_off[k] / 8; g < (h->rep_off[k] + pad8(h->rep_L[k])) / 8; ++g)
            chunk_rep[g] = k;

    mclg_status st = MCLG_OK;
    auto fail = [&](mclg_status s) {
        mclg_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(MCLG_ERR_CUDA);
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(MCLG_ERR_CUDA);
    if (cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return fail(MCLG_ERR_CUDA);
    auto alloc = [&](void **ptr, size_t bytes) {
        if (cudaMalloc(ptr, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    };
    const size_t planes = 3 * h->lay.P * sizeof(uint16_t);
    if (!alloc((void **)&h->d_B[0], planes) || !alloc((void **)&h->d_B[1], planes) ||
        !alloc((void **)&h->d_err, sizeof(uint32_t)) ||
        !alloc((void **)&h->d_totals, 2 * sizeof(unsigned long long)) ||
        !alloc((void **)&h->d_unit_counter, sizeof(uint32_t)) ||
        !alloc((void **)&h->d_t, sizeof(uint32_t)) ||
        !alloc((void **)&h->d_stage, 3 * S * sizeof(uint16_t)) ||
        !alloc((void **)&h->lay.d_abi_off, replicas * sizeof(uint64_t)) ||
        !alloc((void **)&h->lay.d_rep_off, replicas * sizeof(uint64_t)) ||
        !alloc((void **)&h->lay.d_rep_L, replicas * sizeof(uint32_t)) ||
        !alloc((void **)&h->lay.d_rep_id, replicas * sizeof(uint32_t)) ||
        !alloc((void **)&h->lay.d_chunk_rep, chunk_rep.size() * sizeof(uint32_t)))
        return fail(MCLG_ERR_NOMEM);
    h->halo = (prm.flags & MCLG_HALO) != 0;
    if (h->halo && !alloc((void **)&h->d_halo, 2 * sizeof(uint16_t))) return fail(MCLG_ERR_NOMEM);
    if (cudaMemcpy(h->lay.d_abi_off, h->abi_off.data(), replicas * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->lay.d_rep_off, h->rep_off.data(), replicas * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->lay.d_rep_L, h->rep_L.data(), replicas * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->lay.d_rep_id, h->order.data(), replicas * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->lay.d_chunk_rep, chunk_rep.data(), chunk_rep.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->d_err, 0, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(h->d_B[0], 0, planes) != cudaSuccess || cudaMemset(h->d_B[1], 0, planes) != cudaSuccess)
        return fail(MCLG_ERR_CUDA);
    if (prm.flags & MCLG_STATS) {
        const uint32_t Lc = L[0];
        if (!alloc((void **)&h->st.s1, Lc * 3 * sizeof(long long)) ||
            !alloc((void **)&h->st.s2, Lc * 6 * sizeof(long long)) ||
            !alloc((void **)&h->st.snb, Lc * 9 * sizeof(long long)) ||
            !alloc((void **)&h->st.mean32, Lc * 3 * sizeof(float)) ||
            !alloc((void **)&h->st.mean32c, Lc * 3 * sizeof(float)) ||
            !alloc((void **)&h->st.m2, Lc * 6 * sizeof(float)) ||
            !alloc((void **)&h->st.m2c, Lc * 6 * sizeof(float)) ||
            !alloc((void **)&h->st.count, 3 * sizeof(unsigned long long)) ||
            !alloc((void **)&h->d_stats_from, sizeof(uint32_t)) ||
            !alloc((void **)&h->d_stat_partials, stats_partials_bytes(Lc, replicas)))
            return fail(MCLG_ERR_NOMEM);
        *out = h;
        st = mclg_stats_reset(h);
        if (st != MCLG_OK) {
            *out = nullptr;
            return fail(st);
        }
    }
    *out = h;
    return MCLG_OK;
}

mclg_status mclg_set_state(mclg_handle h, const uint16_t *n, uint64_t t)
{
    if (!h || !n || t >= kMaxT) return MCLG_ERR_ARG;
    MCLG_CK(cudaSetDevice(h->device));
    return upload_state(h, n, t);
}

mclg_status mclg_init(mclg_handle h, const double *rho, const double *u)
{
    if (!h || !rho || !u) return MCLG_ERR_ARG;
    MCLG_CK(cudaSetDevice(h->device));
    std::vector<uint16_t> n;
    try {
        n.resize(3 * h->S);
    } catch (...) {
        return MCLG_ERR_NOMEM;
    }
    // split the nodes into ranges of at most 64K nodes, spread over the host cores
    struct Task { uint32_t r, xb, xe; };
    std::vector<Task> tasks;
    for (uint32_t r = 0; r < h->R; ++r)
        for (uint32_t xb = 0; xb < h->L[r]; xb += 65536u)
            tasks.push_back({r, xb, std::min<uint32_t>(h->L[r], xb + 65536u)});
    unsigned nth = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 64u));
    nth = std::min<unsigned>(nth, unsigned(tasks.size()));
    std::vector<int> errs(nth, 0);
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < nth; ++w)
        pool.emplace_back([&, w]() {
            for (size_t i = w; i < tasks.size(); i += nth)
                errs[w] |= init_range(h, rho, u, n.data(), tasks[i].r, tasks[i].xb, tasks[i].xe);
        });
    for (auto &th : pool) th.join();
    int err = 0;
    for (int e : errs) err |= e;
    if (err & 8) return MCLG_ERR_ARG;
    mclg_status s = upload_state(h, n.data(), 0);
    if (s != MCLG_OK) return s;
    if (err & 1) {
        h->sticky |= kErrOverflow;
        return MCLG_ERR_OVERFLOW;
    }
    return MCLG_OK;
}

mclg_status mclg_get_state(mclg_handle h, uint16_t *n, uint64_t *t)
{
    if (!h || !n) return MCLG_ERR_ARG;
    if (!h->has_state || (h->halo && !h->halo_ready)) return MCLG_ERR_STATE;
    MCLG_CK(cudaSetDevice(h->device));
    const bool dev = is_device_ptr(n);
    uint16_t *dst = dev ? n : h->d_stage;
    MCLG_CK(launch_from_device_form(h->d_B[h->cur], dst, h->S, h->lay, streaming(h) ? 1 : 0,
                                    h->halo ? h->d_halo : nullptr, h->stream));
    if (!dev)
        MCLG_CK(cudaMemcpyAsync(n, h->d_stage, 3 * h->S * sizeof(uint16_t), cudaMemcpyDeviceToHost,
                                h->stream));
    if (t) *t = h->t;
    return collect_errors(h);
}

mclg_status mclg_step(mclg_handle h, uint64_t n_steps)
{
    if (!h) return MCLG_ERR_ARG;
    if (!h->has_state) return MCLG_ERR_STATE;
    if (h->t + n_steps > kMaxT) return MCLG_ERR_ARG;
    if (h->sticky) return status_from_bits(h->sticky);
    if (n_steps == 0) return MCLG_OK;
    if (h->halo) {
        // a block exchanges its edge values after every step
        if (n_steps != 1) return MCLG_ERR_ARG;
        if (!h->halo_ready) return MCLG_ERR_STATE;
    }
    MCLG_CK(cudaSetDevice(h->device));
    const uint32_t mode = effective_mode(h);
    if (h->prm.sampler == MCLG_SAMPLER_SLICE) {
        mclg_status st = ensure_slice_tables(h);
        if (st != MCLG_OK) return st;
    }
    if (mode == MCLG_MODE_PLAIN || mode == 3u) {
        if (!h->plain_tuned) {
            mclg_status st = autotune_plain(h, mode, 0, h->R);
            if (st != MCLG_OK) return st;
        }
        if (mode == 3u || h->R == 1) {
            // one launch (plus statistics) per step: replay captured graphs
            int c = h->cur;
            mclg_status st = plain_steps(h, h->cur, h->t, n_steps, 0, h->R, h->stream, &c);
            if (st != MCLG_OK) return st;
            h->cur = c;
            h->t += n_steps;
            if (h->halo) {
                h->halo_ready = false;  // the neighbours' values for the new time are still to come
                h->stepped = true;
            }
            if (h->prm.flags & MCLG_STATS) h->stats_count += n_steps * h->R;
        } else {
            // the per-replica baseline: one launch per replica and step
            for (uint64_t s = 0; s < n_steps; ++s) {
                MCLG_CK(plain_per_replica_step(h, h->d_B[h->cur], h->d_B[h->cur ^ 1], h->t,
                                               h->stream));
                h->cur ^= 1;
                h->t += 1;
            }
        }
        return MCLG_OK;
    }
    // persistent: small replicas stay on chip for all n_steps (chunks of at
    // most 2^16 steps per launch); large replicas step beside them on the aux
    // stream with one batched plain launch per step
    if (!h->tuned) {
        mclg_status s = autotune(h);
        if (s != MCLG_OK) return s;
    }
    if (!h->plain_tuned && h->n_small < h->R) {
        // variant for the long replicas, which step with batched plain launches
        mclg_status st = autotune_plain(h, 3u, h->n_small, h->R);
        if (st != MCLG_OK) return st;
    }
    const int start = h->cur;
    const int final_buf = int((uint64_t(start) + n_steps) & 1u);
    // Long replicas step with one batched plain launch per step.  When they
    // alone fill the GPU they go first on the handle's stream; otherwise they
    // run beside the persistent kernel on the second stream.
    const uint64_t long_nodes = h->lay.P - h->small_chunks * 8u;
    const bool has_long = h->n_small < h->R;
    const bool beside = has_long && long_nodes < (uint64_t(1) << 20);
    cudaStream_t long_stream = beside ? h->aux : h->stream;
    if (beside) {
        MCLG_CK(cudaEventRecord(h->ev_fork, h->stream));
        MCLG_CK(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    }
    if (has_long) {
        int c = start;
        mclg_status st = plain_steps(h, start, h->t, n_steps, h->n_small, h->R, long_stream, &c);
        if (st != MCLG_OK) return st;
        if (beside) MCLG_CK(cudaEventRecord(h->ev_join, h->aux));
    }
    // Each CTA reads its own unit into shared memory before it writes the unit
    // back, and units do not overlap, so launches after the first work in place.
    uint64_t done = 0;
    const uint16_t *in = h->d_B[start];
    uint16_t *outb = h->d_B[final_buf];
    while (done < n_steps && h->n_small > 0) {
        const uint32_t chunk = uint32_t(std::min<uint64_t>(n_steps - done, 65536u));
        PersistentArgs a = persistent_args(h, in, outb, h->t + done, chunk, h->d_units, h->p_cap);
        MCLG_CK(launch_persistent(a, uint32_t(h->units.size()), h->p_threads, h->stream));
        in = outb;
        done += chunk;
    }
    if (beside) MCLG_CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    h->cur = final_buf;
    h->t += n_steps;
    return MCLG_OK;
}

mclg_status mclg_moments(mclg_handle h, int32_t *N, int32_t *J, int64_t *totals)
{
    if (!h) return MCLG_ERR_ARG;
    if (!h->has_state || (h->halo && !h->halo_ready)) return MCLG_ERR_STATE;
    MCLG_CK(cudaSetDevice(h->device));
    const bool devN = N && is_device_ptr(N), devJ = J && is_device_ptr(J);
    if ((N && !devN) || (J && !devJ)) {
        if (!h->d_stageNJ && cudaMalloc(&h->d_stageNJ, 2 * h->S * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            return MCLG_ERR_NOMEM;
        }
    }
    int32_t *dN = N ? (devN ? N : h->d_stageNJ) : nullptr;
    int32_t *dJ = J ? (devJ ? J : h->d_stageNJ + h->S) : nullptr;
    MCLG_CK(cudaMemsetAsync(h->d_totals, 0, 2 * sizeof(unsigned long long), h->stream));
    MCLG_CK(launch_moments(h->d_B[h->cur], dN, dJ, h->lay, streaming(h) ? 1 : 0,
                           h->halo ? h->d_halo : nullptr, h->d_totals, h->stream));
    if (N && !devN)
        MCLG_CK(cudaMemcpyAsync(N, dN, h->S * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    if (J && !devJ)
        MCLG_CK(cudaMemcpyAsync(J, dJ, h->S * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    unsigned long long tot[2] = {0, 0};
    MCLG_CK(cudaMemcpyAsync(tot, h->d_totals, sizeof(tot), cudaMemcpyDeviceToHost, h->stream));
    mclg_status s = collect_errors(h);
    if (totals) {
        totals[0] = (int64_t)tot[0];
        totals[1] = (int64_t)tot[1];
    }
    return s;
}

mclg_status mclg_stats_reset(mclg_handle h)
{
    if (!h) return MCLG_ERR_ARG;
    if (!(h->prm.flags & MCLG_STATS)) return MCLG_ERR_ARG;
    MCLG_CK(cudaSetDevice(h->device));
    const size_t Lc = h->L[0];
    MCLG_CK(cudaMemsetAsync(h->st.s1, 0, Lc * 3 * sizeof(long long), h->stream));
    MCLG_CK(cudaMemsetAsync(h->st.s2, 0, Lc * 6 * sizeof(long long), h->stream));
    MCLG_CK(cudaMemsetAsync(h->st.snb, 0, Lc * 9 * sizeof(long long), h->stream));
    MCLG_CK(cudaMemsetAsync(h->st.mean32, 0, Lc * 3 * sizeof(float), h->stream));
    MCLG_CK(cudaMemsetAsync(h->st.mean32c, 0, Lc * 3 * sizeof(float), h->stream));
    MCLG_CK(cudaMemsetAsync(h->st.m2, 0, Lc * 6 * sizeof(float), h->stream));
    MCLG_CK(cudaMemsetAsync(h->st.m2c, 0, Lc * 6 * sizeof(float), h->stream));
    MCLG_CK(cudaMemsetAsync(h->st.count, 0, 3 * sizeof(unsigned long long), h->stream));
    MCLG_CK(cudaMemsetAsync(h->d_stat_partials, 0, stats_partials_bytes(uint32_t(Lc), h->R),
                            h->stream));
    h->stats_count = 0;
    return MCLG_OK;
}

mclg_status mclg_stats_read(mclg_handle h, int64_t *s1, int64_t *s2, int64_t *snb, float *cov32,
                            double *cov64, uint64_t *count)
{
    if (!h) return MCLG_ERR_ARG;
    if (!(h->prm.flags & MCLG_STATS)) return MCLG_ERR_ARG;
    MCLG_CK(cudaSetDevice(h->device));
    const size_t Lc = h->L[0];
    std::vector<long long> a1(Lc * 3), a2(Lc * 6), anb(Lc * 9);
    std::vector<float> m2(Lc * 6);
    unsigned long long cnt = 0;
    MCLG_CK(cudaMemcpyAsync(a1.data(), h->st.s1, a1.size() * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    MCLG_CK(cudaMemcpyAsync(a2.data(), h->st.s2, a2.size() * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    MCLG_CK(cudaMemcpyAsync(anb.data(), h->st.snb, anb.size() * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    MCLG_CK(cudaMemcpyAsync(m2.data(), h->st.m2, m2.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    MCLG_CK(cudaMemcpyAsync(&cnt, h->st.count, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
    mclg_status s = collect_errors(h);
    if (s1) std::memcpy(s1, a1.data(), a1.size() * sizeof(int64_t));
    if (s2) std::memcpy(s2, a2.data(), a2.size() * sizeof(int64_t));
    if (snb) std::memcpy(snb, anb.data(), anb.size() * sizeof(int64_t));
    static const int pi[6] = {0, 0, 0, 1, 1, 2}, pj[6] = {0, 1, 2, 1, 2, 2};
    for (size_t x = 0; x < Lc; ++x)
        for (int q = 0; q < 6; ++q) {
            if (cov32) cov32[6 * x + q] = cnt ? m2[6 * x + q] / float(cnt) : 0.0f;
            if (cov64) {
                if (!cnt) {
                    cov64[6 * x + q] = 0.0;
                    continue;
                }
                const __int128 num = (__int128)cnt * a2[6 * x + q] -
                                     (__int128)a1[3 * x + pi[q]] * a1[3 * x + pj[q]];
                cov64[6 * x + q] = double((long double)num / ((long double)cnt * (long double)cnt));
            }
        }
    if (count) *count = cnt;
    return s;
}

mclg_status mclg_sync(mclg_handle h)
{
    if (!h) return MCLG_ERR_ARG;
    MCLG_CK(cudaSetDevice(h->device));
    return collect_errors(h);
}

uint64_t mclg_time(mclg_handle h) { return h ? h->t : 0; }

mclg_status mclg_halo_get(mclg_handle h, uint16_t *out)
{
    if (!h || !out || !h->halo) return MCLG_ERR_ARG;
    if (!h->stepped) return MCLG_ERR_STATE;
    MCLG_CK(cudaSetDevice(h->device));
    // post-collision values of the last step, kept where they were collided
    // (the device form): v = -1 of node 0 and v = +1 of node L - 1
    const uint16_t *B = h->d_B[h->cur];
    const bool dev = is_device_ptr(out);
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    MCLG_CK(cudaMemcpyAsync(out, B + h->rep_off[0], sizeof(uint16_t), kind, h->stream));
    MCLG_CK(cudaMemcpyAsync(out + 1, B + 2 * h->lay.P + h->rep_off[0] + h->L[0] - 1,
                            sizeof(uint16_t), kind, h->stream));
    if (!dev) return collect_errors(h);
    return MCLG_OK;
}

mclg_status mclg_halo_put(mclg_handle h, const uint16_t *in)
{
    if (!h || !in || !h->halo) return MCLG_ERR_ARG;
    if (!h->stepped) return MCLG_ERR_STATE;
    MCLG_CK(cudaSetDevice(h->device));
    const bool dev = is_device_ptr(in);
    MCLG_CK(cudaMemcpyAsync(h->d_halo, in, 2 * sizeof(uint16_t),
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    if (!dev) MCLG_CK(cudaStreamSynchronize(h->stream));  // the caller may reuse `in` on return
    h->halo_ready = true;
    return MCLG_OK;
}

mclg_status mclg_slice_row(uint32_t N, int32_t J, uint32_t b, uint32_t C, uint32_t lambda_num,
                           uint32_t lambda_den, uint64_t *F, int32_t *dmin, int32_t *dmax,
                           uint16_t *record)
{
    const uint32_t Jp = uint32_t(J < 0 ? -int64_t(J) : J);
    if (!F || !dmin || !dmax || C > uint32_t(kSliceMaxC) || N < 2 || Jp > N || b > N - Jp ||
        ((N - Jp - b) & 1u) || lambda_den < 1 || lambda_den > 256 || lambda_num > lambda_den)
        return MCLG_ERR_ARG;
    // the exact law's numerators over D^C, shifted by 2^64, must fit the
    // builder's 512-bit integers: D = 8 N^2 lambda_den < 2^44
    if (8ull * uint64_t(N) * N * lambda_den >= kSliceMaxD) return MCLG_ERR_ARG;
    int lo = 0, hi = 0;
    build_slice_row(N, Jp, b, C, lambda_num, lambda_den, F, lo, hi);
    if (record) build_slice_record(F, hi - lo, -lo, record);
    *dmin = lo;
    *dmax = hi;
    return MCLG_OK;
}

mclg_status mclg_tuning(mclg_handle h, uint32_t cfg[6])
{
    if (!h || !cfg) return MCLG_ERR_ARG;
    cfg[4] = h->tuned ? h->p_variant : 0u;
    cfg[5] = fused_stats(h) && h->plain_tuned ? h->stats_config : 0u;
    const uint32_t vec = h->prm.sampler == MCLG_SAMPLER_SLICE ? slice_variant_vec(h->plain_variant)
                                                               : plain_variant_vec(h->plain_variant);
    cfg[0] = h->plain_tuned ? vec * 100u + h->plain_variant : 0u;
    cfg[1] = h->tuned ? h->p_threads : 0u;
    cfg[2] = h->tuned ? h->p_cap : 0u;
    cfg[3] = h->tuned ? uint32_t(h->units.size()) : 0u;
    return MCLG_OK;
}

mclg_status mclg_philox(const uint32_t *ctr, uint64_t n, uint64_t seed, uint32_t *out, void *cuda_stream)
{
    if ((!ctr || !out) && n) return MCLG_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    MCLG_CK(launch_philox(ctr, n, uint32_t(seed), uint32_t(seed >> 32), out, s));
    MCLG_CK(cudaStreamSynchronize(s));
    return MCLG_OK;
}

}  // extern "C"
