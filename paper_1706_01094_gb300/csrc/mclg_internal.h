// Internal declarations shared by the library's translation units (not part
// of the public C ABI in include/mclg.h).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "mclg_device.cuh"

namespace mclg {

constexpr uint32_t kPlainThreads = 256;          // threads per CTA of the plain kernel
constexpr uint32_t kSliceThreads = 128;          // threads per CTA of the slice kernel (measured best)
constexpr uint32_t kPersistentMaxThreads = 512;  // upper bound on persistent CTA size
constexpr uint32_t kMaxUnitReplicas = 512;       // replicas packed into one persistent CTA
constexpr uint32_t kMaxUnitNodes = 4096;         // longest replica kept in a persistent CTA
constexpr uint32_t kPersistentVariants = 3;      // register bounds of the persistent kernel
constexpr int kSliceMaxC = 10;                   // slice sampler: sub-collisions per step
constexpr int kSliceRowU64 = 20;                 // secondary row: 2C entries
constexpr int kSliceRecordLanes = 8;             // 15-bit values per 16-byte record
constexpr uint32_t kSliceMaxN = 1024;            // largest mass the slice tables may cover (records < 2^32)
constexpr uint64_t kSliceMaxD = uint64_t(1) << 44;  // exact-law denominator base D = 8 N^2 lambda_den
constexpr uint32_t kSliceDefaultN = 256;         // slice tables' mass range unless set
constexpr uint32_t kPlainVariants = 6;           // plain-kernel launch variants (see launch_plain)
constexpr uint32_t kSliceVariants = 20;          // slice-kernel launch variants (see launch_slice)
constexpr uint32_t kSliceTbFirst = 14;           // of which the temporally blocked ones: 14 ..
constexpr uint32_t kSliceClassicVariants = 6;    // of which k_step_slice; the rest single-replica forms

// Device-resident description of the internal replica order.
struct Layout {
    uint64_t P = 0;                   // padded nodes per plane (multiple of 8)
    uint64_t *d_abi_off = nullptr;    // [R] ABI offset of replica id r (prefix sum of L)
    uint64_t *d_rep_off = nullptr;    // [R] internal offset of internal replica k
    uint32_t *d_rep_L = nullptr;      // [R] length of internal replica k
    uint32_t *d_rep_id = nullptr;     // [R] replica id r (ABI index, RNG key) of internal k
    uint32_t *d_chunk_rep = nullptr;  // [P/8] internal replica of each 8-node chunk
};

struct PlainArgs {
    const uint16_t *in;
    uint16_t *out;
    uint64_t P;
    uint64_t g_begin, g_end;  // chunk range (whole replicas)
    const uint32_t *chunk_rep;
    const uint64_t *rep_off;
    const uint32_t *rep_L;
    const uint32_t *rep_id;
    uint64_t one_off;  // single-replica launch: offset, length, id
    uint32_t one_L, one_rid;
    uint32_t t, C, lam_n, lam_d, k0, k1;
    uint32_t *err;
    uint32_t variant;  // plain-kernel variant (nodes per thread, register bound)
    uint32_t stream;   // 1: pull-stream before colliding, 0: collide only
    uint32_t galilean; // 1: per-node rate lambda / sqrt(1 + 3 u^2) (galilean_q)
    uint32_t r0;       // random-stream index of replica id 0
    const uint32_t *t_dev;  // if set, the time step is *t_dev + t (graph replays)
    // a block of a larger lattice (single-replica launches only): halo_in[0] is the
    // v = +1 value entering node 0 from the left, halo_in[1] the v = -1 value entering
    // node L - 1 from the right; nullptr for a periodic replica
    const uint16_t *halo_in;
    uint32_t x_base;   // global index of node 0 in the random numbers' counters
    RoundKeys rk;      // Philox round keys of the seed
};

struct Unit {
    uint64_t node_begin;  // internal node offset of the unit's first replica
    uint32_t nodes;       // padded nodes in the unit
    uint32_t rep_begin, rep_end;  // internal replica range
};

struct SliceTables {
    uint32_t n_max;             // tables cover N <= n_max (N < 2: identity)
    uint32_t rec_hb;            // n_max / 2 + 1: records per (N, |J|)
    const uint32_t *rowstart;   // [(n_max + 1)^2] first row of each (N, |J|) slice
    // [(n_max + 1)^2 rec_hb] the 16-byte record of state (N, |J|, b) at
    // (N (n_max + 1) + |J|) rec_hb + b / 2: lane j (16 bits, half j & 1 of
    // word j / 2) holds the top 15 bits of F[c0 - 4 + j] (see mclg_slice.cuh)
    const uint4 *record;
    const unsigned long long *secondary;  // [rows][kSliceRowU64]
    // nodes heavier than n_max, left for the sequential pass of the same step
    unsigned long long *heavy_pos;  // [heavy_cap] device-form node positions
    uint32_t *heavy_ctl;            // {count, overflow, blocks done}, zero between steps
    uint32_t heavy_cap;
};

struct PersistentArgs {
    const uint16_t *in;
    uint16_t *out;
    uint64_t P;
    const Unit *units;
    const uint64_t *rep_off;
    const uint32_t *rep_L;
    const uint32_t *rep_id;
    uint32_t cap;  // shared-memory nodes per buffer (>= every unit's nodes)
    uint32_t n_units;           // units in `units` (set by launch_persistent)
    uint32_t variant;           // register bound: 0, 1, 2 = 1, 2, 3 CTAs of 512 threads per SM
    uint32_t *unit_counter;     // work-queue counter, zeroed by launch_persistent
    uint32_t t0, n_steps, C, lam_n, lam_d, k0, k1;
    uint32_t *err;
    uint32_t stream;  // 1: pull-stream before colliding, 0: collide only
    uint32_t galilean; // 1: per-node rate lambda / sqrt(1 + 3 u^2) (galilean_q)
    uint32_t r0;      // random-stream index of replica id 0
    uint32_t slice;   // 1: the slice sampler (tables below, sequential draws beyond them)
    SliceTables tab;
    RoundKeys rk;     // Philox round keys of the seed
};

struct StatsBuffers {
    long long *s1, *s2, *snb;   // [L*3], [L*6], [L*9]
    float *mean32, *mean32c;    // [L*3] running means and their compensation
    float *m2, *m2c;            // [L*6] running co-moments and their compensation
    unsigned long long *count;  // [3]: samples per position, finishing ticket of the merge
                                // pass, samples in the batch not merged yet
};

// The statistics accumulated by the slice kernel's statistics form (one pass
// over the state per step: the kernel of step t adds the field it reads, n(t),
// when t >= *stats_from).
struct StatsArgs {
    uint32_t R;                        // replicas, all of length PlainArgs::one_L, ABI order
    uint64_t stride;                   // node offset between consecutive replicas
    const uint32_t *stats_from;        // first time step whose input field is a sample
    unsigned long long *batch;         // [L][18] sums of the batch
    unsigned long long *batch_count;   // samples in the batch
    uint32_t config;                   // launch configuration (see launch_slice_stats)
};
constexpr uint32_t kStatsConfigs = 4;  // statistics-form launch configurations

cudaError_t launch_plain(const PlainArgs &p, bool one, cudaStream_t s);

// Slice sampler (the C sub-collisions of a node drawn at once from tables).
uint64_t slice_rows(uint32_t n_max);
void build_slice_tables(uint32_t n_max, uint32_t C, uint32_t lam_n, uint32_t lam_d, bool galilean,
                        std::vector<uint32_t> &rowstart, std::vector<uint16_t> &record,
                        std::vector<uint64_t> &secondary);
uint64_t slice_records(uint32_t n_max);
constexpr uint32_t kHeavyCap = 1u << 20;         // heavy-node list entries (overflow: scan)
constexpr uint32_t kHeavyBlocks = 76;            // CTAs of the heavy-node pass of one replica (usually empty)
constexpr uint32_t kHeavyBatchBlocks = 608;      // of a launch over several replicas (many heavy nodes)
cudaError_t launch_slice(const PlainArgs &p, bool one, const SliceTables &tab, cudaStream_t s);
// Temporally blocked slice steps of one replica: n_steps <= slice_tb_steps(config)
// steps in one launch, from p.in to p.out (heavy nodes collided in place).
constexpr uint32_t kSliceTbConfigs = 6;
uint32_t slice_tb_steps(uint32_t config);
cudaError_t launch_slice_tb(const PlainArgs &p, const SliceTables &tab, uint32_t n_steps,
                            uint32_t config, cudaStream_t s);
void build_slice_record(const uint64_t *F, int n, int c0, uint16_t *record);
uint32_t slice_variant_vec(uint32_t variant);
void build_slice_row(uint32_t N, uint32_t J, uint32_t b, uint32_t C, uint32_t lam_n, uint32_t lam_d,
                     uint64_t *F, int &dmin, int &dmax);
uint32_t plain_variant_vec(uint32_t variant);
size_t persistent_smem_bytes(uint32_t cap);
cudaError_t launch_persistent(const PersistentArgs &p, uint32_t n_units, uint32_t threads,
                              cudaStream_t s);
cudaError_t launch_to_device_form(const uint16_t *n, uint64_t S, uint16_t *B, const Layout &lay,
                                  int stream, cudaStream_t s);
// halo (or nullptr): for a block of a larger lattice, the two arriving values
// that complete the canonical field (see PlainArgs::halo_in)
cudaError_t launch_from_device_form(const uint16_t *B, uint16_t *n, uint64_t S, const Layout &lay,
                                    int stream, const uint16_t *halo, cudaStream_t s);
cudaError_t launch_moments(const uint16_t *B, int32_t *N, int32_t *J, const Layout &lay, int stream,
                           const uint16_t *halo, unsigned long long *totals, cudaStream_t s);
size_t stats_partials_bytes(uint32_t L, uint32_t R);
// Statistics: the partial pass adds one field's exact sums to the batch sums
// (and R to the batch's sample count); the merge pass folds the batch into the
// int64 accumulators and the FP32 running moments and clears it.
cudaError_t launch_stats_partial(const uint16_t *B, uint64_t P, uint32_t L, uint32_t R,
                                 uint64_t stride, int stream, unsigned long long *batch,
                                 unsigned long long *batch_count, cudaStream_t s);
cudaError_t launch_stats_merge(unsigned long long *batch, uint32_t L, const StatsBuffers &st,
                               cudaStream_t s);
// One slice-sampler step of every replica with the statistics of its input field
// (then the heavy-node pass).
cudaError_t launch_slice_stats(const PlainArgs &p, const SliceTables &tab, const StatsArgs &sa,
                               cudaStream_t s);
cudaError_t launch_set_time(uint32_t *t_dev, uint32_t value, cudaStream_t s);
cudaError_t launch_advance_time(uint32_t *t_dev, uint32_t by, cudaStream_t s);
cudaError_t launch_philox(const uint32_t *ctr, uint64_t n, uint32_t k0, uint32_t k1, uint32_t *out,
                          cudaStream_t s);

}  // namespace mclg
