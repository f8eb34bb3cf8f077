// The slice sampler's draw of one node (Sec. III: the C sub-collisions of a
// node drawn at once from the exact C-step law of its (N, J) slice, Sec.
// III.A), shared by the per-step slice kernels and the persistent kernel.
#pragma once
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
    const uint32_t below = b >> 1;  // the state's row within its slice (b has the parity of N - |J|)
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

}  // namespace mclg
