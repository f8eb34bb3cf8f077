// Allocation-free node moments: the same N, J and totals as mclg_moments,
// computed from a caller-owned device field with no device allocation.
//
// Who needs it: callers whose device memory is owned by someone else's pool
// (a host framework's caching allocator may hold nearly all of the GPU, so a
// raw cudaMalloc from this library would fail or fragment that pool), and
// latency-sensitive loops that cannot accept the device-wide synchronisation
// that cudaMalloc/cudaFree may imply.  Such callers pass their own input and
// output buffers; the only scratch this path needs (per-block partial sums of
// the two-pass reduction) lives in a fixed file-scope device array that every
// GPU loading this library keeps until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/mclg.h"

namespace {

constexpr uint32_t kThreads = 256;           // threads per block
constexpr uint32_t kNodesPerThread = 8;      // nodes summed by each thread
constexpr uint32_t kMaxBlocks = 32768;       // partial-sum slots in the scratch array
constexpr uint64_t kMaxNodes = uint64_t(kMaxBlocks) * kThreads * kNodesPerThread;  // 2^26
constexpr int kMaxDevices = 64;

// Scratch: [2 * b] and [2 * b + 1] hold block b's (sum N, sum J); the last two
// slots hold the final totals.  512 KiB + 16 B per device.  Every slot that a
// call reads is written earlier in the same call, so nothing has to be zeroed.
static __device__ __align__(256) long long g_moments_scratch[2 * kMaxBlocks + 2];

// Device address of the scratch array for each device, looked up once with
// that device current (the host-side name is not a device address).
long long *g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_lock;

cudaError_t scratch_for_current_device(long long **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_setup_lock);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_moments_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<long long *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Pass 1: per-node N = n_-1 + n_0 + n_+1 and J = n_+1 - n_-1 of the canonical
// field (Sec. III, Sec. IV.A), and each block's partial sums into the scratch.
__global__ void __launch_bounds__(kThreads)
    k_moments_partials(const uint16_t *__restrict__ n, uint64_t S, int32_t *__restrict__ N,
                       int32_t *__restrict__ J, long long *__restrict__ partials)
{
    long long sn = 0, sj = 0;
    const uint64_t base = uint64_t(blockIdx.x) * kThreads * kNodesPerThread;
    for (uint32_t k = 0; k < kNodesPerThread; ++k) {
        const uint64_t x = base + uint64_t(k) * kThreads + threadIdx.x;
        if (x < S) {
            const int32_t a = n[x], b = n[S + x], c = n[2 * S + x];
            if (N) N[x] = a + b + c;
            if (J) J[x] = c - a;
            sn += a + b + c;
            sj += c - a;
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        sn += __shfl_down_sync(0xFFFFFFFFu, sn, d);
        sj += __shfl_down_sync(0xFFFFFFFFu, sj, d);
    }
    __shared__ long long ws[2][kThreads / 32];
    const uint32_t w = threadIdx.x >> 5;
    if ((threadIdx.x & 31u) == 0) {
        ws[0][w] = sn;
        ws[1][w] = sj;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tn = 0, tj = 0;
        for (uint32_t k = 0; k < kThreads / 32; ++k) {
            tn += ws[0][k];
            tj += ws[1][k];
        }
        partials[2 * blockIdx.x] = tn;
        partials[2 * blockIdx.x + 1] = tj;
    }
}

// Pass 2: one block sums the partials of pass 1 into the final two slots.
__global__ void __launch_bounds__(kThreads) k_moments_final(long long *__restrict__ partials,
                                                           uint32_t blocks)
{
    long long sn = 0, sj = 0;
    for (uint32_t b = threadIdx.x; b < blocks; b += kThreads) {
        sn += partials[2 * b];
        sj += partials[2 * b + 1];
    }
    for (int d = 16; d > 0; d >>= 1) {
        sn += __shfl_down_sync(0xFFFFFFFFu, sn, d);
        sj += __shfl_down_sync(0xFFFFFFFFu, sj, d);
    }
    __shared__ long long ws[2][kThreads / 32];
    const uint32_t w = threadIdx.x >> 5;
    if ((threadIdx.x & 31u) == 0) {
        ws[0][w] = sn;
        ws[1][w] = sj;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tn = 0, tj = 0;
        for (uint32_t k = 0; k < kThreads / 32; ++k) {
            tn += ws[0][k];
            tj += ws[1][k];
        }
        partials[2 * kMaxBlocks] = tn;
        partials[2 * kMaxBlocks + 1] = tj;
    }
}

// The device that holds p, or -1 when p is not device memory (host memory,
// or an address the runtime does not know).  Managed memory counts as the
// device it is attributed to.
int device_of(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the lookup failure (entry checked that nothing else was pending)
        return -1;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? a.device : -1;
}

}  // namespace

extern "C" mclg_status mclg_moments_noalloc(const uint16_t *n, uint64_t S, int32_t *N, int32_t *J,
                                            int64_t *totals, void *cuda_stream)
{
    if (!n || S == 0) return MCLG_ERR_ARG;
    if (S > kMaxNodes) return MCLG_ERR_ARG;  // beyond the fixed scratch: 2^26 nodes
    // an error left pending by earlier work of the caller is reported, not consumed
    if (cudaPeekAtLastError() != cudaSuccess) return MCLG_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MCLG_ERR_CUDA;
    // every device buffer must live on the current device: the kernels run there
    if (device_of(n) != dev || (N && device_of(N) != dev) || (J && device_of(J) != dev))
        return MCLG_ERR_ARG;
    const int tot_dev = totals ? device_of(totals) : -1;
    if (tot_dev >= 0 && tot_dev != dev) return MCLG_ERR_ARG;
    long long *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return MCLG_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const uint32_t blocks = uint32_t((S + uint64_t(kThreads) * kNodesPerThread - 1) /
                                     (uint64_t(kThreads) * kNodesPerThread));
    k_moments_partials<<<blocks, kThreads, 0, s>>>(n, S, N, J, scratch);
    if (cudaGetLastError() != cudaSuccess) return MCLG_ERR_CUDA;
    k_moments_final<<<1, kThreads, 0, s>>>(scratch, blocks);
    if (cudaGetLastError() != cudaSuccess) return MCLG_ERR_CUDA;
    if (totals) {
        const cudaMemcpyKind kind = tot_dev >= 0 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (cudaMemcpyAsync(totals, scratch + 2 * kMaxBlocks, 2 * sizeof(long long), kind, s) !=
            cudaSuccess)
            return MCLG_ERR_CUDA;
        if (kind == cudaMemcpyDeviceToHost && cudaStreamSynchronize(s) != cudaSuccess)
            return MCLG_ERR_CUDA;
    }
    return MCLG_OK;
}
