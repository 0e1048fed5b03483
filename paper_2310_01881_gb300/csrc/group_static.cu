// group_static.cu -- leaf grouping (K-b) for callers that cannot allocate device memory.
//
// The paper has no counterpart: this is a library convenience.  Some callers are
// not allowed to allocate at call time -- a frame loop whose device memory budget
// is fixed up front, or an engine that forbids cudaMalloc/cudaFree on its render
// thread because those calls can synchronise the whole device and stall every other
// stream.  amnerf_group_by_leaf_static groups crossings by leaf like the render
// pipeline does, but keeps its scratch (per-leaf write cursors, tile offsets and
// totals) in the file-scope device array below instead of context memory, so it
// calls no allocator at all.  The caller passes the inputs and the outputs.
//
// Limits and sharing:
//   - at most kStaticLeaves (4096) leaves; n_rays * maxc < 2^32;
//   - the array (about 33 KB) stays resident on every device that loads the library
//     until the process exits;
//   - every call shares the array and leaves the last call's contents in it; the
//     cursors are rewritten by each call before use, the caller's `counts` output is
//     cleared by the call; two calls whose work overlaps on the GPU (different
//     streams, no ordering between them) race on the array.
//   - The first call on a device resolves the array's device address with
//     cudaGetSymbolAddress (a host-side name of a __device__ array is not a device
//     address).  With lazy module loading that lookup may load this library's device
//     code and data, which allocates and synchronises: the first call is a warm-up
//     to make outside any no-allocation region and before any stream capture.
//   - The address is cached per device index for the life of the process; a device
//     or primary-context reset invalidates it, so the entry point must not be called
//     after one.
#include <mutex>

#include "amnerf_internal.h"

namespace amnerf {
namespace {

constexpr int kStaticLeaves = kMaxLeaves;
// cursor [4096] | tile offsets [4097] | pad | totals (4 x u64)
constexpr int kCursorOff = 0;
constexpr int kTileOff = kStaticLeaves;
constexpr int kStatsOff = 2 * kStaticLeaves + 8;  // 8-byte aligned word index
constexpr int kStaticWords = kStatsOff + 8;

static __device__ __align__(256) uint32_t g_group_scratch[kStaticWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_group_scratch on the current device (resolved once per device).
cudaError_t scratch_for_current_device(uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_group_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

constexpr int kThreads = 256;
constexpr int kItems = 16;

// Per-leaf crossing counts; crossings with a leaf id >= n_leaves are ignored.
__global__ void __launch_bounds__(kThreads) k_histogram_static(const uint8_t* __restrict__ n_x,
                                                               const uint16_t* __restrict__ leaf, uint32_t n_slots,
                                                               int maxc, uint32_t* __restrict__ counts, int n_leaves) {
    extern __shared__ uint32_t s_cnt[];
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();
    const uint32_t base = blockIdx.x * (uint32_t)(kThreads * kItems);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t s = base + (uint32_t)(i * kThreads) + threadIdx.x;
        if (s < n_slots) {
            const uint32_t ray = s / (uint32_t)maxc;
            if (s - ray * (uint32_t)maxc < (uint32_t)__ldg(n_x + ray)) {
                const uint32_t l = __ldg(leaf + s);
                if (l < (uint32_t)n_leaves) atomicAdd(&s_cnt[l], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(&counts[i], s_cnt[i]);
}

// Scatter of crossing ids into their leaf segments (shared-memory binned, one global
// atomic per touched leaf per CTA); the same rule for invalid leaf ids.
__global__ void __launch_bounds__(kThreads) k_scatter_static(const uint8_t* __restrict__ n_x,
                                                             const uint16_t* __restrict__ leaf, uint32_t n_slots,
                                                             int maxc, uint32_t* __restrict__ cursor,
                                                             uint32_t* __restrict__ order, int n_leaves) {
    extern __shared__ uint32_t sm[];
    uint32_t* s_cnt = sm;
    uint32_t* s_base = sm + n_leaves;
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();
    const uint32_t base = blockIdx.x * (uint32_t)(kThreads * kItems);
    uint32_t lf[kItems], rk[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t s = base + (uint32_t)(i * kThreads) + threadIdx.x;
        rk[i] = 0xffffffffu;
        lf[i] = 0u;
        if (s < n_slots) {
            const uint32_t ray = s / (uint32_t)maxc;
            if (s - ray * (uint32_t)maxc < (uint32_t)__ldg(n_x + ray)) {
                const uint32_t l = __ldg(leaf + s);
                if (l < (uint32_t)n_leaves) {
                    lf[i] = l;
                    rk[i] = atomicAdd(&s_cnt[l], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) {
        const uint32_t c = s_cnt[i];
        s_base[i] = c ? atomicAdd(&cursor[i], c) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (rk[i] != 0xffffffffu) order[s_base[lf[i]] + rk[i]] = base + (uint32_t)(i * kThreads) + threadIdx.x;
}

}  // namespace
}  // namespace amnerf

using namespace amnerf;

extern "C" amnerf_status amnerf_group_by_leaf_static(const uint8_t* n_x, const uint16_t* leaf, int64_t n_rays,
                                                     int maxc, int n_leaves, uint32_t* counts, uint32_t* offsets,
                                                     uint32_t* order, void* cuda_stream) {
    if (n_leaves < 1 || n_leaves > kStaticLeaves) return AMNERF_E_INVAL;  // beyond the static scratch
    if (maxc < 1 || maxc > 255 || n_rays < 0) return AMNERF_E_INVAL;
    if ((uint64_t)n_rays * (uint64_t)maxc >= (1ull << 32)) return AMNERF_E_INVAL;
    if (!counts || !offsets || (n_rays > 0 && (!n_x || !leaf || !order))) return AMNERF_E_INVAL;
    uint32_t* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return AMNERF_E_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const uint32_t n_slots = (uint32_t)((uint64_t)n_rays * (uint64_t)maxc);
    uint32_t* cursor = scratch + kCursorOff;
    uint32_t* tile_off = scratch + kTileOff;
    uint64_t* stats = reinterpret_cast<uint64_t*>(scratch + kStatsOff);
    if (cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)n_leaves, s) != cudaSuccess) return AMNERF_E_CUDA;
    const uint32_t per = (uint32_t)(kThreads * kItems);
    const unsigned blocks = (n_slots + per - 1) / per;
    if (blocks) {
        k_histogram_static<<<blocks, kThreads, sizeof(uint32_t) * n_leaves, s>>>(n_x, leaf, n_slots, maxc, counts,
                                                                                 n_leaves);
        if (cudaGetLastError() != cudaSuccess) return AMNERF_E_CUDA;
    }
    if (launch_scan(s, counts, n_leaves, kTileRows / 8, offsets, tile_off, cursor, stats) != cudaSuccess)
        return AMNERF_E_CUDA;
    if (blocks) {
        k_scatter_static<<<blocks, kThreads, 2 * sizeof(uint32_t) * n_leaves, s>>>(n_x, leaf, n_slots, maxc, cursor,
                                                                                   order, n_leaves);
        if (cudaGetLastError() != cudaSuccess) return AMNERF_E_CUDA;
    }
    return AMNERF_OK;
}
