// k_group.cu -- K-b: group crossings by leaf (Sec. 3.5 and Fig. "parallel": samples
// are sorted by node id so that every node's network runs as one dense batch).
//
// The keys are small integers (network ids < 8192: leaves, and inner nodes with
// adaptive hierarchical sampling), so the sort is a one-digit counting sort.  Per-leaf
// totals come from K-a's histogram; one CTA scans them into crossing offsets and
// network-tile offsets (a tile holds 128 / steps crossings of one leaf).
// The scatter stages its binning in shared memory: each CTA ranks its crossings per
// leaf with shared atomics, reserves one contiguous range per touched leaf with a
// single global atomic, then writes every crossing id into its leaf's segment.  Up to
// 32 crossings per ray, a thread takes one ray and reads only its ids; beyond, a
// thread takes 16 slots of the crossing list.
// Counts and offsets are exact; the order inside a segment is not specified (the
// network result of a sample does not depend on its position in the batch).
#include "amnerf_internal.h"

namespace amnerf {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanPer = kMaxNets / kScanThreads;  // 8 networks per thread

__global__ void __launch_bounds__(kScanThreads) k_scan(const uint32_t* __restrict__ counts, int n_leaves, int cpt,
                                                       uint32_t* __restrict__ offsets,
                                                       uint32_t* __restrict__ tile_off,
                                                       uint32_t* __restrict__ cursor, uint64_t* __restrict__ stats,
                                                       uint64_t* __restrict__ acc) {
    __shared__ uint32_t s_c[32], s_t[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t c[kScanPer], t[kScanPer];
    uint32_t sc = 0, st = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        const int i = tid * kScanPer + j;
        c[j] = i < n_leaves ? counts[i] : 0u;
        t[j] = (c[j] + (uint32_t)cpt - 1u) / (uint32_t)cpt;
        sc += c[j];
        st += t[j];
    }
    // inclusive warp scan of the per-thread sums
    uint32_t ic = sc, it = st;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yc = __shfl_up_sync(0xffffffffu, ic, o);
        const uint32_t yt = __shfl_up_sync(0xffffffffu, it, o);
        if (lane >= o) {
            ic += yc;
            it += yt;
        }
    }
    if (lane == 31) {
        s_c[warp] = ic;
        s_t[warp] = it;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t wc = s_c[lane], wt = s_t[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yc = __shfl_up_sync(0xffffffffu, wc, o);
            const uint32_t yt = __shfl_up_sync(0xffffffffu, wt, o);
            if (lane >= o) {
                wc += yc;
                wt += yt;
            }
        }
        s_c[lane] = wc;  // inclusive over warps
        s_t[lane] = wt;
    }
    __syncthreads();
    uint32_t rc = (warp ? s_c[warp - 1] : 0u) + ic - sc;  // exclusive start of this thread
    uint32_t rt = (warp ? s_t[warp - 1] : 0u) + it - st;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        const int i = tid * kScanPer + j;
        if (i < n_leaves) {
            offsets[i] = rc;
            cursor[i] = rc;
            tile_off[i] = rt;
        }
        rc += c[j];
        rt += t[j];
    }
    if (tid == kScanThreads - 1) {
        offsets[n_leaves] = rc;
        tile_off[n_leaves] = rt;
        stats[0] = rc;  // crossings
        stats[1] = rt;  // tiles
        if (acc) {      // running totals over the waves of one render
            acc[0] += rc;
            acc[1] += rt;
        }
    }
}

constexpr int kScatterThreads = 256;
constexpr int kScatterItems = 16;

__global__ void __launch_bounds__(kScatterThreads) k_scatter(const uint8_t* __restrict__ n_x,
                                                             const uint16_t* __restrict__ xleaf, uint32_t n_slots,
                                                             int maxc, uint32_t* __restrict__ cursor,
                                                             uint32_t* __restrict__ order, int n_leaves) {
    extern __shared__ uint32_t sm[];
    uint32_t* s_cnt = sm;
    uint32_t* s_base = sm + n_leaves;
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();
    const uint32_t base = blockIdx.x * (uint32_t)(kScatterThreads * kScatterItems);
    // s / maxc as a multiply-high: with m = ceil(2^32 / maxc), q = floor(s m / 2^32) is
    // the quotient or one more (s m / 2^32 < s / maxc + 1), which one compare fixes
    const uint32_t m = maxc > 1 ? (uint32_t)(((1ull << 32) + (uint64_t)maxc - 1ull) / (uint64_t)maxc) : 0u;
    auto ray_of = [&](uint32_t s) -> uint32_t {
        if (maxc == 1) return s;
        uint32_t q = __umulhi(s, m);
        if ((uint64_t)q * (uint32_t)maxc > s) --q;
        return q;
    };
    uint16_t lf[kScatterItems];
    uint32_t rk[kScatterItems];
    uint8_t nx[kScatterItems];
    // all loads first (the slot's leaf is read whether or not the slot holds a crossing;
    // slots past a ray's count are ignored)
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
        const uint32_t s = base + (uint32_t)(i * kScatterThreads) + threadIdx.x;
        lf[i] = 0;
        nx[i] = 0;
        if (s < n_slots) {
            const uint32_t ray = ray_of(s);
            nx[i] = __ldg(n_x + ray);
            lf[i] = __ldg(xleaf + s);
        }
    }
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
        const uint32_t s = base + (uint32_t)(i * kScatterThreads) + threadIdx.x;
        rk[i] = 0xffffffffu;
        if (s < n_slots) {
            const uint32_t ray = ray_of(s);
            const uint32_t k = s - ray * (uint32_t)maxc;
            if (k < (uint32_t)nx[i]) rk[i] = atomicAdd(&s_cnt[lf[i]], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) {
        const uint32_t c = s_cnt[i];
        s_base[i] = c ? atomicAdd(&cursor[i], c) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
        if (rk[i] != 0xffffffffu) {
            const uint32_t s = base + (uint32_t)(i * kScatterThreads) + threadIdx.x;
            order[s_base[lf[i]] + rk[i]] = s;
        }
    }
}

// The same binning with one thread per ray (maxc <= kRayScatterMaxc): a thread reads
// only its own ray's network ids (16 bytes at a time when maxc is a multiple of 8)
// instead of every slot of the crossing list, ranks them with shared atomics (ranks
// and ids kept in shared memory as [slot][thread]), and after the CTA's one global
// atomic per touched leaf writes the crossing ids into their segments.
constexpr int kRayScatterThreads = 256;
constexpr int kRayScatterMaxc = 32;

// Rank of this lane's crossing among the CTA's crossings of network id: the lanes of
// the warp now at the same id (neighbouring rays usually cross the same leaves) take
// one shared atomic together and are ranked by lane.
__device__ __forceinline__ uint32_t warp_rank(uint32_t* s_cnt, uint32_t id) {
    const uint32_t act = __activemask();
    const uint32_t peers = __match_any_sync(act, id);
    const int leader = __ffs(peers) - 1;
    const int lane = (int)(threadIdx.x & 31);
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&s_cnt[id], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

template <bool VEC>
__global__ void __launch_bounds__(kRayScatterThreads) k_scatter_rays(const uint8_t* __restrict__ n_x,
                                                                     const uint16_t* __restrict__ xleaf,
                                                                     uint32_t n_rays, int maxc,
                                                                     uint32_t* __restrict__ cursor,
                                                                     uint32_t* __restrict__ order, int n_leaves) {
    extern __shared__ uint32_t sm[];
    uint32_t* s_cnt = sm;
    uint32_t* s_base = sm + n_leaves;
    uint16_t* s_id = reinterpret_cast<uint16_t*>(sm + 2 * n_leaves) + threadIdx.x;
    uint16_t* s_rk = s_id + (size_t)maxc * kRayScatterThreads;
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();
    const uint32_t r = blockIdx.x * (uint32_t)kRayScatterThreads + threadIdx.x;
    const int nx = r < n_rays ? min((int)__ldg(n_x + r), maxc) : 0;
    const size_t base = (size_t)r * (size_t)maxc;
    if (VEC) {
        for (int k0 = 0; k0 < nx; k0 += 8) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(xleaf + base + k0));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = k0 + i;
                if (k < nx) {
                    const uint32_t id = (w[i >> 1] >> (16 * (i & 1))) & 0xffffu;
                    s_id[k * kRayScatterThreads] = (uint16_t)id;
                    s_rk[k * kRayScatterThreads] = (uint16_t)warp_rank(s_cnt, id);
                }
            }
        }
    } else {
        for (int k = 0; k < nx; ++k) {
            const uint32_t id = __ldg(xleaf + base + k);
            s_id[k * kRayScatterThreads] = (uint16_t)id;
            s_rk[k * kRayScatterThreads] = (uint16_t)warp_rank(s_cnt, id);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) {
        const uint32_t c = s_cnt[i];
        s_base[i] = c ? atomicAdd(&cursor[i], c) : 0u;
    }
    __syncthreads();
    for (int k = 0; k < nx; ++k) {
        const uint32_t id = s_id[k * kRayScatterThreads];
        order[s_base[id] + s_rk[k * kRayScatterThreads]] = (uint32_t)(base + (size_t)k);
    }
}

// One wave of a render: crossings k_lo <= k < min(n_x, k_lo + W) of the rays still
// alive (alive == NULL: every ray), visited as n_rays x W items (ray-major), so a wave
// reads only its own slots.  COUNT: only the per-leaf totals (added to cursor, which
// then holds counts) for the scan; else the same binning as k_scatter.
template <bool COUNT>
__global__ void __launch_bounds__(kScatterThreads) k_scatter_wave(const uint8_t* __restrict__ n_x,
                                                                  const uint16_t* __restrict__ xleaf,
                                                                  uint32_t n_items, int maxc, int k_lo, int W,
                                                                  const uint8_t* __restrict__ alive,
                                                                  uint32_t* __restrict__ cursor,
                                                                  uint32_t* __restrict__ order, int n_leaves) {
    extern __shared__ uint32_t sm[];
    uint32_t* s_cnt = sm;
    uint32_t* s_base = sm + n_leaves;
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();
    const uint32_t base = blockIdx.x * (uint32_t)(kScatterThreads * kScatterItems);
    uint16_t lf[kScatterItems];
    uint32_t rk[kScatterItems], sl[kScatterItems];
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
        const uint32_t it = base + (uint32_t)(i * kScatterThreads) + threadIdx.x;
        lf[i] = 0;
        sl[i] = 0xffffffffu;
        if (it < n_items) {
            const uint32_t ray = it / (uint32_t)W;
            const uint32_t k = (uint32_t)k_lo + (it - ray * (uint32_t)W);
            if ((!alive || __ldg(alive + ray)) && k < (uint32_t)__ldg(n_x + ray)) {
                sl[i] = ray * (uint32_t)maxc + k;
                lf[i] = __ldg(xleaf + sl[i]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) rk[i] = sl[i] != 0xffffffffu ? atomicAdd(&s_cnt[lf[i]], 1u) : 0xffffffffu;
    __syncthreads();
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) {
        const uint32_t c = s_cnt[i];
        s_base[i] = c ? atomicAdd(&cursor[i], c) : 0u;
    }
    if (COUNT) return;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i)
        if (rk[i] != 0xffffffffu) order[s_base[lf[i]] + rk[i]] = sl[i];
}

}  // namespace

cudaError_t launch_scan(cudaStream_t s, const uint32_t* counts, int n_leaves, int cpt, uint32_t* offsets,
                        uint32_t* tile_off, uint32_t* cursor, uint64_t* stats, uint64_t* acc) {
    k_scan<<<1, kScanThreads, 0, s>>>(counts, n_leaves, cpt, offsets, tile_off, cursor, stats, acc);
    return cudaGetLastError();
}

cudaError_t launch_scatter(cudaStream_t s, const uint8_t* n_x, const uint16_t* xleaf, uint32_t n_rays, int maxc,
                           uint32_t* cursor, uint32_t* order, int n_leaves) {
    const uint64_t n_slots = (uint64_t)n_rays * (uint64_t)maxc;
    if (n_slots == 0) return cudaSuccess;
    if (maxc <= kRayScatterMaxc) {
        const unsigned blocks = (n_rays + kRayScatterThreads - 1) / kRayScatterThreads;
        const size_t smem = 2 * sizeof(uint32_t) * (size_t)n_leaves +
                            2 * sizeof(uint16_t) * (size_t)maxc * kRayScatterThreads;
        if ((maxc & 7) == 0)
            k_scatter_rays<true><<<blocks, kRayScatterThreads, smem, s>>>(n_x, xleaf, n_rays, maxc, cursor, order,
                                                                          n_leaves);
        else
            k_scatter_rays<false><<<blocks, kRayScatterThreads, smem, s>>>(n_x, xleaf, n_rays, maxc, cursor, order,
                                                                           n_leaves);
        return cudaGetLastError();
    }
    const uint64_t per = (uint64_t)kScatterThreads * kScatterItems;
    const unsigned blocks = (unsigned)((n_slots + per - 1) / per);
    const size_t smem = 2 * sizeof(uint32_t) * (size_t)n_leaves;
    k_scatter<<<blocks, kScatterThreads, smem, s>>>(n_x, xleaf, (uint32_t)n_slots, maxc, cursor, order, n_leaves);
    return cudaGetLastError();
}

cudaError_t launch_scatter_wave(cudaStream_t s, bool count, const uint8_t* n_x, const uint16_t* xleaf,
                                uint32_t n_rays, int maxc, int k_lo, int k_hi, const uint8_t* alive, uint32_t* cursor,
                                uint32_t* order, int n_leaves) {
    const int W = k_hi - k_lo;
    const uint64_t n_items = (uint64_t)n_rays * (uint64_t)W;
    if (n_items == 0 || W <= 0) return cudaSuccess;
    const uint64_t per = (uint64_t)kScatterThreads * kScatterItems;
    const unsigned blocks = (unsigned)((n_items + per - 1) / per);
    const size_t smem = 2 * sizeof(uint32_t) * (size_t)n_leaves;
    if (count)
        k_scatter_wave<true><<<blocks, kScatterThreads, smem, s>>>(n_x, xleaf, (uint32_t)n_items, maxc, k_lo, W, alive,
                                                                   cursor, order, n_leaves);
    else
        k_scatter_wave<false><<<blocks, kScatterThreads, smem, s>>>(n_x, xleaf, (uint32_t)n_items, maxc, k_lo, W,
                                                                    alive, cursor, order, n_leaves);
    return cudaGetLastError();
}

namespace {

// Crossings given by the caller (render from crossings): per ray r, n_x[r] <= maxc
// crossings k with network leaf[r maxc + k] and interval (t_in, t_out).  Copies them
// into the render's crossing list and counts them per network (shared-memory
// histogram, one atomic per touched network per CTA).  A network id >= n_nets or a
// count above maxc is recorded in the error word and replaced by 0 / maxc, so later
// stages stay in bounds.
__global__ void __launch_bounds__(256) k_load_crossings(const uint8_t* __restrict__ n_x_in,
                                                        const uint16_t* __restrict__ leaf_in,
                                                        const float* __restrict__ t_in, const float* __restrict__ t_out,
                                                        uint32_t n_rays, int maxc, int n_nets,
                                                        uint8_t* __restrict__ n_x, float2* __restrict__ xing,
                                                        uint16_t* __restrict__ xleaf, uint32_t* __restrict__ counts,
                                                        int* __restrict__ err) {
    extern __shared__ uint32_t s_cnt[];
    for (int i = threadIdx.x; i < n_nets; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_rays) {
        int c = __ldg(n_x_in + r);
        if (c > maxc) {
            atomicCAS(err, 0, kDevErrBounds);
            c = maxc;
        }
        n_x[r] = (uint8_t)c;
        const size_t base = (size_t)r * (size_t)maxc;
        for (int k = 0; k < c; ++k) {
            uint32_t l = __ldg(leaf_in + base + k);
            if (l >= (uint32_t)n_nets) {
                atomicCAS(err, 0, kDevErrBounds);
                l = 0u;
            }
            xleaf[base + k] = (uint16_t)l;
            xing[base + k] = make_float2(__ldg(t_in + base + k), __ldg(t_out + base + k));
            atomicAdd(&s_cnt[l], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_nets; i += blockDim.x) {
        const uint32_t c = s_cnt[i];
        if (c) atomicAdd(&counts[i], c);
    }
}

}  // namespace

cudaError_t launch_load_crossings(cudaStream_t s, const uint8_t* n_x_in, const uint16_t* leaf_in, const float* t_in,
                                  const float* t_out, uint32_t n_rays, int maxc, int n_nets, uint8_t* n_x,
                                  float2* xing, uint16_t* xleaf, uint32_t* counts, int* err) {
    if (n_rays == 0) return cudaSuccess;
    const unsigned blocks = (n_rays + 255) / 256;
    k_load_crossings<<<blocks, 256, sizeof(uint32_t) * (size_t)n_nets, s>>>(n_x_in, leaf_in, t_in, t_out, n_rays, maxc,
                                                                           n_nets, n_x, xing, xleaf, counts, err);
    return cudaGetLastError();
}

cudaError_t prepare_group() {
    // two counters per network: up to 64 KB of dynamic shared memory
    const int smem = (int)(2 * sizeof(uint32_t) * kMaxNets);
    cudaError_t e = cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_scatter_wave<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_scatter_wave<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    // the per-ray scatter also keeps each thread's ids and ranks
    const int smem_r = smem + (int)(2 * sizeof(uint16_t) * kRayScatterMaxc * kRayScatterThreads);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_scatter_rays<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_r);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_scatter_rays<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_r);
    return e;
}

}  // namespace amnerf
