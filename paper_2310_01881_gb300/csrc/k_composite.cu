// k_composite.cu -- K-d: per-ray front-to-back compositing (Sec. 3.1, "traditional
// volumetric rendering": the NeRF quadrature) with early ray termination.
//
// Definition, per ray over its samples in slot order: T = 1; stop once T < t_term;
// tau = sigma * delta, e = exp(-tau), alpha = 1 - e, w = T alpha; C += w c,
// D += w t, T = T e.  rgb = C + T bg, depth = D, opacity = 1 - T.
//
// Persistent warps take rays in a grid-stride loop (the next ray's crossing count is
// loaded while the current one is composited).  A warp handles a ray 32 SPL
// consecutive slots per pass, SPL per lane (1 for
// rays of at most 32 samples, else 2): the per-lane products of the factors e are
// combined by a warp-shuffle multiplicative scan, so each lane gets the
// transmittance in front of its samples (the carried T times the exclusive product,
// then times its earlier factors); samples whose transmittance is below t_term are
// dropped (a prefix, since the product only decreases), and the warp stops at the
// first pass that terminates.
// The sample position t and width delta are rebuilt from the crossing list in the
// same FP32 operation order as the traversal/sampling step (t at the stratum
// midpoint, or at the stratified jitter's fraction of it: jit_fraction).  Optionally (training
// targets of the proposal sampler) every composited weight is also added to the
// depth bin of its sample, and the residual transmittance is stored as bin 64.
#include <cuda_fp16.h>

#include "amnerf_internal.h"

namespace amnerf {
namespace {

constexpr int kWarpsPerBlock = 8;

struct RayAcc {
    float T, cr, cg, cb, dd;
    uint32_t composited;
};

// Slot s of the per-sample outputs: float4, or 4 x FP16 (sigma, r, g, b) when HALF.
template <bool HALF>
__device__ __forceinline__ float4 load_slot(const void* __restrict__ slot_out, size_t s) {
    if constexpr (HALF) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(slot_out) + s);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    } else {
        return __ldg(reinterpret_cast<const float4*>(slot_out) + s);
    }
}

// A slot as stored (uint2 = 4 x FP16, or float4), loaded with a volatile load: issued
// where it stands, so a thread's loads of whole crossings are in flight before the
// first of them is used; slot_value converts it.
template <bool HALF>
struct RawSlot {
    uint32_t a, b, c, d;  // HALF uses a, b
};

template <bool HALF>
__device__ __forceinline__ RawSlot<HALF> load_slot_now(const void* __restrict__ slot_out, size_t s) {
    RawSlot<HALF> r{0u, 0u, 0u, 0u};
    if constexpr (HALF) {
        asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];"
                     : "=r"(r.a), "=r"(r.b)
                     : "l"(reinterpret_cast<const uint2*>(slot_out) + s));
    } else {
        asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r.a), "=r"(r.b), "=r"(r.c), "=r"(r.d)
                     : "l"(reinterpret_cast<const float4*>(slot_out) + s));
    }
    return r;
}

// Slots s and s + 1 (s even: 16-byte aligned in the FP16 layout) with one 16-byte load.
__device__ __forceinline__ void load_slot_pair_now(const void* __restrict__ slot_out, size_t s, RawSlot<true>& r0,
                                                   RawSlot<true>& r1) {
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0.a), "=r"(r0.b), "=r"(r1.a), "=r"(r1.b)
                 : "l"(reinterpret_cast<const uint2*>(slot_out) + s));
}

// All kSteps slots of crossing k (slots k * kSteps ...): 16-byte loads.
template <bool HALF, int kSteps>
__device__ __forceinline__ void load_crossing_now(const void* __restrict__ slot_out, size_t first,
                                                  RawSlot<HALF> (&v)[kSteps]) {
    if constexpr (HALF) {
#pragma unroll
        for (int j = 0; j < kSteps; j += 2) load_slot_pair_now(slot_out, first + j, v[j], v[j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < kSteps; ++j) v[j] = load_slot_now<HALF>(slot_out, first + j);
    }
}

template <bool HALF>
__device__ __forceinline__ float4 slot_value(const RawSlot<HALF>& r) {
    if constexpr (HALF) {
        const float2 fa = __half22float2(*reinterpret_cast<const __half2*>(&r.a));
        const float2 fb = __half22float2(*reinterpret_cast<const __half2*>(&r.b));
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    } else {
        return make_float4(__uint_as_float(r.a), __uint_as_float(r.b), __uint_as_float(r.c), __uint_as_float(r.d));
    }
}

// One ray by one warp, SPL consecutive slots per lane (32 SPL slots per pass).
// Samples sit at fraction jit_fraction(jitter, key, k, steps, j) of their strata.
template <int SPL, bool HALF>
__device__ __forceinline__ void composite_ray(const float2* __restrict__ xing, const void* __restrict__ slot_out,
                                              int ns, int steps, int lg_steps, float inv_steps, size_t xbase,
                                              size_t sbase, uint64_t jitter, uint64_t key,
                                              float t_term, int lane, float r0, float bw, float* sbins, RayAcc& A) {
    for (int s0 = 0; s0 < ns; s0 += 32 * SPL) {
        float4 v[SPL];
        float e[SPL], t[SPL];
        bool val[SPL];
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
            const int s = s0 + SPL * lane + i;
            val[i] = s < ns;
            v[i] = val[i] ? load_slot<HALF>(slot_out, sbase + s) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
            e[i] = 1.0f;
            t[i] = 0.f;
            if (val[i]) {
                const int s = s0 + SPL * lane + i;
                const int k = s >> lg_steps;  // steps is a power of two
                const int j = s & (steps - 1);
                const float2 x = __ldg(xing + xbase + k);
                const float delta = __fmul_rn(__fsub_rn(x.y, x.x), inv_steps);
                const float u = jitter ? jit_fraction(jitter, key, k, steps, j) : 0.5f;
                t[i] = __fadd_rn(x.x, __fmul_rn(__fadd_rn((float)j, u), delta));
                e[i] = expf(-__fmul_rn(v[i].x, delta));
            }
        }
        // inclusive multiplicative scan of the per-lane products over the warp
        float p = e[0];
#pragma unroll
        for (int i = 1; i < SPL; ++i) p *= e[i];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xffffffffu, p, o);
            if (lane >= o) p = p * y;
        }
        float pex = __shfl_up_sync(0xffffffffu, p, 1);
        if (lane == 0) pex = 1.0f;
        float Tc = A.T * pex;  // transmittance in front of this lane's first slot
        float after = Tc;      // ... and behind its last composited slot
        bool prev = true;
        unsigned act_bits[SPL], val_bits[SPL];
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
            const bool act = val[i] && prev && !(Tc < t_term);
            if (act) {
                const float w = Tc * (1.0f - e[i]);
                A.cr += w * v[i].y;
                A.cg += w * v[i].z;
                A.cb += w * v[i].w;
                A.dd += w * t[i];
                if (sbins) {  // depth bin of the sample: floor((t - t0) / w), clamped to [0, 63]
                    int k = bw > 0.0f ? (int)floorf(__fdiv_rn(__fsub_rn(t[i], r0), bw)) : 0;
                    k = k < 0 ? 0 : (k > 63 ? 63 : k);
                    atomicAdd(&sbins[k], w);
                }
                after = Tc * e[i];
            }
            Tc = Tc * e[i];
            prev = act;
            act_bits[i] = __ballot_sync(0xffffffffu, act);
            val_bits[i] = __ballot_sync(0xffffffffu, val[i]);
        }
        bool term = false;
#pragma unroll
        for (int i = 0; i < SPL; ++i) {
            A.composited += __popc(act_bits[i]);
            term = term || act_bits[i] != val_bits[i];
        }
        if (term) {  // terminated inside this pass: T behind the last composited slot
            const int last = 31 - __clz(act_bits[0] | 1u);
            const float Tl = __shfl_sync(0xffffffffu, after, last);
            A.T = act_bits[0] ? Tl : A.T;
            break;
        }
        A.T = A.T * __shfl_sync(0xffffffffu, p, 31);
    }
}

template <bool HALF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 6) k_composite(
    const uint8_t* __restrict__ n_x, const float2* __restrict__ xing, const void* __restrict__ slot_out,
    uint32_t n, int steps, int maxc, int cap, float t_term, float bg0, float bg1, float bg2,
    float* __restrict__ rgb, float* __restrict__ depth, float* __restrict__ opacity,
    unsigned long long* __restrict__ n_comp, uint64_t jitter, const float* __restrict__ ro,
    const float* __restrict__ rd, const float2* __restrict__ root, float* __restrict__ bins) {
    __shared__ uint32_t s_comp[kWarpsPerBlock];
    __shared__ float s_bins[kWarpsPerBlock][65];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t stride = gridDim.x * kWarpsPerBlock;
    uint32_t composited = 0;
    const float inv_steps = 1.0f / (float)steps;  // exact: steps is a power of two
    const int lg = __ffs(steps) - 1;
    // each warp takes rays ray, ray + stride, ...; the next ray's crossing count is
    // loaded while the current ray is composited
    uint32_t ray = blockIdx.x * kWarpsPerBlock + wib;
    int nx_next = ray < n ? (int)__ldg(n_x + ray) : 0;
    for (; ray < n; ray += stride) {
        const int ns = nx_next * steps;
        const uint32_t ray2 = ray + stride;
        nx_next = ray2 < n ? (int)__ldg(n_x + ray2) : 0;
        float r0 = 0.f, bw = 0.f;
        if (bins) {
            __syncwarp();
            for (int b = lane; b < 65; b += 32) s_bins[wib][b] = 0.0f;
            const float2 rt = __ldg(root + ray);
            r0 = rt.x;
            bw = __fmul_rn(__fsub_rn(rt.y, rt.x), 0.015625f);
            __syncwarp();
        }
        const size_t xbase = (size_t)ray * maxc;
        const size_t sbase = (size_t)ray * cap;
        RayAcc A{1.0f, 0.f, 0.f, 0.f, 0.f, 0u};
        float* sb = bins ? s_bins[wib] : nullptr;
        uint64_t key = 0;
        if (jitter) {  // the ray's jitter key (the same loads in every lane)
            float o[3], d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = __ldg(ro + 3 * (size_t)ray + a);
                d[a] = __ldg(rd + 3 * (size_t)ray + a);
            }
            key = jit_ray_key(jitter, o, d);
        }
        // short rays: one slot per lane; longer ones: two (twice the bytes in flight)
        if (ns <= 32)
            composite_ray<1, HALF>(xing, slot_out, ns, steps, lg, inv_steps, xbase, sbase, jitter, key, t_term, lane,
                                   r0, bw, sb, A);
        else
            composite_ray<2, HALF>(xing, slot_out, ns, steps, lg, inv_steps, xbase, sbase, jitter, key, t_term, lane,
                                   r0, bw, sb, A);
        float T = A.T, cr = A.cr, cg = A.cg, cb = A.cb, dd = A.dd;
        composited += A.composited;
        // warp sums of (cr, cg, cb, dd) in 6 shuffles: each exchange halves the values a
        // lane carries until lanes 8i hold sum i (i = 0..3) after the last three steps;
        // three more bring them to lane 0
        const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
        const float s0 = __shfl_xor_sync(0xffffffffu, h16 ? cr : cb, 16);
        const float s1 = __shfl_xor_sync(0xffffffffu, h16 ? cg : dd, 16);
        const float w0 = (h16 ? cb : cr) + s0;  // cr | cb over lane pairs
        const float w1 = (h16 ? dd : cg) + s1;  // cg | dd
        float x = (h8 ? w1 : w0) + __shfl_xor_sync(0xffffffffu, h8 ? w0 : w1, 8);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (bins) {
            __syncwarp();
            if (lane == 0) s_bins[wib][64] = T;
            __syncwarp();
            for (int b = lane; b < 65; b += 32) bins[(size_t)ray * 65 + b] = s_bins[wib][b];
        }
        cr = x;
        cg = __shfl_sync(0xffffffffu, x, 8);
        cb = __shfl_sync(0xffffffffu, x, 16);
        dd = __shfl_sync(0xffffffffu, x, 24);
        if (lane == 0) {
            rgb[3 * (size_t)ray + 0] = cr + T * bg0;
            rgb[3 * (size_t)ray + 1] = cg + T * bg1;
            rgb[3 * (size_t)ray + 2] = cb + T * bg2;
            depth[ray] = dd;
            opacity[ray] = 1.0f - T;
        }
    }
    if (lane == 0) s_comp[wib] = composited;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int i = 0; i < kWarpsPerBlock; ++i) tot += s_comp[i];
        if (tot) atomicAdd(n_comp, tot);
    }
}

// One thread per ray, 8 samples per crossing (the workloads' setting): the thread
// composites its ray front to back in the definition's own order.  A crossing's 8
// slots are one aligned 128-byte row piece (64 bytes as FP16), all loaded before the
// crossing is composited, so every thread has a whole line in flight; the warp runs
// until its last ray ends or terminates.
// Waves (st_c != NULL): only crossings k_lo <= k < k_hi are composited.  A later wave
// resumes from the state (rgb and T in st_c, depth in st_d) of the rays still alive,
// and every wave stores the state, whether the ray goes on (alive), and the pixel;
// the operations and their order are those of one pass.
template <bool HALF, bool JIT>
__global__ void __launch_bounds__(256) k_composite_lane(
    const uint8_t* __restrict__ n_x, const float2* __restrict__ xing, const void* __restrict__ slot_out, uint32_t n,
    int maxc, int cap, float t_term, float bg0, float bg1, float bg2, float* __restrict__ rgb,
    float* __restrict__ depth, float* __restrict__ opacity, unsigned long long* __restrict__ n_comp,
    uint64_t jitter, const float* __restrict__ ro, const float* __restrict__ rd, int k_lo, int k_hi,
    float4* __restrict__ st_c, float* __restrict__ st_d, uint8_t* __restrict__ alive_io,
    uint32_t* __restrict__ next_ray) {
    constexpr int kSteps = 8;
    uint32_t comp = 0;
    const bool pers = next_ray != nullptr;
    const uint32_t ctr = (threadIdx.x >> 5) % kRayCounters;  // this warp's counter
    while (true) {
    uint32_t ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (pers) {  // the next 32-ray block b of this warp's counter (b % kRayCounters == ctr)
        uint32_t v = 0;
        if ((threadIdx.x & 31) == 0) v = atomicAdd(next_ray + 32 * ctr, 1u);
        v = __shfl_sync(0xffffffffu, v, 0);
        const uint64_t r0 = ((uint64_t)v * kRayCounters + ctr) * 32u;
        if (r0 >= n) break;
        ray = (uint32_t)r0 + (threadIdx.x & 31);
    }
    // a ray that ended in an earlier wave keeps its pixel
    if (ray < n && (!st_c || k_lo == 0 || alive_io[ray])) {
        float T = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f;
        if (st_c && k_lo > 0) {
            const float4 c = st_c[ray];
            cr = c.x;
            cg = c.y;
            cb = c.z;
            T = c.w;
            dd = st_d[ray];
        }
        const int nx_all = (int)__ldg(n_x + ray);
        const int nx = nx_all < k_hi ? nx_all : k_hi;
        uint64_t key = 0;
        if constexpr (JIT) {  // the ray's jitter key
            float o[3], d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = __ldg(ro + 3 * (size_t)ray + a);
                d[a] = __ldg(rd + 3 * (size_t)ray + a);
            }
            key = jit_ray_key(jitter, o, d);
        }
        const float2* xr = xing + (size_t)ray * maxc;
        const size_t row = (size_t)ray * cap;
        bool alive = true;
        // crossing k + 1's slots are loaded while crossing k is composited
        RawSlot<HALF> vn[kSteps];
        if (k_lo < nx) load_crossing_now<HALF, kSteps>(slot_out, row + (size_t)(k_lo * kSteps), vn);
        for (int k = k_lo; k < nx && alive; ++k) {
            const float2 x = __ldg(xr + k);
            RawSlot<HALF> v[kSteps];
#pragma unroll
            for (int j = 0; j < kSteps; ++j) v[j] = vn[j];
            if (k + 1 < nx) load_crossing_now<HALF, kSteps>(slot_out, row + (size_t)((k + 1) * kSteps), vn);
            // same FP32 operations as the sampling step: delta = (t_out - t_in) / steps
            // (exact: a power of two), t_j = t_in + (j + 1/2) delta
            const float delta = __fmul_rn(__fsub_rn(x.y, x.x), 1.0f / kSteps);
#pragma unroll
            for (int j = 0; j < kSteps; ++j) {
                alive = alive && !(T < t_term);  // stop once T < t_term
                if (alive) {
                    const float4 vj = slot_value<HALF>(v[j]);
                    const float u = JIT ? jit_fraction(jitter, key, k, kSteps, j) : 0.5f;
                    const float t = __fadd_rn(x.x, __fmul_rn(__fadd_rn((float)j, u), delta));
                    const float e = expf(-__fmul_rn(vj.x, delta));
                    const float w = T * (1.0f - e);
                    cr += w * vj.y;
                    cg += w * vj.z;
                    cb += w * vj.w;
                    dd += w * t;
                    T = T * e;
                    ++comp;
                }
            }
        }
        rgb[3 * (size_t)ray + 0] = cr + T * bg0;
        rgb[3 * (size_t)ray + 1] = cg + T * bg1;
        rgb[3 * (size_t)ray + 2] = cb + T * bg2;
        depth[ray] = dd;
        opacity[ray] = 1.0f - T;
        if (st_c) {
            st_c[ray] = make_float4(cr, cg, cb, T);
            st_d[ray] = dd;
            alive_io[ray] = (!(T < t_term) && nx < nx_all) ? 1 : 0;
        }
    }
    if (!pers) break;
    }
    // composited samples: warp sums, one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) comp += __shfl_xor_sync(0xffffffffu, comp, o);
    if ((threadIdx.x & 31) == 0 && comp) atomicAdd(n_comp, (unsigned long long)comp);
}

// Debug view: generated slots (j < n_x[r] * steps) of 4 x FP16 outputs as float4.
__global__ void k_slots_to_f32(const uint8_t* __restrict__ n_x, const void* __restrict__ slot_half,
                               float4* __restrict__ out, uint32_t n, int steps, int cap) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n * cap) return;
    const uint32_t r = (uint32_t)(i / (size_t)cap);
    const int j = (int)(i - (size_t)r * cap);
    if (j < (int)n_x[r] * steps) out[i] = load_slot<true>(slot_half, i);
}

}  // namespace

cudaError_t launch_composite(cudaStream_t s, const uint8_t* n_x, const float2* xing, const void* slot_out,
                             int slot_half, uint32_t n, int steps, int maxc, int cap, float t_term, float bg0,
                             float bg1, float bg2, float* rgb, float* depth, float* opacity, uint64_t* stats,
                             uint64_t jitter, const float* ro, const float* rd, const float2* root, float* bins,
                             int k_lo, int k_hi, float4* st_c, float* st_d, uint8_t* alive,
                             uint32_t* ray_counters) {
    if (n == 0) return cudaSuccess;
    if (st_c && (bins || steps != 8)) return cudaErrorInvalidValue;  // waves: the per-ray kernel only
    if (!bins && steps == 8) {  // one thread per ray
        auto* stc = reinterpret_cast<unsigned long long*>(stats + 2);
        unsigned lb = (n + 255) / 256;
        // one pass: persistent CTAs, each warp taking its rays 32 at a time from one of the
        // ray counters (zeroed at the start of the render), so a CTA waits for its slowest
        // ray once; waves keep one CTA per 256 rays
        uint32_t* next = st_c ? nullptr : ray_counters;
        if (next) {
            static int cap_lane[64] = {0};
            int dev = 0;
            if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
                if (!cap_lane[dev]) {
                    int sms = 0, per = 0;
                    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_composite_lane<true, true>, 256, 0);
                    cap_lane[dev] = sms * (per > 0 ? per : 1);
                }
                if (lb > (unsigned)cap_lane[dev]) lb = (unsigned)cap_lane[dev];
            }
        }
#define AMNERF_LANE(H, J)                                                                                        \
    k_composite_lane<H, J><<<lb, 256, 0, s>>>(n_x, xing, slot_out, n, maxc, cap, t_term, bg0, bg1, bg2, rgb, depth, \
                                              opacity, stc, jitter, ro, rd, k_lo, k_hi, st_c, st_d, alive, next)
        if (slot_half) {
            if (jitter) AMNERF_LANE(true, true);
            else AMNERF_LANE(true, false);
        } else {
            if (jitter) AMNERF_LANE(false, true);
            else AMNERF_LANE(false, false);
        }
#undef AMNERF_LANE
        return cudaGetLastError();
    }
    unsigned blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
    // resident CTAs per device, cached: only a cap on the launch size (any grid gives
    // the same result, the warps stride over the rays)
    static int cap_blocks[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        if (!cap_blocks[dev]) {
            int sms = 0, per = 0, per_h = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_composite<false>, kWarpsPerBlock * 32, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_h, k_composite<true>, kWarpsPerBlock * 32, 0);
            per = per_h > 0 && per_h < per ? per_h : per;
            cap_blocks[dev] = sms * (per > 0 ? per : 1);
        }
        if (cap_blocks[dev] > 0 && blocks > (unsigned)cap_blocks[dev]) blocks = (unsigned)cap_blocks[dev];
    }
    auto* st = reinterpret_cast<unsigned long long*>(stats + 2);
    if (slot_half)
        k_composite<true><<<blocks, kWarpsPerBlock * 32, 0, s>>>(n_x, xing, slot_out, n, steps, maxc, cap, t_term, bg0,
                                                                 bg1, bg2, rgb, depth, opacity, st, jitter, ro, rd,
                                                                 root, bins);
    else
        k_composite<false><<<blocks, kWarpsPerBlock * 32, 0, s>>>(n_x, xing, slot_out, n, steps, maxc, cap, t_term,
                                                                  bg0, bg1, bg2, rgb, depth, opacity, st, jitter, ro,
                                                                  rd, root, bins);
    return cudaGetLastError();
}

cudaError_t launch_slots_to_f32(cudaStream_t s, const uint8_t* n_x, const void* slot_half, float4* out, uint32_t n,
                                int steps, int cap) {
    const size_t total = (size_t)n * cap;
    if (total == 0) return cudaSuccess;
    k_slots_to_f32<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n_x, slot_half, out, n, steps, cap);
    return cudaGetLastError();
}

}  // namespace amnerf
