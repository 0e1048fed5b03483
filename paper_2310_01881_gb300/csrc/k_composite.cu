// k_composite.cu -- K-d: per-ray front-to-back compositing (Sec. 3.1, "traditional
// volumetric rendering": the NeRF quadrature) with early ray termination.
//
// Definition, per ray over its samples in slot order: T = 1; stop once T < t_term;
// tau = sigma * delta, e = exp(-tau), alpha = 1 - e, w = T alpha; C += w c,
// D += w t, T = T e.  rgb = C + T bg, depth = D, opacity = 1 - T.
//
// One warp per ray handles 64 consecutive slots per pass, two per lane: the per-lane
// products of the factors e are combined by a warp-shuffle multiplicative scan, so
// each lane gets the transmittance in front of its two samples (the carried T times
// the exclusive product, then times its first factor); samples whose transmittance
// is below t_term are dropped (a prefix, since the product only decreases), and the
// warp stops at the first pass that terminates.
// The sample position t and width delta are rebuilt from the crossing list in the
// same FP32 operation order as the traversal/sampling step.  Optionally (training
// targets of the proposal sampler) every composited weight is also added to the
// depth bin of its sample, and the residual transmittance is stored as bin 64.
#include "amnerf_internal.h"

namespace amnerf {
namespace {

constexpr int kWarpsPerBlock = 8;

__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_composite(
    const uint8_t* __restrict__ n_x, const float2* __restrict__ xing, const float4* __restrict__ slot_out,
    uint32_t n, int steps, int maxc, int cap, float t_term, float bg0, float bg1, float bg2,
    float* __restrict__ rgb, float* __restrict__ depth, float* __restrict__ opacity,
    unsigned long long* __restrict__ n_comp, const float2* __restrict__ root, float* __restrict__ bins) {
    __shared__ uint32_t s_comp[kWarpsPerBlock];
    __shared__ float s_bins[kWarpsPerBlock][65];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t ray = blockIdx.x * kWarpsPerBlock + wib;
    uint32_t composited = 0;
    float r0 = 0.f, bw = 0.f;
    if (bins) {
        for (int b = lane; b < 65; b += 32) s_bins[wib][b] = 0.0f;
        if (ray < n) {
            const float2 rt = __ldg(root + ray);
            r0 = rt.x;
            bw = __fmul_rn(__fsub_rn(rt.y, rt.x), 0.015625f);
        }
        __syncwarp();
    }
    if (ray < n) {
        const int ns = (int)__ldg(n_x + ray) * steps;
        const float inv_steps = 1.0f / (float)steps;  // exact: steps is a power of two
        const size_t xbase = (size_t)ray * maxc;
        const size_t sbase = (size_t)ray * cap;
        float T = 1.0f;
        float cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f;
        // 64 slots per pass, two consecutive slots per lane (one 32-byte load each)
        for (int s0 = 0; s0 < ns; s0 += 64) {
            const int sa = s0 + 2 * lane, sb = sa + 1;
            const bool va = sa < ns, vb = sb < ns;
            float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
            if (va) v0 = __ldg(slot_out + sbase + sa);
            if (vb) v1 = __ldg(slot_out + sbase + sb);
            float e0 = 1.0f, e1 = 1.0f, t0 = 0.f, t1 = 0.f;
            if (va) {
                const int k = sa / steps;
                const int j = sa - k * steps;
                const float2 x = __ldg(xing + xbase + k);
                const float delta = __fmul_rn(__fsub_rn(x.y, x.x), inv_steps);
                t0 = __fadd_rn(x.x, __fmul_rn((float)j + 0.5f, delta));
                e0 = expf(-__fmul_rn(v0.x, delta));
            }
            if (vb) {
                const int k = sb / steps;
                const int j = sb - k * steps;
                const float2 x = __ldg(xing + xbase + k);
                const float delta = __fmul_rn(__fsub_rn(x.y, x.x), inv_steps);
                t1 = __fadd_rn(x.x, __fmul_rn((float)j + 0.5f, delta));
                e1 = expf(-__fmul_rn(v1.x, delta));
            }
            // inclusive multiplicative scan of the per-lane products e0 e1 over the warp
            float p = e0 * e1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p = p * y;
            }
            float pex = __shfl_up_sync(0xffffffffu, p, 1);
            if (lane == 0) pex = 1.0f;
            const float Ta = T * pex;  // transmittance in front of slot sa
            const float Tb = Ta * e0;  // ... and of slot sb
            const bool aa = va && !(Ta < t_term);
            const bool ab = vb && aa && !(Tb < t_term);
            if (aa) {
                const float w = Ta * (1.0f - e0);
                cr += w * v0.y;
                cg += w * v0.z;
                cb += w * v0.w;
                dd += w * t0;
                if (bins) {  // depth bin of the sample: floor((t - t0) / w), clamped to [0, 63]
                    int k = bw > 0.0f ? (int)floorf(__fdiv_rn(__fsub_rn(t0, r0), bw)) : 0;
                    k = k < 0 ? 0 : (k > 63 ? 63 : k);
                    atomicAdd(&s_bins[wib][k], w);
                }
            }
            if (ab) {
                const float w = Tb * (1.0f - e1);
                cr += w * v1.y;
                cg += w * v1.z;
                cb += w * v1.w;
                dd += w * t1;
                if (bins) {
                    int k = bw > 0.0f ? (int)floorf(__fdiv_rn(__fsub_rn(t1, r0), bw)) : 0;
                    k = k < 0 ? 0 : (k > 63 ? 63 : k);
                    atomicAdd(&s_bins[wib][k], w);
                }
            }
            const unsigned act_a = __ballot_sync(0xffffffffu, aa), act_b = __ballot_sync(0xffffffffu, ab);
            const unsigned val_a = __ballot_sync(0xffffffffu, va), val_b = __ballot_sync(0xffffffffu, vb);
            composited += __popc(act_a) + __popc(act_b);
            if (act_a != val_a || act_b != val_b) {  // terminated inside this pass
                // transmittance behind the last composited slot
                const float after = ab ? Tb * e1 : Ta * e0;
                const int last = 31 - __clz(act_a | 1u);
                const float Tl = __shfl_sync(0xffffffffu, after, last);
                T = act_a ? Tl : T;
                break;
            }
            T = T * __shfl_sync(0xffffffffu, p, 31);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cr += __shfl_xor_sync(0xffffffffu, cr, o);
            cg += __shfl_xor_sync(0xffffffffu, cg, o);
            cb += __shfl_xor_sync(0xffffffffu, cb, o);
            dd += __shfl_xor_sync(0xffffffffu, dd, o);
        }
        if (bins) {
            __syncwarp();
            if (lane == 0) s_bins[wib][64] = T;
            __syncwarp();
            for (int b = lane; b < 65; b += 32) bins[(size_t)ray * 65 + b] = s_bins[wib][b];
        }
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

}  // namespace

cudaError_t launch_composite(cudaStream_t s, const uint8_t* n_x, const float2* xing, const float4* slot_out,
                             uint32_t n, int steps, int maxc, int cap, float t_term, float bg0, float bg1,
                             float bg2, float* rgb, float* depth, float* opacity, uint64_t* stats,
                             const float2* root, float* bins) {
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
    k_composite<<<blocks, kWarpsPerBlock * 32, 0, s>>>(n_x, xing, slot_out, n, steps, maxc, cap, t_term, bg0, bg1,
                                                       bg2, rgb, depth, opacity,
                                                       reinterpret_cast<unsigned long long*>(stats + 2), root, bins);
    return cudaGetLastError();
}

}  // namespace amnerf
