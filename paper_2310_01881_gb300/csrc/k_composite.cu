// k_composite.cu -- K-d: per-ray front-to-back compositing (Sec. 3.1, "traditional
// volumetric rendering": the NeRF quadrature) with early ray termination.
//
// Definition, per ray over its samples in slot order: T = 1; stop once T < t_term;
// tau = sigma * delta, e = exp(-tau), alpha = 1 - e, w = T alpha; C += w c,
// D += w t, T = T e.  rgb = C + T bg, depth = D, opacity = 1 - T.
//
// One warp per ray handles 32 consecutive slots at a time: the per-sample factors e
// are combined by a warp-shuffle multiplicative scan, so lane i gets the
// transmittance in front of its sample (the carried T times the exclusive product);
// lanes whose transmittance is below t_term are dropped (a prefix, since the
// product only decreases), and the warp stops at the first chunk that terminates.
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
        // the next chunk's slot and crossing are loaded before this chunk is scanned
        float4 vn = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 xn = make_float2(0.f, 0.f);
        if (lane < ns) {
            vn = __ldg(slot_out + sbase + lane);
            xn = __ldg(xing + xbase + lane / steps);
        }
        for (int s0 = 0; s0 < ns; s0 += 32) {
            const int s = s0 + lane;
            const bool valid = s < ns;
            float e = 1.0f, sig = 0.f, t = 0.f;
            const float4 v = vn;
            const float2 x = xn;
            if (s + 32 < ns) {
                vn = __ldg(slot_out + sbase + s + 32);
                xn = __ldg(xing + xbase + (s + 32) / steps);
            }
            if (valid) {
                const int k = s / steps;
                const int j = s - k * steps;
                const float delta = __fmul_rn(__fsub_rn(x.y, x.x), inv_steps);
                t = __fadd_rn(x.x, __fmul_rn((float)j + 0.5f, delta));
                sig = __fmul_rn(v.x, delta);
                e = expf(-sig);
            }
            // inclusive multiplicative scan of e over the warp
            float p = e;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p = p * y;
            }
            float pex = __shfl_up_sync(0xffffffffu, p, 1);
            if (lane == 0) pex = 1.0f;
            const float Tb = T * pex;          // transmittance in front of this sample
            const bool active = valid && !(Tb < t_term);
            if (active) {
                const float w = Tb * (1.0f - e);
                cr += w * v.y;
                cg += w * v.z;
                cb += w * v.w;
                dd += w * t;
                if (bins) {  // depth bin of the sample: floor((t - t0) / w), clamped to [0, 63]
                    int k = bw > 0.0f ? (int)floorf(__fdiv_rn(__fsub_rn(t, r0), bw)) : 0;
                    k = k < 0 ? 0 : (k > 63 ? 63 : k);
                    atomicAdd(&s_bins[wib][k], w);
                }
            }
            const unsigned act = __ballot_sync(0xffffffffu, active);
            const unsigned val = __ballot_sync(0xffffffffu, valid);
            composited += __popc(act);
            const int last = 31 - __clz(act | 1u);  // last active lane (0 when none)
            const float Tn = T * __shfl_sync(0xffffffffu, p, last);
            if (act != val) {                       // terminated inside this chunk
                T = act ? Tn : T;
                break;
            }
            T = Tn;
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
