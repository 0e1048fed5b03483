// k_traverse.cu -- K-a: ray x KD-tree traversal and crossing emission
// (Sec. 3.5, Algorithm 1 "Traverse"; sampling of Algorithm 1 "Sampling" is defined
// on the emitted crossings and is evaluated where the samples are consumed).
//
// One thread per ray walks the tree front to back (near child first: the child on
// the origin's side of the split plane; far children wait on a short register
// stack).  Every visited node is tested with the slab method in a fixed FP32
// operation order -- per axis
// t0 = (lo - o) * inv, t1 = (hi - o) * inv with inv = 1 / d correctly rounded, no
// fused multiply-add, NaN-ignoring min/max, entry clamped at 0 -- so the crossing
// list is reproducible bit for bit.  A node whose interval is empty is pruned (its
// leaves' intervals are subsets).  A leaf with exit > entry is emitted as
// (entry, exit) at crossing slot ray * maxc + k and counted in a per-CTA shared-memory
// histogram that is flushed to the per-leaf totals with one atomic per touched leaf.
// Traversal stops after maxc crossings (whole crossings are kept under the cap).
// With the proposal sampler, a leaf crossing [t_in, t_out] is kept only when it
// overlaps a kept depth bin [t0 + k w, t0 + (k + 1) w), w = (t1 - t0) / 64 of the
// ray's root interval [t0, t1] (same FP32 operation order as the oracle); rays that
// fell back keep every crossing.  With empty-space skipping (Sec. 4.1: the density
// grid also marks the empty regions) a leaf crossing is kept only when one of
// its samples -- placed as it would be as the ray's next kept crossing, in the
// sampling step's FP32 order -- lies in a guidance-grid cell above the threshold;
// skipped crossings do not count toward maxc.
// With adaptive hierarchical sampling (Sec. 3.5, Algorithm 1's HCheck; Fig. 1 (c)) an
// inner node is descended only while its extent along its split axis, hi - lo (exact
// for the dyadic boxes of the tree), exceeds lod x entry (the product rounded to FP32):
// a subdivision finer than the ray's footprint at that distance is not resolved, and
// the inner node becomes one crossing of its own network (id L + preorder rank of the
// inner node); the proposal and empty-space rules apply to it as to a leaf.
#include "amnerf_internal.h"

namespace amnerf {
namespace {

__device__ __forceinline__ bool slab(const float4& A, const float4& B, const float o[3], const float inv[3],
                                     float& tin, float& tout) {
    const float lo[3] = {A.x, A.y, A.z};
    const float hi[3] = {B.x, B.y, B.z};
    float tmin[3], tmax[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t0 = __fmul_rn(__fsub_rn(lo[a], o[a]), inv[a]);
        const float t1 = __fmul_rn(__fsub_rn(hi[a], o[a]), inv[a]);
        tmin[a] = fminf(t0, t1);
        tmax[a] = fmaxf(t0, t1);
    }
    float e = fmaxf(fmaxf(tmin[0], tmin[1]), tmin[2]);
    const float x = fminf(fminf(tmax[0], tmax[1]), tmax[2]);
    e = fmaxf(e, 0.0f);
    tin = e;
    tout = x;
    return x > e;
}

// Bin k spans [lo_k, hi_k) with lo_k = r0 + k w and hi_k = r0 + (k + 1) w in FP32;
// both are non-decreasing in k, so the bins a crossing [tin, tout] overlaps
// (tin < hi_k and tout > lo_k) form one run [kmin, kmax]: kmin is the first k with
// hi_k > tin, kmax the last with lo_k < tout.  A first guess by division is moved
// to the exact ends with the same comparisons.
__device__ __forceinline__ float bin_lo(float r0, float bw, int k) { return __fadd_rn(r0, __fmul_rn((float)k, bw)); }

__device__ __forceinline__ bool overlaps_kept(uint64_t kept, float r0, float bw, float tin, float tout) {
    if (!kept || !(bw > 0.0f)) return false;
    const float inv = __frcp_rn(bw);
    int a = (int)fminf(fmaxf(floorf(__fmul_rn(__fsub_rn(tin, r0), inv)), 0.0f), 63.0f);
    while (a > 0 && bin_lo(r0, bw, a) > tin) --a;             // hi_{a-1} = lo_a > tin
    while (a < 64 && !(bin_lo(r0, bw, a + 1) > tin)) ++a;    // hi_a <= tin
    int b = (int)fminf(fmaxf(floorf(__fmul_rn(__fsub_rn(tout, r0), inv)), 0.0f), 63.0f);
    while (b < 63 && bin_lo(r0, bw, b + 1) < tout) ++b;
    while (b >= 0 && !(bin_lo(r0, bw, b) < tout)) --b;
    if (a > b) return false;
    const uint64_t run = (b - a == 63) ? ~0ull : (((2ull << (b - a)) - 1ull) << a);
    return (kept & run) != 0;
}

// Whether a sample of crossing [tin, tout], placed as kept crossing k, lies in an
// occupied cell: t_j = tin + (j + u_j) delta, delta = (tout - tin) / steps, x = o + t d,
// cell = floor((x - lo) * sc) clamped, occupied when the density > thr.
__device__ __forceinline__ bool crossing_occupied(const OccArgs& oc, const float o[3], const float d[3],
                                                  uint64_t key, float tin, float tout, int k) {
    const float delta = __fmul_rn(__fsub_rn(tout, tin), __frcp_rn((float)oc.steps));  // steps: a power of two
    const int G = oc.G;
    for (int j = 0; j < oc.steps; ++j) {
        const float u = jit_fraction(oc.jitter, key, k, oc.steps, j);
        const float t = __fadd_rn(tin, __fmul_rn(__fadd_rn((float)j, u), delta));
        int c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float x = __fadd_rn(o[a], __fmul_rn(t, d[a]));
            const int ci = (int)floorf(__fmul_rn(__fsub_rn(x, oc.lo[a]), oc.sc[a]));
            c[a] = ci < 0 ? 0 : (ci > G - 1 ? G - 1 : ci);
        }
        if (__ldg(oc.grid + (size_t)c[0] + (size_t)G * ((size_t)c[1] + (size_t)G * (size_t)c[2])) > oc.thr)
            return true;
    }
    return false;
}

// HIER: adaptive hierarchical sampling compiled in (its HCheck costs registers, so the
// leaf-only walk is a separate instantiation).
template <bool HIER>
__global__ void __launch_bounds__(256) k_traverse(const float* __restrict__ ro, const float* __restrict__ rd,
                                                  uint32_t n, const DevNode* __restrict__ nodes, int maxc,
                                                  uint8_t* __restrict__ n_x, float2* __restrict__ xing,
                                                  uint16_t* __restrict__ xleaf, uint32_t* __restrict__ counts,
                                                  int n_leaves, int* __restrict__ err,
                                                  const uint64_t* __restrict__ mask,
                                                  const uint8_t* __restrict__ fallback, float2* __restrict__ root_out,
                                                  const OccArgs occ, const HierArgs hier) {
    extern __shared__ uint32_t s_cnt[];
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) s_cnt[i] = 0u;
    __syncthreads();

    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        float o[3], d[3], inv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = __ldg(ro + 3 * (size_t)r + a);
            d[a] = __ldg(rd + 3 * (size_t)r + a);
            inv[a] = __frcp_rn(d[a]);
        }
        // The near child is visited next; far children wait on a stack of 16-bit node
        // indices held in four 64-bit registers (the top entry in the low bits of st0).
        uint64_t st0 = 0, st1 = 0, st2 = 0, st3 = 0;
        int sp = 0;
        int nd = 0;
        bool have = true;  // nd is a node still to visit
        int cnt = 0;
        const size_t base = (size_t)r * (size_t)maxc;
        // proposal sampler: the root interval and this ray's kept depth bins
        float r0 = 0.f, r1 = 0.f;
        {
            const float4 A = __ldg(&nodes[0].a);
            const float4 B = __ldg(&nodes[0].b);
            if (!slab(A, B, o, inv, r0, r1)) r0 = r1 = 0.f;
            if (root_out) root_out[r] = make_float2(r0, r1);
        }
        const uint64_t kept_bins = (mask && !__ldg(fallback + r)) ? __ldg(mask + r) : 0ull;
        const bool masked = mask && !__ldg(fallback + r);
        const float bw = __fmul_rn(__fsub_rn(r1, r0), 0.015625f);  // bin width (t1 - t0) / 64
        const uint64_t key = (occ.grid && occ.jitter) ? jit_ray_key(occ.jitter, o, d) : 0ull;
        while (cnt < maxc) {
            if (!have) {
                if (sp == 0) break;
                nd = (int)(st0 & 0xffffu);
                st0 = (st0 >> 16) | (st1 << 48);
                st1 = (st1 >> 16) | (st2 << 48);
                st2 = (st2 >> 16) | (st3 << 48);
                st3 >>= 16;
                --sp;
            }
            have = false;
            const float4 A = __ldg(&nodes[nd].a);
            const float4 B = __ldg(&nodes[nd].b);
            float tin, tout;
            if (!slab(A, B, o, inv, tin, tout)) continue;
            const uint32_t meta = __float_as_uint(B.w);
            const int axis = (int)(meta & 3u) - 1;
            // HCheck: an inner node finer than the footprint is one crossing of its own network
            bool emit = axis < 0;
            if (HIER && !emit) {
                const float ext = axis == 0 ? __fsub_rn(B.x, A.x) : (axis == 1 ? __fsub_rn(B.y, A.y) : __fsub_rn(B.z, A.z));
                emit = !(ext > __fmul_rn(hier.lod, tin));
            }
            if (emit) {
                if (masked && !overlaps_kept(kept_bins, r0, bw, tin, tout)) continue;
                if (occ.grid && !crossing_occupied(occ, o, d, key, tin, tout, cnt)) continue;
                const uint32_t net = (!HIER || axis < 0) ? meta >> 2 : (uint32_t)__ldg(hier.node_net + nd);
                xing[base + cnt] = make_float2(tin, tout);
                xleaf[base + cnt] = (uint16_t)net;
                atomicAdd(&s_cnt[net], 1u);
                ++cnt;
                continue;
            }
            const float oa = axis == 0 ? o[0] : (axis == 1 ? o[1] : o[2]);
            const float da = axis == 0 ? d[0] : (axis == 1 ? d[1] : d[2]);
            const bool near_left = oa < A.w || (oa == A.w && da <= 0.0f);
            const int left = nd + 1;
            const int right = (int)(meta >> 2);
            if (sp + 1 > kStackDepth) {  // unreachable for depth <= 12; recorded, never trapped
                atomicCAS(err, 0, kDevErrStack);
                break;
            }
            const uint64_t far = (uint64_t)(near_left ? right : left);
            st3 = (st3 << 16) | (st2 >> 48);
            st2 = (st2 << 16) | (st1 >> 48);
            st1 = (st1 << 16) | (st0 >> 48);
            st0 = (st0 << 16) | far;
            ++sp;
            nd = near_left ? left : right;
            have = true;
        }
        n_x[r] = (uint8_t)cnt;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) {
        const uint32_t c = s_cnt[i];
        if (c) atomicAdd(&counts[i], c);
    }
}

}  // namespace

cudaError_t launch_traverse(cudaStream_t s, const float* ro, const float* rd, uint32_t n, const DevNode* nodes,
                            int maxc, uint8_t* n_x, float2* xing, uint16_t* xleaf, uint32_t* counts,
                            int n_leaves, int* err, const uint64_t* mask, const uint8_t* fallback,
                            float2* root_out, const OccArgs& occ, const HierArgs& hier) {
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    const unsigned blocks = (n + threads - 1) / threads;
    const size_t smem = sizeof(uint32_t) * (size_t)n_leaves;
    HierArgs h = hier;
    if (!(h.lod > 0.0f)) h.node_net = nullptr;
    auto kern = h.node_net ? k_traverse<true> : k_traverse<false>;
    kern<<<blocks, threads, smem, s>>>(ro, rd, n, nodes, maxc, n_x, xing, xleaf, counts, n_leaves, err, mask,
                                             fallback, root_out, occ, h);
    return cudaGetLastError();
}

}  // namespace amnerf
