// k_mlp_simt.cu -- K-c, plain FP32 path: per-leaf networks on CUDA cores.
//
// Network (Sec. 3.1 F_Theta, one small same-shaped MLP per leaf, Sec. 3.2 and 4.1):
// input gamma_lx(x) ++ gamma_ld(d) with gamma_L(p) = [p, sin(pi 2^k p), cos(pi 2^k p)]
// for k = 0..L-1 (the sinusoidal positional encoding, Fig. "complex"); `hidden` ReLU layers
// of `width`; head sigma = softplus(z0), rgb = sigmoid(z1..3).
//
// Work unit: a tile of 128 samples = 128 / steps crossings of ONE leaf (Sec. 3.5:
// samples sorted by node id and inferred per node).  Persistent CTAs take
// contiguous tile ranges, so a CTA reloads a leaf's weights only when its range
// crosses a leaf boundary.  Per tile: 128 threads rebuild their sample (crossing ->
// t_j = t_in + (j + 1/2) delta, x_j = o + t_j d, in the traversal's FP32 operation
// order), encode it into a feature-major shared tile, then every layer is a
// 128 x width register-blocked FP32 GEMM from shared memory (512 threads with 4 x 4
// blocks for width 64: the leaf's FP32 weights fill shared memory, so the CTA is
// alone on its SM and needs the warps itself); the head writes
// (sigma, r, g, b) to the sample's slot ray * cap + k * steps + j.
#include "amnerf_internal.h"

namespace amnerf {
namespace {

// threads per CTA: 512 for width 64 (4 x 4 register blocks, 16 warps per SM), 256 for 32
template <int W>
constexpr int kThreadsFor = W == 64 ? 512 : 256;
constexpr int kMaxK0 = 128;

// Leaf layout (floats): W0^T [k0][W], b0 [W], then per layer l>0: W_l^T [W][W], b_l [W],
// then Wo^T [W][4], bo [4]; stride rounded up to 4 floats.
__host__ __device__ inline size_t simt_stride(int width, int hidden, int k0) {
    const size_t n = (size_t)k0 * width + width + (size_t)(hidden - 1) * (width * width + width) + 4 * width + 4;
    return (n + 3) & ~(size_t)3;
}

__device__ __forceinline__ float softplus_f(float z) { return z > 20.0f ? z : log1pf(expf(z)); }
__device__ __forceinline__ float sigmoid_f(float z) { return 1.0f / (1.0f + expf(-z)); }

// out[n][128] = ReLU(in[k][128]^T W^T[k][n] + b), rows interleaved so a warp reads
// contiguous rows.  W = width; thread tile = RPT rows x 4 columns.
template <int W, int KIN>
__device__ __forceinline__ void gemm_layer(const float* __restrict__ in, int kin_rt, const float* __restrict__ wt,
                                           const float* __restrict__ bias, float* __restrict__ out) {
    constexpr int CG = W / 4;            // column groups of 4
    constexpr int RG = kThreadsFor<W> / CG;  // row groups
    constexpr int RPT = kTileRows / RG;  // rows per thread (4 for both widths)
    const int rg = threadIdx.x % RG;
    const int cg = threadIdx.x / RG;
    const int kin = KIN > 0 ? KIN : kin_rt;
    float acc[RPT][4];
    const float4 b4 = *reinterpret_cast<const float4*>(bias + 4 * cg);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        acc[r][0] = b4.x;
        acc[r][1] = b4.y;
        acc[r][2] = b4.z;
        acc[r][3] = b4.w;
    }
#pragma unroll 4
    for (int k = 0; k < kin; ++k) {
        const float4 w4 = *reinterpret_cast<const float4*>(wt + (size_t)k * W + 4 * cg);
        float a[RPT];
#pragma unroll
        for (int q = 0; q < RPT / 4; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(in + (size_t)k * kTileRows + rg * RPT + 4 * q);
            a[4 * q + 0] = v.x;
            a[4 * q + 1] = v.y;
            a[4 * q + 2] = v.z;
            a[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            acc[r][0] = fmaf(a[r], w4.x, acc[r][0]);
            acc[r][1] = fmaf(a[r], w4.y, acc[r][1]);
            acc[r][2] = fmaf(a[r], w4.z, acc[r][2]);
            acc[r][3] = fmaf(a[r], w4.w, acc[r][3]);
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int q = 0; q < RPT / 4; ++q) {
            float4 v;
            v.x = fmaxf(acc[4 * q + 0][c], 0.0f);
            v.y = fmaxf(acc[4 * q + 1][c], 0.0f);
            v.z = fmaxf(acc[4 * q + 2][c], 0.0f);
            v.w = fmaxf(acc[4 * q + 3][c], 0.0f);
            *reinterpret_cast<float4*>(out + (size_t)(4 * cg + c) * kTileRows + rg * RPT + 4 * q) = v;
        }
    }
}

__device__ __forceinline__ int leaf_of_tile(const uint32_t* __restrict__ tile_off, int n_leaves, uint32_t t) {
    // largest l with tile_off[l] <= t
    int lo = 0, hi = n_leaves;  // invariant: tile_off[lo] <= t < tile_off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(tile_off + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// gamma_L(p) written to feature-major shared memory starting at feature f0.
__device__ __forceinline__ void encode_simt(const float p[3], int L, float* __restrict__ sA, int f0, int row) {
#pragma unroll
    for (int a = 0; a < 3; ++a) sA[(f0 + a) * kTileRows + row] = p[a];
    for (int k = 0; k < L; ++k) {
        const float scale = (float)(1 << k);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float s, c;
            sincospif(p[a] * scale, &s, &c);
            sA[(f0 + 3 + 6 * k + a) * kTileRows + row] = s;
            sA[(f0 + 6 + 6 * k + a) * kTileRows + row] = c;
        }
    }
}

// Calibration: the largest value over the valid rows of a feature-major tile
// (non-negative inputs), merged into *dst (one atomic per warp).
__device__ __forceinline__ void tile_absmax(const float* __restrict__ t, int nfeat, int nvalid, float* dst) {
    if (threadIdx.x >= kTileRows) return;
    const int row = threadIdx.x;
    float m = 0.0f;
    if (row < nvalid)
        for (int f = 0; f < nfeat; ++f) m = fmaxf(m, fabsf(t[(size_t)f * kTileRows + row]));
    const unsigned u = __reduce_max_sync(0xffffffffu, __float_as_uint(m));  // m >= 0: bit order = value order
    if ((row & 31) == 0 && u) atomicMax(reinterpret_cast<unsigned*>(dst), u);
}

// HC > 0: the hidden-layer count and input width (90) fixed at compile time.
template <int W, int HC>
__global__ void __launch_bounds__(kThreadsFor<W>, 1) k_mlp_simt(MlpArgs g) {
    extern __shared__ __align__(16) float sm[];
    const size_t wstride = simt_stride(W, g.hidden, g.k0);
    float* sW = sm;                                   // [wstride]
    float* sA = sW + wstride;                         // [max(k0, W)][128]
    float* sH = sA + (size_t)kMaxK0 * kTileRows;      // [W][128]
    uint64_t* sSlot = reinterpret_cast<uint64_t*>(sH + (size_t)W * kTileRows);  // [128]

    // contiguous tile ranges (also each launch of the per-leaf loop)
    const uint32_t t_end = g.t_end == 0xffffffffu ? (uint32_t)g.stats[1] : g.t_end;
    const uint32_t span = t_end > g.t_begin ? t_end - g.t_begin : 0u;
    const uint32_t per = (span + gridDim.x - 1) / gridDim.x;
    const uint32_t t0 = min(g.t_begin + blockIdx.x * per, t_end);
    const uint32_t t1 = min(t0 + per, t_end);
    const int cpt = kTileRows / g.steps;
    const float* wall = reinterpret_cast<const float*>(g.weights);
    int cur = -1;
    for (uint32_t t = t0; t < t1; ++t) {
        const int leaf = leaf_of_tile(g.tile_off, g.n_leaves, t);
        if (leaf != cur) {
            __syncthreads();
            const float4* src = reinterpret_cast<const float4*>(wall + (size_t)leaf * wstride);
            float4* dst = reinterpret_cast<float4*>(sW);
            for (size_t i = threadIdx.x; i < wstride / 4; i += kThreadsFor<W>) dst[i] = __ldg(src + i);
            cur = leaf;
        }
        const uint32_t first = __ldg(g.offsets + leaf) + (t - __ldg(g.tile_off + leaf)) * (uint32_t)cpt;
        const uint32_t endc = __ldg(g.offsets + leaf + 1);
        if (threadIdx.x < kTileRows) {
            const int row = threadIdx.x;
            const int ci = row / g.steps;
            const int j = row - ci * g.steps;
            const uint32_t c = first + (uint32_t)ci;
            uint64_t slot = ~0ull;  // 64-bit: rays * cap may exceed 2^32
            float x[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
            if (c < endc) {
                const uint32_t id = __ldg(g.order + c);
                const uint32_t ray = id / (uint32_t)g.maxc;
                const uint32_t k = id - ray * (uint32_t)g.maxc;
                const float2 xi = __ldg(g.xing + id);
                // steps is a power of two: the product by its reciprocal is the exact quotient
                const float delta = __fmul_rn(__fsub_rn(xi.y, xi.x), __frcp_rn((float)g.steps));
                float o[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    o[a] = __ldg(g.ro + 3 * (size_t)ray + a);
                    d[a] = __ldg(g.rd + 3 * (size_t)ray + a);
                }
                // sample j at fraction u of its stratum (midpoint, or the stratified jitter)
                const float u = g.jitter ? jit_fraction(g.jitter, jit_ray_key(g.jitter, o, d), (int)k, g.steps, j) : 0.5f;
                const float tj = __fadd_rn(xi.x, __fmul_rn(__fadd_rn((float)j, u), delta));
#pragma unroll
                for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(o[a], __fmul_rn(tj, d[a]));
                slot = (uint64_t)ray * (uint64_t)g.cap + (uint64_t)(k * (uint32_t)g.steps + (uint32_t)j);
            }
            encode_simt(x, g.lx, sA, 0, row);
            encode_simt(d, g.ld, sA, 3 + 6 * g.lx, row);
            sSlot[row] = slot;
        }
        __syncthreads();
        // rows of this tile that hold samples (calibration counts only those)
        const int nvalid = (int)min((uint32_t)kTileRows, (endc - first) * (uint32_t)g.steps);
        float* amax = g.amax ? g.amax + (size_t)leaf * g.hidden : nullptr;
        if (amax) tile_absmax(sA, g.k0, nvalid, amax);
        const float* w = sW;
        const float* in = sA;
        float* out = sH;
        int kin = g.k0;
        const int hidden = HC > 0 ? HC : g.hidden;
#pragma unroll
        for (int l = 0; l < hidden; ++l) {
            if (HC > 0 && l == 0) gemm_layer<W, 90>(in, kin, w, w + (size_t)kin * W, out);
            else if (HC > 0) gemm_layer<W, W>(in, kin, w, w + (size_t)kin * W, out);
            else gemm_layer<W, 0>(in, kin, w, w + (size_t)kin * W, out);
            __syncthreads();
            if (amax && l + 1 < g.hidden) tile_absmax(out, W, nvalid, amax + l + 1);
            w += (size_t)kin * W + W;
            kin = W;
            float* tmp = const_cast<float*>(in);
            in = out;
            out = tmp;
        }
        if (threadIdx.x < kTileRows) {
            const int row = threadIdx.x;
            const uint64_t slot = sSlot[row];
            const float* bo = w + 4 * W;
            float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll 8
            for (int k = 0; k < W; ++k) {
                const float h = in[(size_t)k * kTileRows + row];
                const float4 w4 = *reinterpret_cast<const float4*>(w + 4 * k);
                z0 = fmaf(h, w4.x, z0);
                z1 = fmaf(h, w4.y, z1);
                z2 = fmaf(h, w4.z, z2);
                z3 = fmaf(h, w4.w, z3);
            }
            if (slot != ~0ull) {
                float4 o;
                o.x = softplus_f(z0 + bo[0]);
                o.y = sigmoid_f(z1 + bo[1]);
                o.z = sigmoid_f(z2 + bo[2]);
                o.w = sigmoid_f(z3 + bo[3]);
                static_cast<float4*>(g.slot_out)[slot] = o;
            }
        }
        __syncthreads();
    }
}

template <int W>
size_t simt_smem(int hidden, int k0) {
    return sizeof(float) * (simt_stride(W, hidden, k0) + (size_t)kMaxK0 * kTileRows + (size_t)W * kTileRows) +
           sizeof(uint64_t) * kTileRows;
}

template <int W>
cudaError_t prepare_w(int hidden, int k0) {
    const size_t smem = simt_smem<W>(hidden, k0);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_simt<W, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mlp_simt<W, W == 64 ? 4 : 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

template <int W>
cudaError_t launch_w(cudaStream_t s, const MlpArgs& a, int grid) {
    constexpr int HS = W == 64 ? 4 : 2;
    if (a.hidden == HS && a.k0 == 90)
        k_mlp_simt<W, HS><<<grid, kThreadsFor<W>, simt_smem<W>(a.hidden, a.k0), s>>>(a);
    else
        k_mlp_simt<W, 0><<<grid, kThreadsFor<W>, simt_smem<W>(a.hidden, a.k0), s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t simt_leaf_stride_floats(int width, int hidden, int k0) { return simt_stride(width, hidden, k0); }

cudaError_t prepare_mlp_simt(int width, int hidden, int k0) {
    if (k0 > kMaxK0) return cudaErrorInvalidValue;
    if (width == 64) return prepare_w<64>(hidden, k0);
    if (width == 32) return prepare_w<32>(hidden, k0);
    return cudaErrorInvalidValue;
}

cudaError_t launch_mlp_simt(cudaStream_t s, const MlpArgs& a, int grid) {
    if (a.k0 > kMaxK0) return cudaErrorInvalidValue;
    if (a.width == 64) return launch_w<64>(s, a, grid);
    if (a.width == 32) return launch_w<32>(s, a, grid);
    return cudaErrorInvalidValue;
}

}  // namespace amnerf
