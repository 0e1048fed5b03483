// k_proposal.cu -- learned proposal sampler (not in the paper; a sampling network in
// the spirit of the related work of Sec. 2.1): a small MLP predicts, per ray, how
// the compositing weight is distributed over 64 uniform depth bins of the ray's root
// interval plus a background bin, so that only the leaf crossings overlapping the
// predicted bins are sampled.
//
// Network: input gamma_10(entry point o + t0 d) ++ gamma_4(d) (90), two ReLU layers of
// 32, 65 logits, softmax.  Parameters (FP32, flat): W1 [32 x 90], b1 [32], W2 [32 x 32],
// b2 [32], W3 [65 x 32], b3 [65] -- 6113 values.  Training minimises the mean cross-
// entropy against the plain renderer's binned compositing weights with Adam.
//
// Kernels:
//   k_prop_infer   persistent CTAs over tiles of 128 rays: per ray the root slab test
//                  (the traversal's FP32 operation order) and the encoding; per tile
//                  the three layers as register-blocked FP32 products from shared
//                  memory; per ray the softmax and the kept bins: bins by decreasing
//                  mass (ties to the lower index) until the mass reaches `coverage`
//                  (the background counts toward it); more than max_bins depth bins
//                  -> fallback to the plain sampler.
//   k_prop_infer_tc the same for renders on the tensor cores: each CTA converts the FP32
//                  parameters to BF16 operands in shared memory (the bias of each
//                  layer as one more input column against a constant 1), and every
//                  warpgroup runs a tile's three layers as tcgen05 MMAs (128 x 32 x 96,
//                  128 x 32 x 48, 128 x 80 x 48; activations in TMEM), then the softmax
//                  and the same bin selection.  amnerf_proposal_predict keeps the FP32
//                  kernel (its probabilities are the FP32 ones).
//   k_prop_grad    one CTA per 128 rays: each thread runs its ray forward and
//                  backward and leaves its activations and deltas in shared memory;
//                  the CTA then forms the gradient contractions (sum over its rays of
//                  delta x activation) and adds them with one atomic per parameter.
//   k_prop_adam    elementwise Adam update, then clears the gradient.
#include <cstring>

#include "amnerf_internal.h"
#include "tc_common.cuh"

namespace amnerf {
namespace {

constexpr int PIN = 90, PH = 32, PO = 65;
constexpr int NPAR = PH * PIN + PH + PH * PH + PH + PO * PH + PO;
constexpr int OFF_W1 = 0, OFF_B1 = PH * PIN, OFF_W2 = OFF_B1 + PH, OFF_B2 = OFF_W2 + PH * PH,
              OFF_W3 = OFF_B2 + PH, OFF_B3 = OFF_W3 + PO * PH;
constexpr int kRays = 128;  // rays per CTA

__device__ __forceinline__ bool root_slab(const float* box, const float o[3], const float d[3], float& t0,
                                          float& t1) {
    float tmin[3], tmax[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float inv = __frcp_rn(d[a]);
        const float u0 = __fmul_rn(__fsub_rn(box[a], o[a]), inv);
        const float u1 = __fmul_rn(__fsub_rn(box[3 + a], o[a]), inv);
        tmin[a] = fminf(u0, u1);
        tmax[a] = fmaxf(u0, u1);
    }
    float e = fmaxf(fmaxf(tmin[0], tmin[1]), tmin[2]);
    const float x = fminf(fminf(tmax[0], tmax[1]), tmax[2]);
    e = fmaxf(e, 0.0f);
    t0 = e;
    t1 = x;
    return x > e;
}

// The 90 input features of one ray, in the oracle's order; feature f goes to x[f * S].
template <int S>
__device__ __forceinline__ void prop_features(const float o[3], const float d[3], float t0, float* x) {
    float e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) e[a] = __fadd_rn(o[a], __fmul_rn(t0, d[a]));
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a * S] = e[a];
#pragma unroll
    for (int k = 0; k < 10; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) sincospif(e[a] * (float)(1 << k), &x[(3 + 6 * k + a) * S], &x[(6 + 6 * k + a) * S]);
#pragma unroll
    for (int a = 0; a < 3; ++a) x[(63 + a) * S] = d[a];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) sincospif(d[a] * (float)(1 << k), &x[(66 + 6 * k + a) * S], &x[(69 + 6 * k + a) * S]);
}

// Forward pass from features in shared memory row xr (stride 1) with parameters in
// shared memory P; h1, h2 post-ReLU, q softmax.
__device__ __forceinline__ void prop_forward(const float* __restrict__ P, const float* xr, float* h1, float* h2,
                                             float* q) {
#pragma unroll
    for (int o = 0; o < PH; ++o) h1[o] = P[OFF_B1 + o];
    for (int f = 0; f < PIN; ++f) {
        const float v = xr[f];
#pragma unroll
        for (int o = 0; o < PH; ++o) h1[o] = fmaf(P[OFF_W1 + o * PIN + f], v, h1[o]);
    }
#pragma unroll
    for (int o = 0; o < PH; ++o) h1[o] = fmaxf(h1[o], 0.0f);
#pragma unroll
    for (int o = 0; o < PH; ++o) {
        float acc = P[OFF_B2 + o];
#pragma unroll
        for (int i = 0; i < PH; ++i) acc = fmaf(P[OFF_W2 + o * PH + i], h1[i], acc);
        h2[o] = fmaxf(acc, 0.0f);
    }
    float m = -INFINITY;
#pragma unroll
    for (int o = 0; o < PO; ++o) {
        float acc = P[OFF_B3 + o];
#pragma unroll
        for (int i = 0; i < PH; ++i) acc = fmaf(P[OFF_W3 + o * PH + i], h2[i], acc);
        q[o] = acc;
        m = fmaxf(m, acc);
    }
    float s = 0.0f;
#pragma unroll
    for (int o = 0; o < PO; ++o) {
        q[o] = expf(q[o] - m);
        s += q[o];
    }
    const float inv = 1.0f / s;
#pragma unroll
    for (int o = 0; o < PO; ++o) q[o] *= inv;
}

// ---- inference ---------------------------------------------------------------------
// Persistent CTAs over tiles of kRays rays.  Each layer is a (kRays x 32) x K FP32
// product formed from shared memory: activations are stored feature-major
// ([feature][ray]) and weights transposed ([in][out]), so a thread's 4-ray x
// 8-output register block takes one 16-byte activation load and two 16-byte weight
// loads per input feature for 32 FMAs.  Every output is accumulated from its bias
// over the inputs in order, the oracle's order.
constexpr int kW3ld = 68;      // padded row of W3^T (65 used)
constexpr int kInferGroups = 3;  // warpgroups per CTA, one tile each; one CTA per SM
struct InferWeights {
    float W1t[PIN][PH];
    float W2t[PH][PH];
    float W3t[PH][kW3ld];
    float b1[PH], b2[PH], b3[kW3ld];
};
// One warpgroup's tile buffers.  A holds the features [f][ray]; after the first
// layer its rows 0..31 take H2, rows 32..64 the logits 32..64.  B holds H1, then the
// logits 0..31.
struct InferTile {
    float A[PIN][kRays];
    float B[PH][kRays];
};
static_assert(PO <= PIN, "logits 32..64 live in feature rows");

__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory"); }

// Barrier of warpgroup g that also returns whether v holds for any of its threads.
__device__ __forceinline__ bool group_any(int g, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbarrier.red.or.pred q, %2, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(g + 1)
        : "memory");
    return r != 0;
}

// (a * b0 + c0, a * b1 + c1) with one packed FP32 instruction; each half is an
// ordinary correctly rounded fused multiply-add.
__device__ __forceinline__ float2 fma_f32x2(float a, float2 b, float2 c) {
    const float2 aa = make_float2(a, a);
    unsigned long long ua, ub, uc, ud;
    memcpy(&ua, &aa, 8);
    memcpy(&ub, &b, 8);
    memcpy(&uc, &c, 8);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(ud) : "l"(ua), "l"(ub), "l"(uc));
    float2 d;
    memcpy(&d, &ud, 8);
    return d;
}

// out[ob + c][r] = act(bias[ob + c] + sum_k Wt[k][ob + c] in[k][r]) for 32 outputs c.
template <int K, int LDW, bool RELU>
__device__ __forceinline__ void tile_layer(const float (*in)[kRays], const float* Wt, const float* bias, int ob,
                                           float (*out)[kRays]) {
    const int warp = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
    const int r0 = warp * 32 + (lane & 7) * 4;
    const int c0 = ob + (lane >> 3) * 8;
    float acc[4][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float bj = bias[c0 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = bj;
    }
    float2 acc2[4][4];  // (output 2p, output 2p + 1) of ray i
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc2[i][p] = make_float2(acc[i][2 * p], acc[i][2 * p + 1]);
#pragma unroll 3
    for (int k = 0; k < K; ++k) {
        const float4 x = *reinterpret_cast<const float4*>(&in[k][r0]);
        const float4 wa = *reinterpret_cast<const float4*>(Wt + k * LDW + c0);
        const float4 wb = *reinterpret_cast<const float4*>(Wt + k * LDW + c0 + 4);
        const float xv[4] = {x.x, x.y, x.z, x.w};
        const float2 wp[4] = {make_float2(wa.x, wa.y), make_float2(wa.z, wa.w), make_float2(wb.x, wb.y),
                              make_float2(wb.z, wb.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int p = 0; p < 4; ++p) acc2[i][p] = fma_f32x2(xv[i], wp[p], acc2[i][p]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            acc[i][2 * p] = acc2[i][p].x;
            acc[i][2 * p + 1] = acc2[i][p].y;
        }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float4 v = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        if (RELU) v = make_float4(fmaxf(v.x, 0.0f), fmaxf(v.y, 0.0f), fmaxf(v.z, 0.0f), fmaxf(v.w, 0.0f));
        *reinterpret_cast<float4*>(&out[c0 + j][r0]) = v;
    }
}

// Kept bins of one ray from its column of q: bins by decreasing mass, ties to the
// lower index, until the mass reaches `coverage` (the background, bin 64, counts
// toward it but is not kept); a depth bin beyond max_bins means fallback (returns
// true).  The 64 depth masses are sorted (sorting network, descending) and walked
// in that order, so the running sum sees the same values in the same order as a
// repeated arg-max; the background enters before the first depth mass it strictly
// exceeds.  The walk ends at the last kept mass tau, of which the first c_tau bins
// (lowest indices) with q == tau are kept along with every bin with q > tau.
__device__ __forceinline__ bool select_bins(const float (*QB)[kRays], const float (*QA)[kRays], int t,
                                            float coverage, int max_bins, uint64_t& mk) {
#define Q_(b) ((b) < 32 ? QB[(b)][t] : QA[(b)][t])
    float v[64];
#pragma unroll
    for (int b = 0; b < 64; ++b) v[b] = Q_(b);
    // Batcher's odd-even merge sort, descending: 543 compare-exchanges (the bitonic
    // network takes 672), in the same 21 layers
#pragma unroll
    for (int p = 1; p < 64; p <<= 1) {
#pragma unroll
        for (int k = p; k >= 1; k >>= 1) {
            // pairs (a, a + k) with a in the first half of a 2k-period starting at
            // k mod p, both inside one block of 2p
#pragma unroll
            for (int a = 0; a < 64; ++a) {
                const int r = k % p, b = a + k;
                if (a >= r && (a - r) % (2 * k) < k && b < 64 && a / (2 * p) == b / (2 * p)) {
                    const float hi = fmaxf(v[a], v[b]);
                    v[b] = fminf(v[a], v[b]);
                    v[a] = hi;
                }
            }
        }
    }
    const float vbg = Q_(64);
    bool bg_taken = false, fb = false;
    float cum = 0.0f, tau = 0.0f;
    int kept = 0, c_tau = 0;
#pragma unroll
    for (int p = 0; p < 64; ++p) {
        if (!bg_taken && vbg > v[p]) {
            if (!(cum < coverage)) break;
            cum += vbg;
            bg_taken = true;
        }
        if (!(cum < coverage)) break;
        cum += v[p];
        if (kept == max_bins) {
            fb = true;
            break;
        }
        if (kept > 0 && v[p] == tau) {
            ++c_tau;
        } else {
            tau = v[p];
            c_tau = 1;
        }
        ++kept;
    }
    mk = 0;
    if (fb || kept == 0) return fb;
    int eq = 0;
#pragma unroll
    for (int b = 0; b < 64; ++b) {
        const float q = Q_(b);
        const bool take = q > tau || (q == tau && eq < c_tau);
        eq += (q == tau && take) ? 1 : 0;
        mk |= take ? (1ull << b) : 0ull;
    }
    return false;
#undef Q_
}

__global__ void __launch_bounds__(kRays * kInferGroups, 1) k_prop_infer(
    const float* __restrict__ params, float b0, float b1, float b2, float b3, float b4, float b5,
    const float* __restrict__ ro, const float* __restrict__ rd, uint32_t n, float coverage, int max_bins,
    uint64_t* __restrict__ mask, uint8_t* __restrict__ fallback, unsigned long long* __restrict__ n_fallback,
    float* __restrict__ q_out) {
    extern __shared__ __align__(16) uint8_t smraw[];
    InferWeights& S = *reinterpret_cast<InferWeights*>(smraw);
    for (int i = threadIdx.x; i < PH * PIN; i += blockDim.x) S.W1t[i % PIN][i / PIN] = params[OFF_W1 + i];
    for (int i = threadIdx.x; i < PH * PH; i += blockDim.x) S.W2t[i % PH][i / PH] = params[OFF_W2 + i];
    for (int i = threadIdx.x; i < PO * PH; i += blockDim.x) S.W3t[i % PH][i / PH] = params[OFF_W3 + i];
    for (int i = threadIdx.x; i < PH; i += blockDim.x) {
        S.b1[i] = params[OFF_B1 + i];
        S.b2[i] = params[OFF_B2 + i];
    }
    for (int i = threadIdx.x; i < kW3ld; i += blockDim.x) S.b3[i] = i < PO ? params[OFF_B3 + i] : 0.0f;
    __syncthreads();
    const int g = threadIdx.x >> 7;   // warpgroup
    const int t = threadIdx.x & 127;  // ray of the tile
    InferTile& T = reinterpret_cast<InferTile*>(smraw + sizeof(InferWeights))[g];
    const uint32_t n_tiles = (n + kRays - 1) / kRays;
    uint32_t n_fb = 0;
    for (uint32_t tile = blockIdx.x * kInferGroups + g; tile < n_tiles; tile += gridDim.x * kInferGroups) {
        group_sync(g);  // the previous tile's q fully read
        const uint32_t r = tile * kRays + t;
        float o[3] = {0.f, 0.f, 0.f}, d[3] = {1.f, 0.f, 0.f}, t0 = 0.f, t1 = 0.f;
        bool hit = false;
        if (r < n) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = __ldg(ro + 3 * (size_t)r + a);
                d[a] = __ldg(rd + 3 * (size_t)r + a);
            }
            const float box[6] = {b0, b1, b2, b3, b4, b5};
            hit = root_slab(box, o, d, t0, t1);
            if (!hit) t0 = t1 = 0.f;  // as the traversal reports the root interval of a miss
        }
        prop_features<kRays>(o, d, t0, &T.A[0][t]);
        // a tile whose rays all miss the root box keeps no bins (it has no crossings):
        // the network is skipped unless the predictions themselves are requested
        if (!group_any(g, hit) && !q_out) {
            if (r < n) {
                mask[r] = 0ull;
                fallback[r] = 0;
            }
            continue;
        }
        tile_layer<PIN, PH, true>(T.A, &S.W1t[0][0], S.b1, 0, T.B);   // H1 -> B
        group_sync(g);
        tile_layer<PH, PH, true>(T.B, &S.W2t[0][0], S.b2, 0, T.A);    // H2 -> A rows 0..31
        group_sync(g);
        tile_layer<PH, kW3ld, false>(T.A, &S.W3t[0][0], S.b3, 0, T.B);   // logits 0..31 -> B
        tile_layer<PH, kW3ld, false>(T.A, &S.W3t[0][0], S.b3, 32, T.A);  // logits 32..63 -> A rows 32..63
        {  // logit 64 (background), one per thread, into A row 64
            float acc = S.b3[64];
#pragma unroll
            for (int i = 0; i < PH; ++i) acc = fmaf(S.W3t[i][64], T.A[i][t], acc);
            T.A[64][t] = acc;
        }
        group_sync(g);
        if (r < n) {
#define L_(b) (*((b) < 32 ? &T.B[(b)][t] : &T.A[(b)][t]))
            float m = -INFINITY;
#pragma unroll
            for (int b = 0; b < PO; ++b) m = fmaxf(m, L_(b));
            float s = 0.0f;
#pragma unroll
            for (int b = 0; b < PO; ++b) {
                const float e = expf(L_(b) - m);
                L_(b) = e;
                s += e;
            }
            const float inv = 1.0f / s;
#pragma unroll
            for (int b = 0; b < PO; ++b) L_(b) *= inv;
            if (q_out) {
#pragma unroll
                for (int b = 0; b < PO; ++b) q_out[(size_t)r * PO + b] = L_(b);
            }
#undef L_
            uint64_t mk = 0;
            bool fb = select_bins(T.B, T.A, t, coverage, max_bins, mk);
            if (!hit) fb = false;
            mask[r] = fb ? ~0ull : (hit ? mk : 0ull);  // a ray that misses the box keeps nothing
            fallback[r] = fb ? 1 : 0;
            n_fb += fb ? 1u : 0u;
        }
    }
    n_fb = __reduce_add_sync(0xffffffffu, n_fb);
    if ((threadIdx.x & 31) == 0 && n_fb) atomicAdd(n_fallback, (unsigned long long)n_fb);
}

// ---- inference on the tensor cores (renders) ---------------------------------------
constexpr int kPTcGroups = 4;                      // warpgroups (tiles in flight) per CTA
constexpr int kP1K = 96, kP2K = 48, kP3N = 80;     // layer 1 K (90 + bias, padded), layers 2-3 K, layer 3 N
constexpr uint32_t kPW1 = 0;                                        // W1 [32 x 96]
constexpr uint32_t kPW2 = kPW1 + PH * kP1K * 2;                     // W2 [32 x 48]
constexpr uint32_t kPW3 = kPW2 + PH * kP2K * 2;                     // W3 [80 x 48]
constexpr uint32_t kPWBytes = kPW3 + kP3N * kP2K * 2;               // 16 896 B
struct PropTcTile {
    float Q[PO][kRays];  // the tile's probabilities, [bin][ray]
};
struct PropTcCtl {
    uint64_t bar_m[kPTcGroups];
    int flag[kPTcGroups];
    uint32_t tmem_base;
};
constexpr size_t kPTcSmem = kPWBytes + kPTcGroups * sizeof(PropTcTile) + sizeof(PropTcCtl);
static_assert(kPWBytes % 1024 == 512 || kPWBytes % 128 == 0, "weight blob alignment");

// TMEM per warpgroup (128 columns): D (the layer-3 accumulator, 80 FP32 columns; layers
// 1-2 use 32) then A (48 columns: 96 BF16 inputs of layer 1, 48 of layers 2-3).
constexpr uint32_t kPACol = 80;

__global__ void __launch_bounds__(128 * kPTcGroups, 1) k_prop_infer_tc(
    const float* __restrict__ params, float b0, float b1, float b2, float b3, float b4, float b5,
    const float* __restrict__ ro, const float* __restrict__ rd, uint32_t n, float coverage, int max_bins,
    uint64_t* __restrict__ mask, uint8_t* __restrict__ fallback, unsigned long long* __restrict__ n_fallback,
    int* __restrict__ err, float* __restrict__ q_out) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t* wb = sm;
    PropTcTile* tiles = reinterpret_cast<PropTcTile*>(sm + kPWBytes);
    PropTcCtl* ctl = reinterpret_cast<PropTcCtl*>(sm + kPWBytes + kPTcGroups * sizeof(PropTcTile));
    // BF16 operands, K-major core matrices; the bias is input column 90 (layer 1) or 32
    for (int i = threadIdx.x; i < PH * kP1K + PH * kP2K + kP3N * kP2K; i += blockDim.x) {
        float v = 0.0f;
        uint32_t off;
        if (i < PH * kP1K) {
            const int nn = i / kP1K, k = i - nn * kP1K;
            v = k < PIN ? params[OFF_W1 + nn * PIN + k] : (k == PIN ? params[OFF_B1 + nn] : 0.0f);
            off = kPW1 + (uint32_t)tcx::cm_offset(nn, k, kP1K);
        } else if (i < PH * kP1K + PH * kP2K) {
            const int e = i - PH * kP1K, nn = e / kP2K, k = e - nn * kP2K;
            v = k < PH ? params[OFF_W2 + nn * PH + k] : (k == PH ? params[OFF_B2 + nn] : 0.0f);
            off = kPW2 + (uint32_t)tcx::cm_offset(nn, k, kP2K);
        } else {
            const int e = i - PH * kP1K - PH * kP2K, nn = e / kP2K, k = e - nn * kP2K;
            if (nn < PO) v = k < PH ? params[OFF_W3 + nn * PH + k] : (k == PH ? params[OFF_B3 + nn] : 0.0f);
            off = kPW3 + (uint32_t)tcx::cm_offset(nn, k, kP2K);
        }
        *reinterpret_cast<__nv_bfloat16*>(wb + off) = __float2bfloat16_rn(v);
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < kPTcGroups; ++i) tcx::mbar_init(tcx::smem_u32(&ctl->bar_m[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tcx::fence_proxy_async();  // the operands written above are read by the MMAs (async proxy)
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tcx::smem_u32(&ctl->tmem_base)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tcx::tc_fence_before();
    __syncthreads();
    tcx::tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;
    const int g = threadIdx.x >> 7, t = threadIdx.x & 127, q = warp & 3;
    const int bar_id = 1 + g;
    const bool leader = t == 32 * (g & 3);
    const bool leader_warp = warp == 4 * g + (g & 3);  // issues the MMAs, converged (one lane elected)
    const uint32_t bar_m = tcx::smem_u32(&ctl->bar_m[g]);
    volatile int* flag = &ctl->flag[g];
    const uint32_t d_col = tmem + 128u * (uint32_t)g, a_col = d_col + kPACol;
    const uint32_t lane = (uint32_t)(32 * q) << 16;
    const uint32_t d_row = d_col + lane, a_row = a_col + lane;
    const uint32_t w_addr = tcx::smem_u32(wb);
    const uint64_t desc1 = tcx::sdesc(w_addr + kPW1, kP1K * 16u);
    const uint64_t desc2 = tcx::sdesc(w_addr + kPW2, kP2K * 16u);
    const uint64_t desc3 = tcx::sdesc(w_addr + kPW3, kP2K * 16u);
    float (*Q)[kRays] = tiles[g].Q;
    uint32_t ph = 0, n_fb = 0;
    bool ok = true;
    // one layer: MMAs over K = kin from A, into D, N columns; then the group waits
    auto layer = [&](uint64_t desc, int kin, int nout) -> bool {
        if (leader_warp) {
            tcx::tc_fence_after();
            const uint32_t idd = tcx::idesc_bf16(nout);
            for (int kk = 0; kk < kin / 16; ++kk)
                tcx::mma_bf16_ts_warp(d_col, a_col + 8u * kk, desc + 16u * kk, idd, kk > 0 ? 1u : 0u);
            tcx::mma_commit_warp(bar_m);
        }
        const bool got = tcx::group_wait(bar_m, ph, bar_id, flag, leader);
        ph ^= 1u;
        if (got) tcx::tc_fence_after();
        return got;
    };
    // relu of D columns 0..31 as the next layer's A: inputs 0..31, the constant 1 at 32
    auto hidden_to_a = [&]() {
        uint32_t r[32], pk[16];
        tcx::tmem_ld32_nowait(d_row, r);
        tcx::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) pk[i] = tcx::pack_relu_bf16(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
        tcx::tmem_st16(a_row, pk);
        uint32_t c8[8] = {tcx::pack_bf16(1.0f, 0.0f), 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        tcx::tmem_st8(a_row + 16u, c8);
        tcx::tmem_st_wait();
        tcx::tc_fence_before();
        tcx::wg_bar(bar_id);
    };
    const uint32_t n_tiles = (n + kRays - 1) / kRays;
    for (uint32_t tile = blockIdx.x * kPTcGroups + g; tile < n_tiles && ok; tile += gridDim.x * kPTcGroups) {
        const uint32_t r = tile * kRays + t;
        float o[3] = {0.f, 0.f, 0.f}, d[3] = {1.f, 0.f, 0.f}, t0 = 0.f, t1 = 0.f;
        bool hit = false;
        if (r < n) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = __ldg(ro + 3 * (size_t)r + a);
                d[a] = __ldg(rd + 3 * (size_t)r + a);
            }
            const float box[6] = {b0, b1, b2, b3, b4, b5};
            hit = root_slab(box, o, d, t0, t1);
            if (!hit) t0 = t1 = 0.f;
        }
        if (!group_any(g, hit)) {  // no crossings in this tile: nothing to keep
            if (r < n) {
                mask[r] = 0ull;
                fallback[r] = 0;
            }
            continue;
        }
        {  // layer-1 input: gamma_10(o + t0 d) ++ gamma_4(d) as BF16, the constant 1 at 90
            float e[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) e[a] = __fadd_rn(o[a], __fmul_rn(t0, d[a]));
            float f[PIN];
            tcx::encode_freq<10, 0>(e, f);
            tcx::encode_freq<4, 63>(d, f);
            tcx::store_chunk<0>(a_row, f);
            tcx::store_chunk<1>(a_row, f);
            tcx::store_chunk<2>(a_row, f);
            tcx::tmem_st_wait();
            tcx::tc_fence_before();
            tcx::wg_bar(bar_id);
        }
        if (!(ok = layer(desc1, kP1K, PH))) break;
        hidden_to_a();
        if (!(ok = layer(desc2, kP2K, PH))) break;
        hidden_to_a();
        if (!(ok = layer(desc3, kP2K, kP3N))) break;
        // logits 0..64 to registers; once every row has read D, the softmax there and
        // the probabilities to this ray's column of Q
        float v[PO];
        {
            uint32_t lo[64], bg[4];
            tcx::tmem_ld32_nowait(d_row, lo);
            tcx::tmem_ld32_nowait(d_row + 32u, lo + 32);
            tcx::tmem_ld4_nowait(d_row + 64u, bg);  // columns 65..67 are read but not used
            tcx::tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(lo[i]);
            v[64] = __uint_as_float(bg[0]);
        }
        tcx::tc_fence_before();
        tcx::wg_bar(bar_id);  // every row has read D before the next tile's MMAs
        if (r < n) {
            float m = -INFINITY;
#pragma unroll
            for (int b = 0; b < PO; ++b) m = fmaxf(m, v[b]);
            float sum = 0.0f;
#pragma unroll
            for (int b = 0; b < PO; ++b) {
                v[b] = __expf(v[b] - m);
                sum += v[b];
            }
            const float inv = 1.0f / sum;
#pragma unroll
            for (int b = 0; b < PO; ++b) Q[b][t] = v[b] * inv;
            if (q_out) {  // debug copy of this ray's probabilities
#pragma unroll
                for (int b = 0; b < PO; ++b) q_out[(size_t)r * PO + b] = Q[b][t];
            }
            uint64_t mk = 0;
            bool fb = select_bins(Q, Q, t, coverage, max_bins, mk);
            if (!hit) fb = false;
            mask[r] = fb ? ~0ull : (hit ? mk : 0ull);  // a ray that misses the box keeps nothing
            fallback[r] = fb ? 1 : 0;
            n_fb += fb ? 1u : 0u;
        }
    }
    if (!ok && leader) atomicCAS(err, 0, kDevErrTimeout);
    n_fb = __reduce_add_sync(0xffffffffu, n_fb);
    if ((threadIdx.x & 31) == 0 && n_fb) atomicAdd(n_fallback, (unsigned long long)n_fb);
    tcx::tc_fence_before();
    __syncthreads();
    tcx::tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// splitmix64 finaliser: the ray index of batch element i of step s.
__device__ __forceinline__ uint32_t batch_ray(uint64_t seed, uint64_t s, uint32_t i, uint32_t n) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (s * 0x100000001ull + i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)(z % n);
}

struct GradSmem {
    float P[NPAR];
    float X[kRays][PIN + 1];
    float H1[kRays][PH + 1];
    float H2[kRays][PH + 1];
    float DZ[kRays][PO];
    float DH2[kRays][PH + 1];
    float DH1[kRays][PH + 1];
    float loss[kRays];
};

// Gradient of the mean cross-entropy over a batch of B rays (B may span CTAs):
// ray indices come from `idx` (when non-NULL) or from the counter-based hash.
__global__ void __launch_bounds__(kRays) k_prop_grad(const float* __restrict__ params, const float* __restrict__ ro,
                                                     const float* __restrict__ rd, const float2* __restrict__ root,
                                                     const float* __restrict__ targets, uint32_t n, uint32_t B,
                                                     uint64_t seed, uint64_t step, float* __restrict__ grad,
                                                     float* __restrict__ loss) {
    extern __shared__ __align__(16) uint8_t smraw[];
    GradSmem& S = *reinterpret_cast<GradSmem*>(smraw);
    for (int i = threadIdx.x; i < NPAR; i += blockDim.x) S.P[i] = params[i];
    const uint32_t bi = blockIdx.x * kRays + threadIdx.x;
    const bool valid = bi < B;
    const int t = threadIdx.x;
    uint32_t r = 0;
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {1.f, 0.f, 0.f}, t0 = 0.f;
    if (valid) {
        r = B == n && seed == 0 ? bi : batch_ray(seed, step, bi, n);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = __ldg(ro + 3 * (size_t)r + a);
            d[a] = __ldg(rd + 3 * (size_t)r + a);
        }
        t0 = root[r].x;
    }
    prop_features<1>(o, d, t0, S.X[t]);
    __syncthreads();
    float h1[PH], h2[PH], q[PO];
    prop_forward(S.P, S.X[t], h1, h2, q);
    float L = 0.0f;
    if (valid) {
        float ps = 0.0f;
#pragma unroll
        for (int b = 0; b < PO; ++b) {
            const float p = __ldg(targets + (size_t)r * PO + b);
            if (p > 0.0f) L -= p * logf(q[b]);
            ps += p;
            S.DZ[t][b] = -p;
        }
#pragma unroll
        for (int b = 0; b < PO; ++b) S.DZ[t][b] += q[b] * ps;  // dL/dz = q sum(p) - p
    } else {
        for (int b = 0; b < PO; ++b) S.DZ[t][b] = 0.0f;
    }
    S.loss[t] = L;
#pragma unroll
    for (int i = 0; i < PH; ++i) {
        S.H1[t][i] = h1[i];
        S.H2[t][i] = h2[i];
    }
    // back through layer 3 and the second ReLU, then layer 2 and the first ReLU
    float dh2[PH];
#pragma unroll
    for (int i = 0; i < PH; ++i) {
        float acc = 0.0f;
        for (int b = 0; b < PO; ++b) acc = fmaf(S.P[OFF_W3 + b * PH + i], S.DZ[t][b], acc);
        dh2[i] = h2[i] > 0.0f ? acc : 0.0f;
        S.DH2[t][i] = dh2[i];
    }
#pragma unroll
    for (int i = 0; i < PH; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int o2 = 0; o2 < PH; ++o2) acc = fmaf(S.P[OFF_W2 + o2 * PH + i], dh2[o2], acc);
        S.DH1[t][i] = h1[i] > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    // gradient contractions over this CTA's rays, scaled by 1 / B (mean loss)
    const float sc = 1.0f / (float)B;
    for (int e = threadIdx.x; e < NPAR; e += blockDim.x) {
        float acc = 0.0f;
        if (e < OFF_B1) {  // W1[o][f]: sum_r DH1[r][o] X[r][f]
            const int o1 = e / PIN, f = e - o1 * PIN;
            for (int rr = 0; rr < kRays; ++rr) acc = fmaf(S.DH1[rr][o1], S.X[rr][f], acc);
        } else if (e < OFF_W2) {
            const int o1 = e - OFF_B1;
            for (int rr = 0; rr < kRays; ++rr) acc += S.DH1[rr][o1];
        } else if (e < OFF_B2) {
            const int k = e - OFF_W2, o2 = k / PH, i = k - o2 * PH;
            for (int rr = 0; rr < kRays; ++rr) acc = fmaf(S.DH2[rr][o2], S.H1[rr][i], acc);
        } else if (e < OFF_W3) {
            const int o2 = e - OFF_B2;
            for (int rr = 0; rr < kRays; ++rr) acc += S.DH2[rr][o2];
        } else if (e < OFF_B3) {
            const int k = e - OFF_W3, b = k / PH, i = k - b * PH;
            for (int rr = 0; rr < kRays; ++rr) acc = fmaf(S.DZ[rr][b], S.H2[rr][i], acc);
        } else {
            const int b = e - OFF_B3;
            for (int rr = 0; rr < kRays; ++rr) acc += S.DZ[rr][b];
        }
        atomicAdd(grad + e, acc * sc);
    }
    if (threadIdx.x < 32) {
        float l = 0.0f;
        for (int rr = threadIdx.x; rr < kRays; rr += 32) l += S.loss[rr];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
        if (threadIdx.x == 0) atomicAdd(loss, l * sc);
    }
}

// Adam (Kingma and Ba) with bias correction; t counts from 1.  Clears the gradient.
__global__ void k_prop_adam(float* __restrict__ P, float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int t, float lr, float b1, float b2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPAR) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.0f;
}

}  // namespace

int proposal_param_count() { return NPAR; }

constexpr size_t kInferSmem = sizeof(InferWeights) + kInferGroups * sizeof(InferTile);

cudaError_t launch_prop_infer(cudaStream_t s, int infer_grid, const float* params, const float root_box[6],
                              const float* ro, const float* rd, uint32_t n, float coverage, int max_bins,
                              uint64_t* mask, uint8_t* fallback, unsigned long long* n_fallback, float* q_out) {
    if (n == 0) return cudaSuccess;
    if (infer_grid < 1) return cudaErrorNotReady;  // prepare_proposal was not called
    const uint32_t tiles = (n + kRays - 1) / kRays;
    const uint32_t ctas = (tiles + kInferGroups - 1) / kInferGroups;
    const unsigned grid = ctas < (uint32_t)infer_grid ? ctas : (unsigned)infer_grid;
    k_prop_infer<<<grid, kRays * kInferGroups, kInferSmem, s>>>(params, root_box[0], root_box[1], root_box[2],
                                                                root_box[3], root_box[4], root_box[5], ro, rd, n,
                                                                coverage, max_bins, mask, fallback, n_fallback,
                                                                q_out);
    return cudaGetLastError();
}

cudaError_t launch_prop_infer_tc(cudaStream_t s, const float* params, const float root_box[6], const float* ro,
                                 const float* rd, uint32_t n, float coverage, int max_bins, uint64_t* mask,
                                 uint8_t* fallback, unsigned long long* n_fallback, int* err, float* q_out) {
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t tiles = (n + kRays - 1) / kRays;
    const uint32_t ctas = (tiles + kPTcGroups - 1) / kPTcGroups;
    const unsigned grid = ctas < (uint32_t)sms ? ctas : (unsigned)sms;  // one CTA per SM (it holds all of TMEM)
    k_prop_infer_tc<<<grid, 128 * kPTcGroups, kPTcSmem, s>>>(params, root_box[0], root_box[1], root_box[2],
                                                              root_box[3], root_box[4], root_box[5], ro, rd, n,
                                                              coverage, max_bins, mask, fallback, n_fallback, err,
                                                              q_out);
    return cudaGetLastError();
}

cudaError_t prepare_proposal(int* infer_grid) {
    cudaError_t e = cudaFuncSetAttribute(k_prop_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInferSmem);
    if (e != cudaSuccess) return e;
    // the tensor-core inference holds more than half of an SM's shared memory, so two of
    // its CTAs never share an SM (each allocates the whole TMEM)
    e = cudaFuncSetAttribute(k_prop_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPTcSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prop_infer, kRays * kInferGroups, kInferSmem);
    if (e != cudaSuccess) return e;
    *infer_grid = sms * (per_sm > 0 ? per_sm : 1);
    return cudaFuncSetAttribute(k_prop_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem));
}

cudaError_t launch_prop_grad(cudaStream_t s, const float* params, const float* ro, const float* rd,
                             const float2* root, const float* targets, uint32_t n, uint32_t batch, uint64_t seed,
                             uint64_t step, float* grad, float* loss) {
    if (batch == 0) return cudaSuccess;
    k_prop_grad<<<(batch + kRays - 1) / kRays, kRays, sizeof(GradSmem), s>>>(params, ro, rd, root, targets, n, batch,
                                                                            seed, step, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_prop_adam(cudaStream_t s, float* P, float* g, float* m, float* v, int t, float lr) {
    k_prop_adam<<<(NPAR + 255) / 256, 256, 0, s>>>(P, g, m, v, t, lr, 0.9f, 0.999f, 1e-8f);
    return cudaGetLastError();
}

}  // namespace amnerf
