// tc_common.cuh -- helpers of the tcgen05 kernels (the leaf networks in k_mlp_tc.cu and
// the proposal network in k_prop_tc.cu): core-matrix operand layout, BF16 rounding,
// inline PTX for mbarriers, bulk copies, tcgen05 MMA / TMEM loads and stores, and the
// frequency encoding with SFU anchors and double-angle steps.
#pragma once

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "amnerf_internal.h"

namespace amnerf {
namespace tcx {

constexpr unsigned long long kWaitCycles = 4000000000ull;  // ~2 s at 2 GHz

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }


// Core-matrix byte offset of element (row n, column k) of an N x K K-major operand.
__host__ __device__ inline size_t cm_offset(int n, int k, int K) {
    return (size_t)(n >> 3) * (K * 16) + (size_t)(k >> 3) * 128 + (size_t)(n & 7) * 16 + (size_t)(k & 7) * 2;
}


inline uint16_t f2bf(float f) {  // round to nearest even (inputs are finite)
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t r = ((u >> 16) & 1u) + 0x7fffu;
    return (uint16_t)((u + r) >> 16);
}


// ---- PTX helpers -----------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false when the deadline passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase,
                                                  unsigned long long limit = kWaitCycles) {
    if (mbar_test(bar, phase)) return true;
    const unsigned long long t0 = clock64();
    while (!mbar_test(bar, phase)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void wg_bar(int id) { asm volatile("barrier.sync %0, 128;" ::"r"(id) : "memory"); }

// The group's named barrier (128 threads) that also ORs a flag over the group: every
// thread leaves with the same answer, so a group that learns of a failed wait here
// leaves its loop together (no thread is left waiting at a later barrier).
__device__ __forceinline__ bool wg_bar_any(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %2, 0;\n\tbarrier.cta.red.or.pred po, %1, 128, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"(id), "r"(v ? 1u : 0u)
        : "memory");
    return r != 0;
}

// One thread of the group (its leader) polls the mbarrier (bounded) while the other
// 127 sleep at the group's named barrier, so waiting groups take no issue slots from
// working ones.  The flag carries the outcome to the whole group.
__device__ __forceinline__ bool group_wait(uint32_t bar, uint32_t phase, int bar_id, volatile int* flag, bool leader) {
    if (leader) *flag = mbar_wait_bounded(bar, phase) ? 1 : 0;
    wg_bar(bar_id);
    return *flag != 0;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle, LBO = 128 B, SBO = sbo bytes.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) |
           (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major, M = 128.
__device__ __forceinline__ uint32_t idesc_e4m3(int n) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// tcgen05 MMAs with A in TMEM (column address a_tmem) and B from a shared-memory
// descriptor, and the commit that tracks them, executed by a whole converged warp:
// elect.sync picks one lane, which issues the instruction (a converged warp elects its lowest lane every
// time, so one thread issues the MMAs and the commit that tracks them).  Measured on
// GB300, a chain of five dependent 128 x 64 x 16 MMAs issues in about 70 cycles this
// way, against about 270 from a single thread of a diverged warp.
__device__ __forceinline__ void mma_bf16_ts_warp(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                                 uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_e4m3_ts_warp(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                                 uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit_warp(uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* w) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]),
        "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* w) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(w[0]),
                 "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(__float_as_uint(v[0])),
                 "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
                 : "memory");
}

// The N FP32 values at shared address b (the same for every row) into columns [0, N)
// of this thread's TMEM lane: the initial accumulator of a layer's MMAs.
template <int N>
__device__ __forceinline__ void tmem_st_bias(uint32_t taddr, uint32_t b) {
#pragma unroll
    for (int c = 0; c < N / 16; ++c) {
        uint32_t w[16];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(w[4 * i + 0]), "=r"(w[4 * i + 1]), "=r"(w[4 * i + 2]), "=r"(w[4 * i + 3])
                         : "r"(b + 64u * c + 16u * i)
                         : "memory");
        tmem_st16(taddr + 16u * c, w);
    }
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// (a0 * b0, a1 * b1) with one packed FP32 instruction.
__device__ __forceinline__ float2 mul_f32x2(float2 a, float2 b) {
    unsigned long long ua, ub, ud;
    memcpy(&ua, &a, 8);
    memcpy(&ub, &b, 8);
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(ud) : "l"(ua), "l"(ub));
    float2 d;
    memcpy(&d, &ud, 8);
    return d;
}

// (a0 * b0 + c0, a1 * b1 + c1) with one packed FP32 instruction.
__device__ __forceinline__ float2 fma2v(float2 a, float2 b, float2 c) {
    unsigned long long ua, ub, uc, ud;
    memcpy(&ua, &a, 8);
    memcpy(&ub, &b, 8);
    memcpy(&uc, &c, 8);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(ud) : "l"(ua), "l"(ub), "l"(uc));
    float2 d;
    memcpy(&d, &ud, 8);
    return d;
}

// (a * b0 + c0, a * b1 + c1) with one packed FP32 instruction.
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

// 32 consecutive FP32 columns of this thread's TMEM lane, without waiting (pair with
// tmem_ld_wait before the values are used).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
        "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane (load + wait; the E4M3
// epilogues, whose register budget is tighter, read a row in two halves).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    tmem_ld32_nowait(taddr, r);
    tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 4 consecutive FP32 columns of this thread's TMEM lane, without waiting.
__device__ __forceinline__ void tmem_ld4_nowait(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}

// The W FP32 columns of this thread's TMEM lane: all loads issued, then one wait.
template <int W>
__device__ __forceinline__ void tmem_ld_row(uint32_t taddr, float (&v)[W]) {
    uint32_t r[W];
#pragma unroll
    for (int h = 0; h < W / 32; ++h) tmem_ld32_nowait(taddr + 32u * h, r + 32 * h);
    tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < W; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Four values to E4M3 (round to nearest even, saturating), first value in the low byte.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
    uint32_t r;  // the two conversions write the halves of one register
    asm("{\n\t.reg .b16 lo, hi;\n\tcvt.rn.satfinite.e4m3x2.f32 lo, %2, %1;\n\t"
        "cvt.rn.satfinite.e4m3x2.f32 hi, %4, %3;\n\tmov.b32 %0, {lo, hi};\n\t}"
        : "=r"(r)
        : "f"(a), "f"(b), "f"(c), "f"(d));
    return r;
}

// relu of four values to E4M3 (round to nearest even, saturating), first in the low byte.
__device__ __forceinline__ uint32_t pack_relu_e4m3x4(float a, float b, float c, float d) {
    uint32_t r;
    asm("{\n\t.reg .b16 lo, hi;\n\tcvt.rn.satfinite.relu.e4m3x2.f32 lo, %2, %1;\n\t"
        "cvt.rn.satfinite.relu.e4m3x2.f32 hi, %4, %3;\n\tmov.b32 %0, {lo, hi};\n\t}"
        : "=r"(r)
        : "f"(a), "f"(b), "f"(c), "f"(d));
    return r;
}

// Head activations with the SFU exp/log/reciprocal (relative error ~1e-6, far below the
// BF16/E4M3 operand rounding of this path).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float softplus_f(float z) { return z > 20.0f ? z : __logf(1.0f + __expf(z)); }
__device__ __forceinline__ float sigmoid_f(float z) { return rcp_approx(1.0f + __expf(-z)); }

__device__ __forceinline__ int leaf_of_tile(const uint32_t* __restrict__ tile_off, int n_leaves, uint32_t t) {
    int lo = 0, hi = n_leaves;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(tile_off + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// sin(pi 2^k p), cos(pi 2^k p): the argument is reduced exactly to r in [-1, 1]
// (2^k p - 2 rint(2^(k-1) p)), then the SFU sine/cosine of pi r (abs. error ~4e-7).
__device__ __forceinline__ void sincospi_anchor(float p, int k, float* s, float* c) {
    const float y = p * (float)(1 << k);
    const float r = y - 2.0f * rintf(0.5f * y);
    const float a = r * 3.14159265358979f;
    *s = __sinf(a);
    *c = __cosf(a);
}

// gamma_L(p) into f[F0 .. F0 + 3 + 6L) (compile-time indices, so f stays in registers):
// [p, sin(pi 2^k p), cos(pi 2^k p) for k < L], each a 3-vector.  Octaves 0 and 5 are
// anchors; the others follow by the double-angle recurrence (at most 4 doublings from
// an anchor: error < 1e-5).
template <int L, int F0, int N>
__device__ __forceinline__ void encode_freq(const float p[3], float (&f)[N]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) f[F0 + a] = p[a];
    float s[3], c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) sincospi_anchor(p[a], 0, &s[a], &c[a]);
#pragma unroll
    for (int k = 0; k < L; ++k) {
        if (k == 5) {
#pragma unroll
            for (int a = 0; a < 3; ++a) sincospi_anchor(p[a], 5, &s[a], &c[a]);
        } else if (k > 0) {
            // coordinates 0 and 1 as packed pairs, 2 alone; the same operations per
            // value: t = s + s, s' = t c, c' = fma(-t, s, 1) (-t = -2 s exactly)
            const float2 s01 = make_float2(s[0], s[1]), c01 = make_float2(c[0], c[1]);
            const float2 t01 = mul_f32x2(s01, make_float2(2.0f, 2.0f));
            const float2 tn01 = mul_f32x2(s01, make_float2(-2.0f, -2.0f));
            const float2 sn01 = mul_f32x2(t01, c01);
            const float2 cn01 = fma2v(tn01, s01, make_float2(1.0f, 1.0f));
            s[0] = sn01.x;
            s[1] = sn01.y;
            c[0] = cn01.x;
            c[1] = cn01.y;
            const float t = s[2] + s[2];
            const float sn = t * c[2];
            c[2] = fmaf(-t, s[2], 1.0f);
            s[2] = sn;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            f[F0 + 3 + 6 * k + a] = s[a];
            f[F0 + 6 + 6 * k + a] = c[a];
        }
    }
}

// Octaves LO .. HI-1 of gamma(p) into f[F0 ..]: octave k's sin(pi 2^k p) at
// F0 + 6 (k - LO) + a and its cos three later; the anchor is octave LO (SFU after an
// exact argument reduction), the later octaves follow by double-angle steps.
template <int LO, int HI, int F0, int N>
__device__ __forceinline__ void encode_octaves(const float p[3], float (&f)[N]) {
    float s[3], c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) sincospi_anchor(p[a], LO, &s[a], &c[a]);
#pragma unroll
    for (int k = LO; k < HI; ++k) {
        if (k > LO) {
            const float2 s01 = make_float2(s[0], s[1]), c01 = make_float2(c[0], c[1]);
            const float2 t01 = mul_f32x2(s01, make_float2(2.0f, 2.0f));
            const float2 tn01 = mul_f32x2(s01, make_float2(-2.0f, -2.0f));
            const float2 sn01 = mul_f32x2(t01, c01);
            const float2 cn01 = fma2v(tn01, s01, make_float2(1.0f, 1.0f));
            s[0] = sn01.x;
            s[1] = sn01.y;
            c[0] = cn01.x;
            c[1] = cn01.y;
            const float t = s[2] + s[2];
            const float sn = t * c[2];
            c[2] = fmaf(-t, s[2], 1.0f);
            s[2] = sn;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            f[F0 + 6 * (k - LO) + a] = s[a];
            f[F0 + 6 * (k - LO) + 3 + a] = c[a];
        }
    }
}

// Column order of the leaf networks' layer-0 input on the tensor cores (BF16): the
// encoding gamma_10(x) ++ gamma_4(d) (canonical feature c, 90 features) is stored so
// that the first 48 columns hold p_x and x's octaves 0-4, p_d and d's octaves 0-1, and
// the last 48 hold x's octaves 5-9, d's octaves 2-3, the bias input (column 90, a
// constant 1), two more constant-1 columns (91, 92) whose layer-0 weights are zero,
// and zero padding: each half of a row is encoded by its own thread from its own
// anchors.  Columns 80..95 stay in TMEM through the tile's later layers, so the
// constant-1 columns 90..92 also serve as the inputs of those layers' bias terms (one
// K = 16 MMA against the bias split into three BF16 parts).  kperm(k) is the
// canonical feature of column k, -1 for the layer-0 bias input, -3 for the other
// constant-1 columns and -2 for padding.
__host__ __device__ constexpr int kperm(int k) {
    return k < 33 ? k
                  : (k < 48 ? k + 30
                            : (k < 78 ? k - 15 : (k < 90 ? k : (k == 90 ? -1 : (k <= 92 ? -3 : -2)))));
}
constexpr int kOnesStep = 80;  // first column of the K = 16 step that holds the constant-1 columns
constexpr int kOnesCol = 90;   // the constant-1 columns are kOnesCol .. kOnesCol + 2

// Columns [32 C, 32 C + 32) of the layer-0 input in kperm order, from the canonical
// features f, packed two per word and written to this thread's TMEM lane.
template <int C, int N>
__device__ __forceinline__ void store_chunk_perm(uint32_t a_row, const float (&f)[N]) {
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int k0 = 32 * C + 2 * i, k1 = k0 + 1;
        const int c0 = kperm(k0), c1 = kperm(k1);
        const float v0 = c0 >= 0 ? f[c0 >= 0 ? c0 : 0] : (c0 == -2 ? 0.0f : 1.0f);
        const float v1 = c1 >= 0 ? f[c1 >= 0 ? c1 : 0] : (c1 == -2 ? 0.0f : 1.0f);
        w[i] = pack_bf16(v0, v1);
    }
    tmem_st16(a_row + 16u * C, w);
}

// Features [32 c, 32 c + 32) of f packed two per word (even feature in the low half)
// and written to this thread's TMEM lane at A column 16 c; feature N (one past the
// last) is the constant 1 that multiplies the folded bias.
template <int C, int N>
__device__ __forceinline__ void store_chunk(uint32_t a_row, const float (&f)[N]) {
    uint32_t w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int f0 = 32 * C + 2 * i, f1 = f0 + 1;
        const float v0 = f0 < N ? f[f0 < N ? f0 : 0] : (f0 == N ? 1.0f : 0.0f);
        const float v1 = f1 < N ? f[f1 < N ? f1 : 0] : (f1 == N ? 1.0f : 0.0f);
        w[i] = pack_bf16(v0, v1);
    }
    tmem_st16(a_row + 16u * C, w);
}


}  // namespace tcx
}  // namespace amnerf
