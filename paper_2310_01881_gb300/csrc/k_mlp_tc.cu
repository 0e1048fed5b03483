// k_mlp_tc.cu -- K-c on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Same network and work unit as the FP32 path (Sec. 3.1 F_Theta; one small
// same-shaped MLP per leaf, Sec. 3.2; samples grouped by node, Sec. 3.5): a tile is
// 128 samples = 128 / steps crossings of one leaf.  Here every layer is one
// 128 x N x K tensor-core contraction with
//
//   A (activations, 128 x K, BF16)  -- kept in tensor memory (TMEM): row r of the
//                                      tile is TMEM lane r, two BF16 per 32-bit
//                                      column (even k in the low half)
//   B (layer weights, N x K, BF16)  -- the leaf's weights in shared memory, K-major
//                                      no-swizzle core matrices (8 rows x 16 B =
//                                      128 contiguous bytes; K-adjacent core matrices
//                                      128 B apart, 8-row groups K * 16 B apart),
//                                      bulk-copied (TMA engine) once per leaf change
//   D (128 x N, FP32)               -- accumulator in TMEM
//
// Measured on GB300, the tensor pipe retires one 128 x 64 x 16 MMA about every 34
// cycles when several warps issue, and a chain of five dependent ones takes about
// 300 cycles from issue to completion, so these small layers are bound by the
// latency of each tile's per-layer chain; keeping A in TMEM removes the
// shared-memory activation stores and proxy fences from that chain.
//
// Thread r of a warpgroup owns sample row r: it rebuilds the sample, encodes
// gamma(x) ++ gamma(d) and writes it into its TMEM lane (tcgen05.st 32x32b); after
// each MMA it reads its row of D (tcgen05.ld 32x32b: warp q of the group owns lanes
// 32q..32q+31) and writes the next layer's A back into TMEM.  BF16 folds layer 0's
// bias into its contraction (a weight column against a constant-1 input column) and
// writes every later layer's FP32 bias into its accumulator with one more K = 16 MMA
// (three constant-1 input columns of layer 0, still in TMEM, against the bias split
// into three BF16 parts), so the epilogue is ReLU with the conversion
// (cvt.rn.relu.bf16x2) and nothing else.  E4M3 with static scales does the same
// (its scales folded into the weights, its bias through a BF16 MMA); with per-row
// scales it applies its channel scales and bias with one packed FMA per pair first.
// The 4-wide head is one more BF16 MMA (16 rows, 4 used) on relu(h) written into the
// group's D columns; it runs while the group encodes its next tile.  Its accumulator
// sits in 16 TMEM columns that no layer writes, so its outputs (sigma = softplus,
// rgb = sigmoid) are read with the next tile's layer-0 accumulator and activated and
// stored while that tile's last layer's MMAs run.
//
// Several warpgroups per CTA work on different tiles, so one group's epilogue
// overlaps another's MMA.  Each group's leader warp (warp grp % 4 of the group, so
// the leader warps run on different SM sub-partitions) issues the group's MMAs
// converged, one lane elected per instruction, and tracks completion with
// tcgen05.commit on the group's mbarrier, on which every thread of the group then
// waits itself.  Every wait is bounded (clock64 deadline); a wait that runs out is
// ORed over the group at its next barrier, the group records AMNERF_E_TIMEOUT in
// the status word and leaves its tile loop together, and the CTA still frees its
// TMEM before returning.
//
// Encoding: sin/cos(pi 2^k p) at k = 0 and k = 5 come from the SFU after an exact
// argument reduction; the other octaves follow by the double-angle recurrence
// (s' = 2 s c, c' = 1 - 2 s^2), whose error roughly doubles per octave: below 1e-5
// after 4 doublings, far under the BF16 rounding of a feature (2^-9 relative).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "amnerf_internal.h"
#include "tc_common.cuh"

namespace amnerf {
namespace {

using namespace tcx;

constexpr int kLX = 10;  // encodings this kernel is instantiated for
constexpr int kLD = 4;
constexpr int kMaxGroups = 4;
// ---- per-leaf weight blob layout (bytes) -------------------------------------------
// W0 [width x k0p], W1.. [width x kh] in the operand type (BF16, or E4M3 with FP32
// per-output-channel scales sw [hidden][width]); head Wo BF16 [16 x khead]; FP32
// biases b_0..b_{hidden-1} [width] and bo [4].  kh = khead = width.  BF16 folds layer
// 0's bias into its contraction (input column 90, inside the padding to k0p = 96,
// holds the bias and the encoded row carries 1 there).  For every later BF16 layer
// one more K = 16 MMA writes the FP32 bias into the accumulator (block bb, below) in
// the one-thread-per-row kernel; the two-threads-per-row kernel and the head have the
// epilogue of the layer before write the FP32 bias (block bias) into the accumulator
// columns.  The MMAs accumulate onto it.  E4M3 with per-row scales adds its FP32
// bias in the epilogue, after the scales (an E4M3 bias would lose too much); with
// static scales it enters through a BF16 MMA (below).  Both run the head as one more
// BF16 MMA of a 16-row matrix (rows 0..3 used).
// E4M3 with static scales (act_max known per leaf and layer; see pack_tc_leaf) folds
// every scale into the weights: output channel n of layer l has one scale s_(l,n),
// the next layer's E4M3 input of channel n is stored as relu(y_n) / s_(l,n) and that
// scale is folded into the next layer's weight columns (the head's BF16 weights for
// the last layer).  The accumulator is then (y - b) / s, the bias enters as b / s
// through a BF16 bias MMA (block bb, one chunk per layer, against BF16 constant-1
// columns that the kernel writes once into A columns 40..47), and the epilogue is
// ReLU and the conversion; the encoded input is stored unscaled.
// BF16 holds, for each hidden layer l >= 1, its bias as a width x 16 B operand
// (block bb; E4M3 with static scales one for every layer): K columns 10, 11, 12 carry the bias split into three BF16 parts
// (hi = bf16(b), mid = bf16(b - hi), lo = bf16(b - hi - mid); together the 24 bits
// of an FP32 significand), the other columns zero.  Against layer-0 input columns
// 80..95, whose columns 90..92 are constant ones and which no later layer
// overwrites, one K = 16 MMA writes exactly b into the accumulator; the layer's own
// MMAs then accumulate onto it.
constexpr int kBiasK = 16;
struct TcLayout {
    int width, hidden, k0, k0p, kh, khead, es;
    size_t w0, wh, wo, sw, bias, bb, stride;
    __host__ __device__ TcLayout(int w, int h, int k, bool f8)
        : width(w), hidden(h), k0(k), k0p(round_up(f8 ? k : k + 1, f8 ? 32 : 16)), kh(w),
          khead(w), es(f8 ? 1 : 2) {
        w0 = 0;
        wh = w0 + (size_t)w * k0p * es;
        wo = wh + (size_t)(h - 1) * w * kh * es;  // head: 16 x khead BF16 (both precisions)
        sw = wo + (size_t)16 * khead * 2;
        bias = sw + (f8 ? (size_t)h * w * 4 : 0);
        bb = (bias + (size_t)h * w * 4 + 16 + 127) / 128 * 128;  // FP32 biases b_0.. and bo, then bb
        const size_t end = bb + (size_t)(f8 ? h : h - 1) * w * kBiasK * 2;
        stride = (end + 127) / 128 * 128;
    }
};

// E4M3 (K-major, 8-bit): a core matrix is 8 rows x 16 elements.
__host__ __device__ inline size_t cm_offset8(int n, int k, int K) {
    return (size_t)(n >> 3) * (K * 8) + (size_t)(k >> 4) * 128 + (size_t)(n & 7) * 16 + (size_t)(k & 15);
}

// FP32 -> E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; no infinities),
// round to nearest even, saturating at +-448.  Inputs are finite.
uint8_t f2e4m3(float x) {
    const uint8_t sign = std::signbit(x) ? 0x80 : 0x00;
    const float a = std::fabs(x);
    if (a == 0.0f) return sign;
    if (a >= 448.0f) return sign | 0x7e;
    int e = 0;
    std::frexp(a, &e);
    int E = e - 1;                                   // 2^E <= a < 2^(E+1)
    if (E < -6) E = -6;                              // subnormal spacing 2^-9
    float r = std::nearbyint(a / std::ldexp(1.0f, E - 3));
    if (r >= 16.0f) {                                // rounded up into the next binade
        E += 1;
        r = 8.0f;
    }
    if (E > 8 || (E == 8 && r > 14.0f)) return sign | 0x7e;
    if (r < 8.0f) return sign | (uint8_t)r;          // subnormal (E == -6)
    return sign | (uint8_t)(((E + 7) << 3) | ((int)r - 8));
}

struct TcShared {
    uint64_t bar_w[kMaxGroups];
    uint64_t bar_m[kMaxGroups];
    int flag[kMaxGroups];
    uint32_t next_tile[kMaxGroups];  // dynamic schedule: tile grabbed by the group's thread 0
    uint32_t tmem_base;
};

// id / maxc: q = floor(id m / 2^32) with m = ceil(2^32 / maxc) is the quotient or one
// more (id m / 2^32 < id / maxc + 1); one compare fixes it.
__device__ __forceinline__ uint32_t div_maxc(const MlpArgs& g, uint32_t id) {
    if (g.maxc == 1) return id;
    uint32_t q = __umulhi(id, g.maxc_magic);
    if ((uint64_t)q * (uint32_t)g.maxc > id) --q;
    return q;
}

// Crossing of this row in tile t of `leaf` (0xffffffff past the leaf's end).
__device__ __forceinline__ uint32_t row_crossing(const MlpArgs& g, int leaf, uint32_t t, int ci) {
    const uint32_t first = __ldg(g.offsets + leaf) + (t - __ldg(g.tile_off + leaf)) * (uint32_t)(kTileRows >> g.lg_steps);
    const uint32_t c = first + (uint32_t)ci;
    return c < __ldg(g.offsets + leaf + 1) ? __ldg(g.order + c) : 0xffffffffu;
}

// Crossing interval and ray of crossing `id`.
__device__ __forceinline__ void crossing_data(const MlpArgs& g, uint32_t id, float2& xi, float o[3], float d[3]) {
    if (id == 0xffffffffu) return;
    const uint32_t ray = div_maxc(g, id);
    xi = __ldg(g.xing + id);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = __ldg(g.ro + 3 * (size_t)ray + a);
        d[a] = __ldg(g.rd + 3 * (size_t)ray + a);
    }
}

// TMEM columns per warpgroup: D (accumulator, up to 64 FP32 columns), A (up to 48
// columns = 96 BF16 features per lane), then the head accumulator (16 columns), which
// no layer writes: a tile's head result is read during the next tile's layers.
constexpr uint32_t kGroupCols = 128;
constexpr uint32_t kACol = 64;
constexpr uint32_t kHeadCol = 112;

// F8 = false: BF16 operands (kind::f16, K = 16 per MMA, 2 features per TMEM column).
// F8 = true:  E4M3 operands (kind::f8f6f4, K = 32 per MMA, 4 features per column).
//   ST = false: per-output-channel weight scales and a per-row activation scale: each
//               row is quantized as q = h * 448 / max|h_row| and the next accumulator
//               is rescaled by (max|h_row| / 448) * sw[n] before its bias is added.
//   ST = true:  static scales folded in at packing (see TcLayout): each layer's bias
//               enters as one BF16 MMA and the epilogue is ReLU and the conversion,
//               as for BF16.
// HC > 0: the number of hidden layers fixed at compile time, so the layer loop is
// unrolled and every layout offset is a constant (about 12 % faster on the 4 x 64
// network); HC = 0 reads it from the arguments.  The shapes of the workloads here
// (4 x 64 and 2 x 32) are instantiated with HC set.
template <int W>
constexpr int kHiddenFor = W == 64 ? 4 : 2;

// JIT: samples at the stratified jitter's fractions of their strata (g.jitter != 0), else
// at the midpoints.
template <int W, bool F8, bool ST, int HC, bool JIT>
__global__ void __launch_bounds__(128 * kMaxGroups, 1) k_mlp_tc(MlpArgs g, int n_groups, uint32_t tmem_cols) {
    const int hidden = HC > 0 ? HC : g.hidden;  // hidden layers (a compile-time constant when HC > 0)
    constexpr int K0 = (3 + 6 * kLX) + (3 + 6 * kLD);
    constexpr int KI = F8 ? 32 : 16;        // K per MMA instruction
    constexpr int EPW = F8 ? 4 : 2;         // elements per 32-bit TMEM column
    constexpr int K0P = round_up(F8 ? K0 : K0 + 1, KI);  // BF16: + the bias column
    static_assert(K0P / EPW <= (int)(kHeadCol - kACol), "layer-0 input does not fit the A columns");
    static_assert(W <= (int)kACol, "accumulator does not fit the D columns");
    extern __shared__ __align__(1024) uint8_t smem[];
    const TcLayout lay(W, hidden, K0, F8);
    TcShared* sh = reinterpret_cast<TcShared*>(smem + lay.stride * n_groups);

    const int grp = threadIdx.x >> 7;
    const int tig = threadIdx.x & 127;  // row within the tile = TMEM lane
    const int warp = threadIdx.x >> 5;
    const int q = warp & 3;             // TMEM lane quadrant of this warp
    const int bar_id = 1 + grp;
    // the group's leader (MMA issue, waits, weight loads) sits in warp grp % 4 of the
    // group, so the leaders of the 4 groups run on 4 different SM sub-partitions
    const bool leader = tig == 32 * (grp & 3);
    const bool leader_warp = warp == 4 * grp + (grp & 3);  // the leader's warp: issues the MMAs, converged

    if (threadIdx.x == 0) {
        for (int i = 0; i < n_groups; ++i) {
            mbar_init(smem_u32(&sh->bar_w[i]), 1);
            mbar_init(smem_u32(&sh->bar_m[i]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (grp < n_groups) {
        uint8_t* wbuf = smem + lay.stride * grp;
        const uint32_t w_addr = smem_u32(wbuf);
        const uint32_t bar_w = smem_u32(&sh->bar_w[grp]);
        const uint32_t bar_m = smem_u32(&sh->bar_m[grp]);
        const uint32_t lane = (uint32_t)(32 * q) << 16;
        const uint32_t d_col = tmem + kGroupCols * (uint32_t)grp;  // lane 0: MMA operand addresses
        const uint32_t a_col = d_col + kACol;
        const uint32_t d_row = d_col + lane;                          // this warp's lanes
        const uint32_t a_row = a_col + lane;
        const float* bias = reinterpret_cast<const float*>(wbuf + lay.bias);
        // shared-memory descriptors of the first core matrix of W0, W1 and the head; the
        // start-address field holds address / 16 in 14 bits, and every address here is
        // below 2^18, so later core matrices are these plus (offset / 16)
        const uint64_t desc_w0 = sdesc(w_addr + (uint32_t)lay.w0, (uint32_t)K0P * (F8 ? 8u : 16u));
        const uint64_t desc_wh = sdesc(w_addr + (uint32_t)lay.wh, (uint32_t)lay.kh * (F8 ? 8u : 16u));
        const uint64_t desc_wo = sdesc(w_addr + (uint32_t)lay.wo, (uint32_t)lay.khead * 16u);
        const uint64_t desc_bb = sdesc(w_addr + (uint32_t)lay.bb, (uint32_t)kBiasK * 16u);
        const uint8_t* wall = reinterpret_cast<const uint8_t*>(g.weights);
        if constexpr (F8 && ST) {
            // the BF16 constant-1 input columns of the bias MMAs (the K = 16 step at
            // A columns 40..47, ones at its columns 10..12), which no E4M3 operand
            // reaches (layer 0 fills A columns 0..23, later layers 0..W/4-1): written once
            const uint32_t c8[8] = {0u, 0u, 0u, 0u, 0u, pack_bf16(1.0f, 1.0f), pack_bf16(1.0f, 0.0f), 0u};
            static_assert((kOnesCol - kOnesStep) / 2 == 5, "ones at K-step columns 10..12");
            tmem_st8(a_row + (uint32_t)(kOnesStep / 2), c8);
            tmem_st_wait();
        }

        // ---- tile schedule of this worker (one warpgroup)
        const uint32_t t_end = g.t_end == 0xffffffffu ? (uint32_t)g.stats[1] : g.t_end;
        const uint32_t workers = gridDim.x * (uint32_t)n_groups;
        const uint32_t wid = blockIdx.x * (uint32_t)n_groups + (uint32_t)grp;
        uint32_t t_stop = t_end, t_step = 1, t_first;
        if (g.schedule == kSchedInterleaved) {
            t_first = g.t_begin + wid;
            t_step = workers;
        } else if (g.schedule == kSchedDynamic) {
            if (leader) sh->next_tile[grp] = atomicAdd(g.tile_counter, 1u) + g.t_begin;
            wg_bar(bar_id);
            t_first = sh->next_tile[grp];
        } else {  // contiguous (also each launch of the per-leaf loop)
            const uint32_t span = t_end > g.t_begin ? t_end - g.t_begin : 0u;
            const uint32_t per = (span + workers - 1) / workers;
            t_first = min(g.t_begin + wid * per, t_end);
            t_stop = min(t_first + per, t_end);
        }
        volatile int* flag = &sh->flag[grp];
        const int ci = tig / g.steps;          // crossing of this row within a tile
        const int j = tig - ci * g.steps;      // sample of this row within its crossing
        uint32_t ph_w = 0, ph_m = 0;
        int cur = -1;
        bool ok = true;
        // The head MMA of a tile runs while the group encodes its next tile.  Before that
        // tile's first MMA only the leader warp waits for it (the head reads D, which
        // layer 0 overwrites; the other warps see it complete through the layer-0
        // commit); its result, in columns no layer writes, is read with the layer-0
        // accumulator and activated and stored while a later layer's MMAs run.
        bool pending = false;   // head MMA issued, its completion not yet consumed
        bool have_out = false;  // a head result in TMEM waits to be read
        bool zpend = false;     // a head result in registers waits to be stored
        bool head_bad = false;  // the leader warp's wait for a head MMA ran out
        uint64_t slot_prev = ~0ull, slot_z = ~0ull;
        uint32_t zr[4] = {0u, 0u, 0u, 0u};
        auto store_head = [&]() {
            if (slot_z != ~0ull) {  // 4 x FP16; sigma saturates at the FP16 maximum
                uint2 o;
                o.x = pack_f16(fminf(softplus_f(__uint_as_float(zr[0])), 65504.0f), sigmoid_f(__uint_as_float(zr[1])));
                o.y = pack_f16(sigmoid_f(__uint_as_float(zr[2])), sigmoid_f(__uint_as_float(zr[3])));
                static_cast<uint2*>(g.slot_out)[slot_z] = o;
            }
            zpend = false;
        };
        // the whole group waits for the head MMA (a leaf change: it reads the weights)
        auto head_group_wait = [&]() -> bool {
            const bool okh = group_wait(bar_m, ph_m, bar_id, flag, leader);
            ph_m ^= 1u;
            pending = false;
            return okh;
        };

        // software pipeline: the crossing id of the next tile is fetched after the first
        // MMA of the current tile has been waited for, its interval and ray one layer later
        int leaf = t_first < t_stop ? leaf_of_tile(g.tile_off, g.n_leaves, t_first) : 0;
        uint32_t id = t_first < t_stop ? row_crossing(g, leaf, t_first, ci) : 0xffffffffu;
        float2 xi = make_float2(0.f, 0.f);
        float ro[3] = {0.f, 0.f, 0.f}, rd[3] = {0.f, 0.f, 0.f};
        crossing_data(g, id, xi, ro, rd);
        // the looked-up leaf's tile range and crossing range, kept in registers: they
        // change only at leaf changes, so a tile's lookup is one load (its crossing id)
        // instead of a chain of three (the small tables leave L1 under the streaming
        // loads of the intervals and rays)
        uint32_t lk_t0 = 0u, lk_t1 = 0u, lk_x0 = 0u, lk_x1 = 0u;
        auto leaf_ranges = [&](int lf) {
            lk_t0 = __ldg(g.tile_off + lf);
            lk_t1 = __ldg(g.tile_off + lf + 1);
            lk_x0 = __ldg(g.offsets + lf);
            lk_x1 = __ldg(g.offsets + lf + 1);
        };
        if (t_first < t_stop) leaf_ranges(leaf);

        for (uint32_t t = t_first; t < t_stop && ok;) {
            if (leaf != cur) {
                if (pending && !(ok = head_group_wait())) break;  // the head MMA still reads the weights
                wg_bar(bar_id);  // every row is done with the previous leaf's weights and biases
                if (leader) {
                    fence_proxy_async();
                    bulk_load(w_addr, wall + (size_t)leaf * lay.stride, (uint32_t)lay.stride, bar_w);
                }
                ok = group_wait(bar_w, ph_w, bar_id, flag, leader);
                ph_w ^= 1u;
                if (!ok) break;
                cur = leaf;
            }
            // ---- rebuild the sample of this row and encode it into its TMEM lane (layer-0 A)
            uint64_t slot = ~0ull;  // 64-bit: rays * cap may exceed 2^32
            float x[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
            if (id != 0xffffffffu) {
                const uint32_t ray = div_maxc(g, id);
                const uint32_t k = id - ray * (uint32_t)g.maxc;
                // steps is a power of two: the product by its reciprocal is the exact quotient
                const float delta = __fmul_rn(__fsub_rn(xi.y, xi.x), __frcp_rn((float)g.steps));
                const float u = JIT ? jit_fraction(g.jitter, jit_ray_key(g.jitter, ro, rd), (int)k, g.steps, j) : 0.5f;
                const float tj = __fadd_rn(xi.x, __fmul_rn(__fadd_rn((float)j, u), delta));
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    d[a] = rd[a];
                    x[a] = __fadd_rn(ro[a], __fmul_rn(tj, rd[a]));
                }
                slot = (uint64_t)ray * (uint64_t)g.cap + (uint64_t)(k * (uint32_t)g.steps + (uint32_t)j);
            }
            float s_a = 1.0f;  // FP8 only: this row's activation scale for the next MMA
            {
                constexpr int NX = 3 + 6 * kLX;
                float f[K0];
                encode_freq<kLX, 0>(x, f);
                encode_freq<kLD, NX>(d, f);
                if constexpr (!F8) {
                    static_assert(K0P == 96, "layer-0 input is stored in three 32-feature chunks");
                    store_chunk_perm<0>(a_row, f);
                    store_chunk_perm<1>(a_row, f);
                    store_chunk_perm<2>(a_row, f);
                } else {
                    static_assert(K0P == 96, "E4M3 layer-0 input is stored as 16 + 8 columns");
                    float inv = 1.0f;  // static scales: the features as they are
                    if constexpr (!ST) {  // this row's own scale
                        float m = 0.0f;
#pragma unroll
                        for (int i = 0; i < K0; ++i) m = fmaxf(m, fabsf(f[i]));
                        inv = m > 0.0f ? 448.0f / m : 0.0f;
                        s_a = m > 0.0f ? m / 448.0f : 0.0f;
                    }
                    uint32_t w[24];
#pragma unroll
                    for (int i = 0; i < 24; ++i) {
                        // features scaled in pairs; the padding past K0 is zero
                        float e[4];
#pragma unroll
                        for (int u = 0; u < 4; u += 2) {
                            const int f0 = 4 * i + u;
                            if (ST) {
#pragma unroll
                                for (int q = 0; q < 2; ++q) e[u + q] = f0 + q < K0 ? f[f0 + q < K0 ? f0 + q : 0] : 0.0f;
                            } else {
#pragma unroll
                                for (int q = 0; q < 2; ++q) {
                                    const int fq = f0 + q;
                                    e[u + q] = fq < K0 ? f[fq < K0 ? fq : 0] * inv : 0.0f;
                                }
                            }
                        }
                        w[i] = pack_e4m3x4(e[0], e[1], e[2], e[3]);
                    }
                    tmem_st16(a_row, w);
                    tmem_st8(a_row + 16u, w + 16);
                }
            }
            tmem_st_wait();
            tc_fence_before();
            wg_bar(bar_id);
            if (pending) {
                // on expiry the leader issues no more MMAs, so the group's next wait runs
                // out too and the whole group leaves through it
                if (leader_warp) {
                    const bool okw = mbar_wait_bounded(bar_m, ph_m);
                    if (!__all_sync(0xffffffffu, okw)) head_bad = true;
                }
                ph_m ^= 1u;
                pending = false;
            }

            int leaf_n = leaf;
            uint32_t id_n = 0xffffffffu;
            uint32_t t_next = t_stop;

            // ---- hidden layers; the last epilogue issues the head MMA
            int kin = K0P;
#pragma unroll
            for (int l = 0; l < hidden; ++l) {
                if (!ok) break;
                if (leader_warp && !head_bad) {
                    tc_fence_after();
                    // this layer's first weight core matrix, then 256 B (16 descriptor
                    // units) per K step
                    const uint64_t b_desc =
                        l == 0 ? desc_w0
                               : desc_wh + (uint64_t)(((size_t)(l - 1) * W * lay.kh * lay.es) >> 4);
                    if constexpr (F8) {
                        const uint32_t idd = idesc_e4m3(W);
                        // static scales: the layer's bias in accumulator units first (a BF16
                        // MMA of the constant-1 columns against its three-part operand),
                        // then the E4M3 steps accumulate onto it; per-row scales: every
                        // layer starts from zero (scales and bias in the epilogue)
                        if constexpr (ST)
                            mma_bf16_ts_warp(d_col, a_col + (uint32_t)(kOnesStep / 2),
                                             desc_bb + (uint64_t)(((size_t)l * W * kBiasK * 2) >> 4), idesc_bf16(W), 0u);
                        for (int kk = 0; kk < kin / KI; ++kk)
                            mma_e4m3_ts_warp(d_col, a_col + 8u * kk, b_desc + 16u * kk, idd, (ST || kk > 0) ? 1u : 0u);
                    } else {
                        const uint32_t idd = idesc_bf16(W);
                        // layer 0 starts from zero (its bias is folded in); a later layer
                        // first writes its bias (the constant-1 input columns against the
                        // layer's bias operand), then accumulates onto it
                        if (l > 0)
                            mma_bf16_ts_warp(d_col, a_col + (uint32_t)(kOnesStep / 2),
                                             desc_bb + (uint64_t)(((size_t)(l - 1) * W * kBiasK * 2) >> 4), idd, 0u);
                        for (int kk = 0; kk < kin / KI; ++kk)
                            mma_bf16_ts_warp(d_col, a_col + 8u * kk, b_desc + 16u * kk, idd,
                                             (kk > 0 || l > 0) ? 1u : 0u);
                    }
                    mma_commit_warp(bar_m);
                }
                // next tile of this worker, its leaf and this row's crossing id
                auto next_lookup = [&](uint32_t tn) {
                    t_next = tn;
                    if (t_next < t_stop) {
                        if (t_next >= lk_t1 || t_next < lk_t0) {  // another leaf (rare)
                            if (t_next - t <= 8u && t_next >= lk_t1) {
                                while (__ldg(g.tile_off + leaf_n + 1) <= t_next) ++leaf_n;
                            } else {
                                leaf_n = leaf_of_tile(g.tile_off, g.n_leaves, t_next);
                            }
                            leaf_ranges(leaf_n);
                        }
                        const uint32_t c = lk_x0 + (t_next - lk_t0) * (uint32_t)(kTileRows >> g.lg_steps) + (uint32_t)ci;
                        id_n = c < lk_x1 ? __ldg(g.order + c) : 0xffffffffu;
                    }
                };
                const bool dyn = g.schedule == kSchedDynamic;
                if (l == 0 && dyn && leader) sh->next_tile[grp] = atomicAdd(g.tile_counter, 1u) + g.t_begin;
                // The next tile's dependent loads are spread over the layers, each issued
                // while MMAs run and consumed a layer later: static schedules know the next
                // tile already, so its leaf and crossing id are looked up before the layer-0
                // wait; its interval and ray at layer l_xd; the previous tile's outputs are
                // stored at layer l_sh.
                const int l_xd = hidden > 1 ? 1 : 0;
                const int l_sh = hidden > 3 ? 3 : hidden - 1;
                if (!dyn && l == 0) next_lookup(t + t_step);
                if (!dyn && l > 0 && l == l_xd) crossing_data(g, id_n, xi, ro, rd);
                if (zpend && l == l_sh) store_head();
                // Every thread waits for the MMAs itself (the dynamic schedule's first
                // layer keeps the group barrier, which publishes the next tile).  A thread
                // whose wait ran out carries that to the group's next barrier, where the
                // whole group learns of it and leaves together.
                bool late = false;
                if (dyn && l == 0) ok = group_wait(bar_m, ph_m, bar_id, flag, leader);
                else late = !mbar_wait_bounded(bar_m, ph_m);
                ph_m ^= 1u;
                if (!ok) break;
                tc_fence_after();
                if (dyn && l == 0) next_lookup(sh->next_tile[grp]);  // published by the wait's barrier
                if ((dyn || l_xd == 0) && l == l_xd) crossing_data(g, id_n, xi, ro, rd);
                const float* b = bias + (size_t)l * W;
                const float* sw = reinterpret_cast<const float*>(wbuf + lay.sw) + (size_t)l * W;
                const bool last = l + 1 == hidden;
                // the previous tile's head result: loaded now, waited for with D below
                if (l == 0 && have_out) {
                    tmem_ld4_nowait(d_row + kHeadCol, zr);
                    slot_z = slot_prev;
                    have_out = false;
                    zpend = true;
                }
                // pre-activation of 4 consecutive columns c0..c0+3 of this row
                auto pre4 = [&](const float* v, int c0, float2& p01, float2& p23) {
                    if constexpr (F8 && !ST) {
                        const float4 bb = *reinterpret_cast<const float4*>(b + c0);
                        const float4 ss = *reinterpret_cast<const float4*>(sw + c0);
                        p01 = fma_f32x2(s_a, mul_f32x2(make_float2(v[0], v[1]), make_float2(ss.x, ss.y)),
                                        make_float2(bb.x, bb.y));
                        p23 = fma_f32x2(s_a, mul_f32x2(make_float2(v[2], v[3]), make_float2(ss.z, ss.w)),
                                        make_float2(bb.z, bb.w));
                    } else {  // the bias is already in the accumulator, the scales in the weights
                        p01 = make_float2(v[0], v[1]);
                        p23 = make_float2(v[2], v[3]);
                    }
                };
                if (!last) {
                    if constexpr (!F8) {
                        float vr[W];
                        tmem_ld_row<W>(d_row, vr);
#pragma unroll
                        for (int h = 0; h < W / 32; ++h) {
                            const float* v = vr + 32 * h;
                            uint32_t pk[16];
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                float2 p01, p23;
                                pre4(v + 4 * c, 32 * h + 4 * c, p01, p23);
                                pk[2 * c + 0] = pack_relu_bf16(p01.x, p01.y);
                                pk[2 * c + 1] = pack_relu_bf16(p23.x, p23.y);
                            }
                            tmem_st16(a_row + 16u * h, pk);
                        }
                    } else if constexpr (ST) {
                        // relu(acc) is the next layer's E4M3 input (its channel scales are
                        // this layer's output-channel scales, folded into the next weights)
                        float vr[W];
                        tmem_ld_row<W>(d_row, vr);
                        uint32_t pk[W / 4];
#pragma unroll
                        for (int c = 0; c < W / 4; ++c)
                            pk[c] = pack_relu_e4m3x4(vr[4 * c], vr[4 * c + 1], vr[4 * c + 2], vr[4 * c + 3]);
                        if constexpr (W / 4 == 16) tmem_st16(a_row, pk);
                        else tmem_st8(a_row, pk);
                    } else {
                        float hv[W];
#pragma unroll
                        for (int h = 0; h < W / 32; ++h) {
                            float v[32];
                            tmem_ld32(d_row + 32u * h, v);
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                float2 p01, p23;
                                pre4(v + 4 * c, 32 * h + 4 * c, p01, p23);
                                hv[32 * h + 4 * c + 0] = fmaxf(p01.x, 0.f);
                                hv[32 * h + 4 * c + 1] = fmaxf(p01.y, 0.f);
                                hv[32 * h + 4 * c + 2] = fmaxf(p23.x, 0.f);
                                hv[32 * h + 4 * c + 3] = fmaxf(p23.y, 0.f);
                            }
                        }
                        float m = 0.0f;
#pragma unroll
                        for (int n = 0; n < W; ++n) m = fmaxf(m, hv[n]);
                        const float inv = m > 0.0f ? 448.0f / m : 0.0f;
                        s_a = m > 0.0f ? m / 448.0f : 0.0f;
                        uint32_t pk[W / 4];
#pragma unroll
                        for (int i = 0; i < W / 4; ++i)
                            pk[i] = pack_e4m3x4(hv[4 * i] * inv, hv[4 * i + 1] * inv, hv[4 * i + 2] * inv,
                                                hv[4 * i + 3] * inv);
                        if constexpr (W / 4 == 16) tmem_st16(a_row, pk);
                        else tmem_st8(a_row, pk);
                    }
                    tmem_st_wait();
                    tc_fence_before();
                    if (wg_bar_any(bar_id, late)) {
                        ok = false;
                        break;
                    }
                    kin = lay.kh;
                } else {
                    // relu(h) as BF16 into this group's D columns (each 32-column block is
                    // read before it is overwritten), the head bias into D columns
                    // kHeadCol..+3, then the head MMA (16 x khead) accumulates onto it
                    if constexpr (!F8) {
                        float vr[W];
                        tmem_ld_row<W>(d_row, vr);
#pragma unroll
                        for (int h = 0; h < W / 32; ++h) {
                            const float* v = vr + 32 * h;
                            uint32_t pk[16];
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                pk[2 * c + 0] = pack_relu_bf16(v[4 * c + 0], v[4 * c + 1]);
                                pk[2 * c + 1] = pack_relu_bf16(v[4 * c + 2], v[4 * c + 3]);
                            }
                            tmem_st16(d_row + 16u * h, pk);
                        }
                    } else {  // E4M3: per-row scales need the channel scales and the bias
#pragma unroll
                        for (int h = 0; h < W / 32; ++h) {
                            float v[32];
                            uint32_t pk[16];
                            tmem_ld32(d_row + 32u * h, v);
#pragma unroll
                            for (int c = 0; c < 8; ++c) {
                                float2 p01, p23;
                                pre4(v + 4 * c, 32 * h + 4 * c, p01, p23);
                                pk[2 * c + 0] = pack_relu_bf16(p01.x, p01.y);
                                pk[2 * c + 1] = pack_relu_bf16(p23.x, p23.y);
                            }
                            tmem_st16(d_row + 16u * h, pk);
                        }
                    }
                    tmem_st4(d_row + kHeadCol, bias + (size_t)hidden * W);
                    tmem_st_wait();
                    tc_fence_before();
                    if (wg_bar_any(bar_id, late)) {
                        ok = false;
                        break;
                    }
                    if (leader_warp) {
                        tc_fence_after();
                        const uint32_t idd = idesc_bf16(16);
                        for (int kk = 0; kk < lay.khead / 16; ++kk)
                            mma_bf16_ts_warp(d_col + kHeadCol, d_col + 8u * kk, desc_wo + 16u * kk, idd, 1u);
                        mma_commit_warp(bar_m);
                    }
                    pending = true;
                    have_out = true;
                    slot_prev = slot;
                }
            }
            if (zpend) store_head();  // one hidden layer: stored after the head MMA issue
            leaf = leaf_n;
            id = id_n;
            t = t_next;
        }
        if (ok && pending) ok = head_group_wait();
        if (ok && have_out) {
            tc_fence_after();
            tmem_ld4_nowait(d_row + kHeadCol, zr);
            tmem_ld_wait();
            slot_z = slot_prev;
            store_head();
        }
        if (!ok && leader) atomicCAS(g.err, 0, kDevErrTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ---- BF16 network with two threads per sample row ------------------------------------
// The same network, tiles, weights and TMEM layout as k_mlp_tc<W, false, ...>, with
// 256 threads per warpgroup pair: warps 0-3 of a group handle the low half of every
// row (TMEM lane quadrant = warp % 4), warps 4-7 the high half.  A row's encoding is
// split by column half (kperm: each half from its own SFU anchors), and every epilogue
// reads, converts and stores W/2 of the row's accumulator columns per thread, so a
// tile's ALU work is spread over twice as many warps (more latency hidden per SM)
// without more TMEM.  The head MMA reads relu(h) from the A columns like a hidden
// layer; the next tile's encoding is computed while it runs and stored into A once it
// has completed.
constexpr int kTPR = 2;  // threads per sample row

__device__ __forceinline__ void bar_sync(int id, int n) {
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ bool group_wait_n(uint32_t bar, uint32_t phase, int bar_id, int n, volatile int* flag,
                                             bool leader) {
    if (leader) *flag = mbar_wait_bounded(bar, phase) ? 1 : 0;
    bar_sync(bar_id, n);
    return *flag != 0;
}

// N consecutive FP32 columns of this thread's TMEM lane (N = 16 or 32), one wait.
template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[N]) {
    uint32_t r[32];
    if constexpr (N == 32) {
        tmem_ld32_nowait(taddr, r);
    } else {
        static_assert(N == 16, "16 or 32 columns");
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr)
            : "memory");
    }
    tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = __uint_as_float(r[i]);
}

// N packed words into this thread's TMEM lane (N = 8 or 16).
template <int N>
__device__ __forceinline__ void tmem_st_words(uint32_t taddr, const uint32_t* w) {
    if constexpr (N == 16) tmem_st16(taddr, w);
    else tmem_st8(taddr, w);
}

// The layer-0 input half `half` of a row (48 features in kperm order) packed into 24
// words: half 0 = p_x, x octaves 0-4, p_d, d octaves 0-1; half 1 = x octaves 5-9,
// d octaves 2-3, the three constant-1 columns and zero padding.  The anchors are those of
// encode_freq (x at octaves 0 and 5, d at 0), so the features are bit-identical.
__device__ __forceinline__ void encode_half(int half, const float x[3], const float d[3], uint32_t (&w)[24]) {
    float f[48];
    if (half == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            f[a] = x[a];
            f[33 + a] = d[a];
        }
        encode_octaves<0, 5, 3>(x, f);
        encode_octaves<0, 2, 36>(d, f);
    } else {
        encode_octaves<5, 10, 0>(x, f);
        // d's octaves 2-3 from the anchor at octave 0, as the one-thread-per-row kernel
        // computes them (both kernels give the same features)
        float fd[24];
        encode_octaves<0, 4, 0>(d, fd);
#pragma unroll
        for (int i = 0; i < 12; ++i) f[30 + i] = fd[12 + i];
        f[42] = f[43] = f[44] = 1.0f;   // columns 90..92 (kperm)
#pragma unroll
        for (int i = 45; i < 48; ++i) f[i] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 24; ++i) w[i] = pack_bf16(f[2 * i], f[2 * i + 1]);
}

// MAXG: the most groups a launch of this instantiation uses (its register budget is
// 65536 / (256 MAXG) per thread: 64 at four groups, 80 at three).
template <int W, int HC, bool JIT, int MAXG>
__global__ void __launch_bounds__(128 * kTPR * MAXG, 1) k_mlp_tc2(MlpArgs g, int n_groups, uint32_t tmem_cols) {
    const int hidden = HC > 0 ? HC : g.hidden;
    constexpr int K0 = (3 + 6 * kLX) + (3 + 6 * kLD);
    constexpr int K0P = 96;
    static_assert(K0 + 1 <= K0P && kLX == 10 && kLD == 4, "kperm is laid out for gamma_10(x) ++ gamma_4(d)");
    constexpr int CPT = W / kTPR;  // accumulator columns per thread
    constexpr int GT = 128 * kTPR; // threads per group
    extern __shared__ __align__(1024) uint8_t smem[];
    const TcLayout lay(W, hidden, K0, false);
    TcShared* sh = reinterpret_cast<TcShared*>(smem + lay.stride * n_groups);

    const int grp = threadIdx.x / GT;
    const int tig = threadIdx.x % GT;
    const int wig = tig >> 5;            // warp within the group
    const int q = wig & 3;               // TMEM lane quadrant (global warp index % 4)
    const int half = wig >> 2;           // column half of the row
    const int row = 32 * q + (tig & 31); // sample row = TMEM lane
    const int warp = threadIdx.x >> 5;
    const int bar_id = 1 + grp;
    const bool leader = tig == 32 * (grp & 3);
    const bool leader_warp = wig == (grp & 3);  // the leader's warp: issues the MMAs, converged

    if (threadIdx.x == 0) {
        for (int i = 0; i < n_groups; ++i) {
            mbar_init(smem_u32(&sh->bar_w[i]), 1);
            mbar_init(smem_u32(&sh->bar_m[i]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (grp < n_groups) {
        uint8_t* wbuf = smem + lay.stride * grp;
        const uint32_t w_addr = smem_u32(wbuf);
        const uint32_t bar_w = smem_u32(&sh->bar_w[grp]);
        const uint32_t bar_m = smem_u32(&sh->bar_m[grp]);
        const uint32_t lane = (uint32_t)(32 * q) << 16;
        const uint32_t d_col = tmem + kGroupCols * (uint32_t)grp;
        const uint32_t a_col = d_col + kACol;
        const uint32_t d_row = d_col + lane;
        const uint32_t a_row = a_col + lane;
        const float* bias = reinterpret_cast<const float*>(wbuf + lay.bias);
        const uint32_t bias_s = smem_u32(bias);
        const uint64_t desc_w0 = sdesc(w_addr + (uint32_t)lay.w0, (uint32_t)K0P * 16u);
        const uint64_t desc_wh = sdesc(w_addr + (uint32_t)lay.wh, (uint32_t)lay.kh * 16u);
        const uint64_t desc_wo = sdesc(w_addr + (uint32_t)lay.wo, (uint32_t)lay.khead * 16u);
        const uint64_t desc_bb = sdesc(w_addr + (uint32_t)lay.bb, (uint32_t)kBiasK * 16u);
        const uint8_t* wall = reinterpret_cast<const uint8_t*>(g.weights);

        const uint32_t t_end = g.t_end == 0xffffffffu ? (uint32_t)g.stats[1] : g.t_end;
        const uint32_t workers = gridDim.x * (uint32_t)n_groups;
        const uint32_t wid = blockIdx.x * (uint32_t)n_groups + (uint32_t)grp;
        uint32_t t_stop = t_end, t_step = 1, t_first;
        if (g.schedule == kSchedInterleaved) {
            t_first = g.t_begin + wid;
            t_step = workers;
        } else if (g.schedule == kSchedDynamic) {
            if (leader) sh->next_tile[grp] = atomicAdd(g.tile_counter, 1u) + g.t_begin;
            bar_sync(bar_id, GT);
            t_first = sh->next_tile[grp];
        } else {
            const uint32_t span = t_end > g.t_begin ? t_end - g.t_begin : 0u;
            const uint32_t per = (span + workers - 1) / workers;
            t_first = min(g.t_begin + wid * per, t_end);
            t_stop = min(t_first + per, t_end);
        }
        volatile int* flag = &sh->flag[grp];
        const int ci = row / g.steps;
        const int j = row - ci * g.steps;
        uint32_t ph_w = 0, ph_m = 0;
        int cur = -1;
        bool ok = true;
        bool pending = false;   // head MMA issued, its completion not yet consumed
        bool have_out = false;  // a head result in TMEM waits to be read
        bool zpend = false;     // a head result in registers waits to be stored (half 0)
        uint64_t slot_prev = ~0ull, slot_z = ~0ull;
        uint32_t zr[4] = {0u, 0u, 0u, 0u};
        auto store_head = [&]() {
            if (slot_z != ~0ull) {
                uint2 o;
                o.x = pack_f16(fminf(softplus_f(__uint_as_float(zr[0])), 65504.0f), sigmoid_f(__uint_as_float(zr[1])));
                o.y = pack_f16(sigmoid_f(__uint_as_float(zr[2])), sigmoid_f(__uint_as_float(zr[3])));
                static_cast<uint2*>(g.slot_out)[slot_z] = o;
            }
            zpend = false;
        };

        int leaf = t_first < t_stop ? leaf_of_tile(g.tile_off, g.n_leaves, t_first) : 0;
        uint32_t id = t_first < t_stop ? row_crossing(g, leaf, t_first, ci) : 0xffffffffu;
        float2 xi = make_float2(0.f, 0.f);
        float ro[3] = {0.f, 0.f, 0.f}, rd[3] = {0.f, 0.f, 0.f};
        crossing_data(g, id, xi, ro, rd);

        for (uint32_t t = t_first; t < t_stop && ok;) {
            if (leaf != cur) {
                if (pending) {  // the head MMA still reads the weights
                    ok = group_wait_n(bar_m, ph_m, bar_id, GT, flag, leader);
                    ph_m ^= 1u;
                    pending = false;
                    if (!ok) break;
                }
                bar_sync(bar_id, GT);
                if (leader) {
                    fence_proxy_async();
                    bulk_load(w_addr, wall + (size_t)leaf * lay.stride, (uint32_t)lay.stride, bar_w);
                }
                ok = group_wait_n(bar_w, ph_w, bar_id, GT, flag, leader);
                ph_w ^= 1u;
                if (!ok) break;
                cur = leaf;
            }
            // ---- this row's sample and its half of the layer-0 input
            uint64_t slot = ~0ull;
            float x[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
            if (id != 0xffffffffu) {
                const uint32_t ray = div_maxc(g, id);
                const uint32_t k = id - ray * (uint32_t)g.maxc;
                const float delta = __fmul_rn(__fsub_rn(xi.y, xi.x), __frcp_rn((float)g.steps));
                const float u = JIT ? jit_fraction(g.jitter, jit_ray_key(g.jitter, ro, rd), (int)k, g.steps, j) : 0.5f;
                const float tj = __fadd_rn(xi.x, __fmul_rn(__fadd_rn((float)j, u), delta));
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    d[a] = rd[a];
                    x[a] = __fadd_rn(ro[a], __fmul_rn(tj, rd[a]));
                }
                slot = (uint64_t)ray * (uint64_t)g.cap + (uint64_t)(k * (uint32_t)g.steps + (uint32_t)j);
            }
            {
                uint32_t w[24];
                encode_half(half, x, d, w);
                if (pending) {  // the previous tile's head MMA reads the A columns
                    ok = group_wait_n(bar_m, ph_m, bar_id, GT, flag, leader);
                    ph_m ^= 1u;
                    pending = false;
                    if (!ok) break;
                    tc_fence_after();
                }
                tmem_st16(a_row + 24u * (uint32_t)half, w);
                tmem_st8(a_row + 24u * (uint32_t)half + 16u, w + 16);
            }
            tmem_st_wait();
            tc_fence_before();
            bar_sync(bar_id, GT);

            int leaf_n = leaf;
            uint32_t id_n = 0xffffffffu;
            uint32_t t_next = t_stop;
            int kin = K0P;
#pragma unroll
            for (int l = 0; l < hidden; ++l) {
                if (!ok) break;
                if (leader_warp) {
                    tc_fence_after();
                    const uint64_t b_desc = l == 0 ? desc_w0 : desc_wh + (uint64_t)(((size_t)(l - 1) * W * lay.kh * 2) >> 4);
                    const uint32_t idd = idesc_bf16(W);
                    for (int kk = 0; kk < kin / 16; ++kk)
                        mma_bf16_ts_warp(d_col, a_col + 8u * kk, b_desc + 16u * kk, idd, (kk > 0 || l > 0) ? 1u : 0u);
                    mma_commit_warp(bar_m);
                }
                auto next_lookup = [&](uint32_t tn) {
                    t_next = tn;
                    if (t_next < t_stop) {
                        if (t_next - t <= 8u) {
                            while (__ldg(g.tile_off + leaf_n + 1) <= t_next) ++leaf_n;
                        } else {
                            leaf_n = leaf_of_tile(g.tile_off, g.n_leaves, t_next);
                        }
                        id_n = row_crossing(g, leaf_n, t_next, ci);
                    }
                };
                const bool dyn = g.schedule == kSchedDynamic;
                if (l == 0 && dyn && leader) sh->next_tile[grp] = atomicAdd(g.tile_counter, 1u) + g.t_begin;
                const int l_xd = hidden > 2 ? 2 : hidden - 1;
                const int l_sh = hidden > 3 ? 3 : hidden - 1;
                if (!dyn && l == 0) next_lookup(t + t_step);
                if (!dyn && l > 0 && l == l_xd) crossing_data(g, id_n, xi, ro, rd);
                if (zpend && l == l_sh) store_head();
                ok = group_wait_n(bar_m, ph_m, bar_id, GT, flag, leader);
                ph_m ^= 1u;
                if (!ok) break;
                tc_fence_after();
                if (dyn && l == 0) next_lookup(sh->next_tile[grp]);
                if ((dyn || l_xd == 0) && l == l_xd) crossing_data(g, id_n, xi, ro, rd);
                const bool last = l + 1 == hidden;
                if (l == 0 && have_out && half == 0) {  // the previous tile's head result
                    tmem_ld4_nowait(d_row + kHeadCol, zr);
                    slot_z = slot_prev;
                    zpend = true;
                }
                if (l == 0) have_out = false;
                // relu of this thread's accumulator half, as BF16, into the next input's
                // A columns (also for the head, whose MMA reads the A columns)
                {
                    float v[CPT];
                    tmem_ld_cols<CPT>(d_row + (uint32_t)(CPT * half), v);
                    uint32_t pk[CPT / 2];
#pragma unroll
                    for (int c = 0; c < CPT / 2; ++c) pk[c] = pack_relu_bf16(v[2 * c], v[2 * c + 1]);
                    tmem_st_words<CPT / 2>(a_row + (uint32_t)(CPT / 2 * half), pk);
                }
                if (!last) {
                    // layer l + 1 accumulates onto its bias (this thread's columns)
                    tmem_st_wait();
                    tmem_st_bias<CPT>(d_row + (uint32_t)(CPT * half),
                                      bias_s + 4u * (uint32_t)((l + 1) * W + CPT * half));
                    tmem_st_wait();
                    tc_fence_before();
                    bar_sync(bar_id, GT);
                    kin = lay.kh;
                } else {
                    if (half == 0) tmem_st4(d_row + kHeadCol, bias + (size_t)hidden * W);
                    tmem_st_wait();
                    tc_fence_before();
                    bar_sync(bar_id, GT);
                    if (leader_warp) {
                        tc_fence_after();
                        const uint32_t idd = idesc_bf16(16);
                        for (int kk = 0; kk < lay.khead / 16; ++kk)
                            mma_bf16_ts_warp(d_col + kHeadCol, a_col + 8u * kk, desc_wo + 16u * kk, idd, 1u);
                        mma_commit_warp(bar_m);
                    }
                    pending = true;
                    have_out = true;
                    slot_prev = slot;
                }
            }
            if (zpend) store_head();  // one hidden layer: stored after the head MMA issue
            leaf = leaf_n;
            id = id_n;
            t = t_next;
        }
        if (ok && pending) {
            ok = group_wait_n(bar_m, ph_m, bar_id, GT, flag, leader);
            ph_m ^= 1u;
            pending = false;
        }
        if (ok && have_out && half == 0) {
            tc_fence_after();
            tmem_ld4_nowait(d_row + kHeadCol, zr);
            tmem_ld_wait();
            slot_z = slot_prev;
            store_head();
        }
        if (!ok && leader) atomicCAS(g.err, 0, kDevErrTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// Failure-detection self-test: waits, with the network kernel's bounded-wait helper,
// on an mbarrier phase that nothing completes; the wait runs out after `limit`
// cycles and the kernel records a timeout in the status word and returns.
__global__ void k_wait_selftest(unsigned long long limit, int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(smem_u32(&bar), 0, limit)) atomicCAS(err, 0, kDevErrTimeout);
}

template <int W, bool F8>
int max_groups_for(int hidden, int max_smem) {
    constexpr int K0 = (3 + 6 * kLX) + (3 + 6 * kLD);
    const TcLayout lay(W, hidden, K0, F8);
    int groups = (int)((max_smem - (int)sizeof(TcShared) - 64) / (int)lay.stride);
    return groups > kMaxGroups ? kMaxGroups : groups;
}

template <int W, bool F8>
cudaError_t prepare_w(int hidden, int* max_groups) {
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    *max_groups = max_groups_for<W, F8>(hidden, max_smem);
    if (*max_groups < 1) return cudaErrorInvalidConfiguration;
    const void* fns[8] = {(const void*)k_mlp_tc<W, F8, false, 0, false>,
                          (const void*)k_mlp_tc<W, F8, false, kHiddenFor<W>, false>,
                          (const void*)k_mlp_tc<W, F8, F8, 0, false>,
                          (const void*)k_mlp_tc<W, F8, F8, kHiddenFor<W>, false>,
                          (const void*)k_mlp_tc<W, F8, false, 0, true>,
                          (const void*)k_mlp_tc<W, F8, false, kHiddenFor<W>, true>,
                          (const void*)k_mlp_tc<W, F8, F8, 0, true>,
                          (const void*)k_mlp_tc<W, F8, F8, kHiddenFor<W>, true>};
    for (const void* f : fns) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// BF16 with two threads per row (k_mlp_tc2): the same shared memory per group.
template <int W>
cudaError_t prepare_w2() {
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const void* fns[8] = {(const void*)k_mlp_tc2<W, 0, false, 3>, (const void*)k_mlp_tc2<W, kHiddenFor<W>, false, 3>,
                          (const void*)k_mlp_tc2<W, 0, true, 3>, (const void*)k_mlp_tc2<W, kHiddenFor<W>, true, 3>,
                          (const void*)k_mlp_tc2<W, 0, false, 4>, (const void*)k_mlp_tc2<W, kHiddenFor<W>, false, 4>,
                          (const void*)k_mlp_tc2<W, 0, true, 4>, (const void*)k_mlp_tc2<W, kHiddenFor<W>, true, 4>};
    for (const void* f : fns) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int W>
cudaError_t launch_w2(cudaStream_t s, const MlpArgs& a, int grid) {
    constexpr int K0 = (3 + 6 * kLX) + (3 + 6 * kLD);
    const TcLayout lay(W, a.hidden, K0, false);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int groups = a.groups;
    if (groups < 1 || groups > max_groups_for<W, false>(a.hidden, max_smem)) return cudaErrorInvalidConfiguration;
    const uint32_t cols = 512;
    size_t smem = lay.stride * groups + sizeof(TcShared) + 64;
    if (smem < (size_t)max_smem / 2 + 1024) smem = (size_t)max_smem / 2 + 1024;
    const bool hc = a.hidden == kHiddenFor<W>;
    const int threads = 128 * kTPR * groups;
#define AMNERF_TC2(HC_, J_, G_) k_mlp_tc2<W, HC_, J_, G_><<<grid, threads, smem, s>>>(a, groups, cols)
    if (groups <= 3) {
        if (a.jitter) { if (hc) AMNERF_TC2(kHiddenFor<W>, true, 3); else AMNERF_TC2(0, true, 3); }
        else { if (hc) AMNERF_TC2(kHiddenFor<W>, false, 3); else AMNERF_TC2(0, false, 3); }
    } else {
        if (a.jitter) { if (hc) AMNERF_TC2(kHiddenFor<W>, true, 4); else AMNERF_TC2(0, true, 4); }
        else { if (hc) AMNERF_TC2(kHiddenFor<W>, false, 4); else AMNERF_TC2(0, false, 4); }
    }
#undef AMNERF_TC2
    return cudaGetLastError();
}

template <int W, bool F8>
cudaError_t launch_w(cudaStream_t s, const MlpArgs& a, int grid) {
    constexpr int K0 = (3 + 6 * kLX) + (3 + 6 * kLD);
    const TcLayout lay(W, a.hidden, K0, F8);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int groups = a.groups;
    if (groups < 1 || groups > max_groups_for<W, F8>(a.hidden, max_smem)) return cudaErrorInvalidConfiguration;
    const uint32_t cols = 512;  // kGroupCols per group: the whole TMEM, so one CTA per SM
    // at least half of the SM's shared memory, so that a second CTA can never become
    // resident on the SM and wait in tcgen05.alloc for columns this CTA holds
    size_t smem = lay.stride * groups + sizeof(TcShared) + 64;
    if (smem < (size_t)max_smem / 2 + 1024) smem = (size_t)max_smem / 2 + 1024;
    const bool hc = a.hidden == kHiddenFor<W>;
    const bool st = F8 && a.act_static;
#define AMNERF_TC(ST_, HC_, J_) k_mlp_tc<W, F8, ST_, HC_, J_><<<grid, 128 * groups, smem, s>>>(a, groups, cols)
    if (a.jitter) {
        if (st) { if (hc) AMNERF_TC(F8, kHiddenFor<W>, true); else AMNERF_TC(F8, 0, true); }
        else { if (hc) AMNERF_TC(false, kHiddenFor<W>, true); else AMNERF_TC(false, 0, true); }
    } else {
        if (st) { if (hc) AMNERF_TC(F8, kHiddenFor<W>, false); else AMNERF_TC(F8, 0, false); }
        else { if (hc) AMNERF_TC(false, kHiddenFor<W>, false); else AMNERF_TC(false, 0, false); }
    }
#undef AMNERF_TC
    return cudaGetLastError();
}

}  // namespace

size_t tc_leaf_stride_bytes(int width, int hidden, int k0, int prec) {
    if (prec != 1 && prec != 2) return 0;
    if (k0 != (3 + 6 * kLX) + (3 + 6 * kLD)) return 0;  // the encodings this build instantiates
    return TcLayout(width, hidden, k0, prec == 2).stride;
}

void pack_tc_leaf(const float* src, uint8_t* dst, int width, int hidden, int k0, int prec, const float* act_max) {
    const bool f8 = prec == 2;
    const bool stat = f8 && act_max;
    const TcLayout lay(width, hidden, k0, f8);
    std::memset(dst, 0, lay.stride);
    const float* w = src;
    float* bias = reinterpret_cast<float*>(dst + lay.bias);
    float* sw = reinterpret_cast<float*>(dst + lay.sw);
    auto bf_value = [](uint16_t b) {
        const uint32_t u = (uint32_t)b << 16;
        float f;
        std::memcpy(&f, &u, 4);
        return f;
    };
    // the bias b of output n as three BF16 parts in bias operand `chunk` (block bb)
    auto put_bias_operand = [&](int chunk, int n, float b) {
        uint8_t* base = dst + lay.bb + (size_t)chunk * width * kBiasK * 2;
        const uint16_t hi = f2bf(b);
        const float r1 = b - bf_value(hi);  // exact: b and hi share their leading bits
        const uint16_t mid = f2bf(r1);
        const uint16_t lo = f2bf(r1 - bf_value(mid));
        const uint16_t parts[3] = {hi, mid, lo};
        for (int i = 0; i < 3; ++i) std::memcpy(base + cm_offset(n, kOnesCol - kOnesStep + i, kBiasK), &parts[i], 2);
    };
    // E4M3, per-row activation scales: per-output-channel weight scales
    // s = max|W_row| / 448 (1 for a zero row); the epilogue rescales and adds the bias.
    // E4M3, static scales: layer l's E4M3 input q has one scale per input channel,
    // alpha_k (layer 0: 1, the encoded features are stored as they are: within +-448,
    // and E4M3's absolute error is smallest on the small ones).
    // Output channel n gets s_n = max(max_k |W[n,k] alpha_k|, act_max_(l+1)) / 448 (the
    // second term below the last hidden layer; 1 when both are 0), so that the stored
    // weights W alpha / s and the next layer's input relu(y) / s both stay within
    // +-448.  The accumulator is then (y - b) / s: the bias enters as b / s (a BF16
    // operand), the epilogue is relu and the conversion, the next layer's channel
    // scales are these s, and the head's BF16 weights take the last layer's s.
    std::vector<float> alpha((size_t)(k0 > width ? k0 : width), 1.0f), s_out((size_t)width);
    int kin = k0;
    for (int l = 0; l < hidden; ++l) {
        const int K = l == 0 ? lay.k0p : lay.kh;
        uint8_t* base = dst + (l == 0 ? lay.w0 : lay.wh + (size_t)(l - 1) * width * lay.kh * lay.es);
        const float* bl = w + (size_t)width * kin;  // this layer's biases
        for (int n = 0; n < width; ++n) {
            const float* row = w + (size_t)n * kin;
            if (f8) {
                float m = 0.0f;
                for (int k = 0; k < kin; ++k) m = std::fmax(m, std::fabs(row[k] * alpha[k]));
                float sc;
                if (stat) {
                    const float amax_next = l + 1 < hidden ? act_max[l + 1] : 0.0f;
                    sc = std::fmax(m, amax_next) / 448.0f;
                    if (!(sc > 0.0f)) sc = 1.0f;
                } else {
                    sc = m > 0.0f ? m / 448.0f : 1.0f;
                }
                s_out[n] = sc;
                sw[(size_t)l * width + n] = sc;
                for (int k = 0; k < kin; ++k) base[cm_offset8(n, k, K)] = f2e4m3(row[k] * alpha[k] / sc);
                bias[(size_t)l * width + n] = stat ? bl[n] / sc : bl[n];
                if (stat) put_bias_operand(l, n, bl[n] / sc);
            } else if (l == 0) {
                // layer 0 in the kernels' column order (kperm), its bias at the bias input
                for (int k = 0; k < K; ++k) {
                    const int c = kperm(k);
                    const float v = c >= 0 ? row[c] : (c == -1 ? bl[n] : 0.0f);
                    const uint16_t b = f2bf(v);
                    std::memcpy(base + cm_offset(n, k, K), &b, 2);
                }
                bias[n] = bl[n];
            } else {
                for (int k = 0; k < kin; ++k) {
                    const uint16_t b = f2bf(row[k]);
                    std::memcpy(base + cm_offset(n, k, K), &b, 2);
                }
                bias[(size_t)l * width + n] = bl[n];
                put_bias_operand(l - 1, n, bl[n]);  // hidden layers 1.. : block bb, chunk l - 1
            }
        }
        if (stat)
            for (int n = 0; n < width; ++n) alpha[n] = s_out[n];
        w += (size_t)width * kin + width;
        kin = width;
    }
    {  // head: rows 0..3 of a 16 x khead BF16 matrix (its bias stays FP32)
        uint8_t* hb = dst + lay.wo;
        for (int n = 0; n < 4; ++n) {
            for (int k = 0; k < width; ++k) {
                const uint16_t b = f2bf(w[(size_t)n * width + k] * (stat ? alpha[k] : 1.0f));
                std::memcpy(hb + cm_offset(n, k, lay.khead), &b, 2);
            }
        }
    }
    w += 4 * width;
    for (int n = 0; n < 4; ++n) bias[(size_t)hidden * width + n] = w[n];
}

cudaError_t launch_wait_selftest(cudaStream_t s, unsigned long long limit, int* err) {
    k_wait_selftest<<<1, 32, 0, s>>>(limit, err);
    return cudaGetLastError();
}

cudaError_t prepare_mlp_tc(int width, int hidden, int k0, int prec, int* max_groups) {
    if ((prec != 1 && prec != 2) || k0 != (3 + 6 * kLX) + (3 + 6 * kLD)) return cudaErrorNotSupported;
    const bool f8 = prec == 2;
    if (width == 64) {
        if (f8) return prepare_w<64, true>(hidden, max_groups);
        const cudaError_t e = prepare_w<64, false>(hidden, max_groups);
        return e != cudaSuccess ? e : prepare_w2<64>();
    }
    if (width == 32) {
        if (f8) return prepare_w<32, true>(hidden, max_groups);
        const cudaError_t e = prepare_w<32, false>(hidden, max_groups);
        return e != cudaSuccess ? e : prepare_w2<32>();
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_mlp_tc(cudaStream_t s, const MlpArgs& a, int grid, int prec) {
    const bool f8 = prec == 2;
    if (prec != 1 && prec != 2) return cudaErrorNotSupported;
    if (!f8 && a.width_split == 2) {  // BF16, two threads per sample row
        if (a.width == 64) return launch_w2<64>(s, a, grid);
        if (a.width == 32) return launch_w2<32>(s, a, grid);
        return cudaErrorInvalidValue;
    }
    if (a.width == 64) return f8 ? launch_w<64, true>(s, a, grid) : launch_w<64, false>(s, a, grid);
    if (a.width == 32) return f8 ? launch_w<32, true>(s, a, grid) : launch_w<32, false>(s, a, grid);
    return cudaErrorInvalidValue;
}

}  // namespace amnerf
