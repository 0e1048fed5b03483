// k_traverse.cu -- K-a: ray x KD-tree traversal and crossing emission
// (Sec. 3.5, Algorithm 1 "Traverse"; sampling of Algorithm 1 "Sampling" is defined
// on the emitted crossings and is evaluated where the samples are consumed).
//
// One thread per ray walks the tree front to back (near child first; a far child that
// the ray also crosses waits on a short stack in shared memory).  The crossing
// interval of a box is the slab test in a fixed FP32 operation order -- per axis
// t0 = (lo - o) * inv, t1 = (hi - o) * inv with inv = 1 / d correctly rounded, no
// fused multiply-add, NaN-ignoring min/max, entry = max over the axes of min(t0, t1)
// clamped at 0, exit = min of max(t0, t1) -- so the crossing list is reproducible bit
// for bit.  The walk evaluates it once, at the root, and then carries (entry, exit)
// down.  A child's box differs from its parent's only in one face, the split plane s
// on the split axis a, so its interval is the parent's with the axis-a pair replaced
// by the min/max of (t(lo_a), t(s)) (left child) or (t(s), t(hi_a)) (right child).
// Every face value t(f) = (f - o_a) * inv_a is the same rounded number wherever it is
// computed and is monotone in f (for inv_a = +-inf it is -inf, NaN or +inf by the side
// of o_a), so the child's axis-a entry is no smaller and its exit no larger than the
// parent's: the max (min) over the axes is max(parent entry, child axis entry)
// (min(parent exit, child axis exit)), the value the full slab test of the child
// gives.  For d_a >= +0 the left child's axis-a entry is the parent's and its exit is
// t(s), and the right child's entry is t(s) and its exit the parent's (mirrored for
// d_a <= -0), so with ts = t(s) the child the ray meets first spans (e, min(x, ts)) and
// the other (max(e, ts), x); a ts of NaN (d_a = 0 with o_a on the plane) leaves both
// children empty.  Only children with exit > entry are entered or pushed (with their
// interval), so empty boxes cost nothing, leaves need no test of their own, and an
// inner node costs one subtraction and one multiplication.  When both children are
// crossed, the ray meets the plane inside (e, x), after its origin, so the first child
// is the one on the origin's side: the near child.
// A leaf is emitted as (entry, exit) at crossing slot ray * maxc + k and counted in a
// per-CTA shared-memory histogram that is flushed to the per-leaf totals with one
// atomic per touched leaf.  Traversal stops after maxc crossings (whole crossings are
// kept under the cap).  When maxc is a multiple of 8 the crossings are written in whole
// 32-byte sectors (a group of four per store) and the network ids in 16-byte chunks,
// each ray's row of ids written whole: a partly written sector costs the memory a read
// of the rest of it when it leaves L2, and those scattered reads bounded the walk.
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
    const float hi[3] = {A.w, B.x, B.y};
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

// Threads per traversal CTA.  Shared memory, in this order: the per-CTA histogram;
// with whole-sector stores, each thread's current group of four crossings
// ([slot][thread] float2) and chunk of eight network ids ([pair][thread], two uint16
// per word); the
// stack of pending far children as [level][thread] (the (entry, exit) pairs, then the
// node ids).  The stack holds one entry per level of the tree at most (a far child is
// pushed only by an inner node on the current path), so it is sized by the tree's depth.
constexpr int kTravThreads = 256;

__host__ __device__ constexpr size_t trav_hist_bytes(int n_nets) { return ((size_t)n_nets * 4 + 15) & ~(size_t)15; }
__host__ __device__ constexpr size_t trav_stage_bytes(bool vec) {
    return vec ? (size_t)kTravThreads * (4 * sizeof(float2) + 8 * sizeof(uint16_t)) : 0;
}
__host__ __device__ constexpr size_t trav_smem_bytes(int n_nets, int depth, bool vec) {
    return trav_hist_bytes(n_nets) + trav_stage_bytes(vec) +
           (size_t)depth * kTravThreads * (sizeof(float2) + sizeof(uint16_t));
}

// Launch-wide arguments of the walk.
struct TravArgs {
    const float* ro;
    const float* rd;
    uint32_t n;
    const DevNode* nodes;
    const float2* walk;  // per node (split, meta as float bits): the walk's one 8-byte load
    int maxc;
    uint8_t* n_x;
    float2* xing;
    uint16_t* xleaf;
    uint32_t* counts;
    int* err;
    const uint64_t* mask;
    const uint8_t* fallback;
    float2* root_out;
    OccArgs occ;
    HierArgs hier;
    int depth;  // stack entries per thread: the tree's depth
    uint32_t* next_ray;  // persistent CTAs: kRayCounters ray counters (see the kernel)
};

// Features compiled into one instantiation of the walk, so that a render keeps in
// registers only the state its features use.
constexpr int kFHier = 1;  // adaptive hierarchical sampling (HCheck)
constexpr int kFMask = 2;  // proposal masks
constexpr int kFOcc = 4;   // empty-space skipping
constexpr int kFVec = 8;   // whole-sector stores (maxc a multiple of 8)

// Streaming accesses (each ray's inputs are read once, its crossing rows written once)
// bypass L1, which keeps the tree's nodes: the walk reads those about 35 times per ray.
__device__ __forceinline__ float ld_stream(const float* p) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_stream(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.global.L1::no_allocate.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// One ray's walk: its constants and the position of the walk.
struct RayWalk {
    float o[3], d[3], inv[3];
    float r0, bw;         // proposal: root interval start, bin width
    uint64_t kept_bins;   // proposal: kept depth bins
    uint64_t key;         // empty-space skipping: jitter key
    uint32_t r;
    size_t base;          // the ray's first crossing slot
    int nd, sp, cnt;
    float e, x;           // interval of node nd (exit > entry)
    bool masked;
};

// This thread's columns of the shared-memory areas.
struct TravSmem {
    uint32_t* cnt;   // the CTA's histogram
    float2* grp;     // group of four crossings, [slot * kTravThreads]
    uint16_t* chk;   // chunk of eight network ids: ids 2i, 2i+1 in word [i * kTravThreads] (two halves)
    float2* ex;      // pending (entry, exit), [level * kTravThreads]
    uint16_t* nd;    // pending node ids, [level * kTravThreads]
};

// Loads ray r and intersects the root; returns false when the ray misses the tree
// (its crossing count is written then).
template <int F>
__device__ __forceinline__ bool walk_init(const TravArgs& t, RayWalk& w, uint32_t r) {
    w.r = r;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w.o[a] = ld_stream(t.ro + 3 * (size_t)r + a);
        w.d[a] = ld_stream(t.rd + 3 * (size_t)r + a);
        w.inv[a] = __frcp_rn(w.d[a]);
    }
    float r0 = 0.f, r1 = 0.f;
    const float4 A = __ldg(&t.nodes[0].a);
    const float4 B = __ldg(&t.nodes[0].b);
    const bool hit = slab(A, B, w.o, w.inv, r0, r1);
    if (!hit) r0 = r1 = 0.f;
    if (t.root_out) t.root_out[r] = make_float2(r0, r1);
    if (F & kFMask) {
        w.masked = !__ldg(t.fallback + r);
        w.kept_bins = w.masked ? __ldg(t.mask + r) : 0ull;
        w.r0 = r0;
        w.bw = __fmul_rn(__fsub_rn(r1, r0), 0.015625f);  // bin width (t1 - t0) / 64
    }
    if (F & kFOcc) w.key = t.occ.jitter ? jit_ray_key(t.occ.jitter, w.o, w.d) : 0ull;
    w.base = (size_t)r * (size_t)t.maxc;
    w.nd = 0;
    w.sp = 0;
    w.cnt = 0;
    w.e = r0;
    w.x = r1;
    if (!hit) t.n_x[r] = 0;
    return hit;
}

__device__ __forceinline__ float sel3(int a, const float v[3]) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); }

// The staged group of four crossings as one 32-byte sector at dst (32-byte aligned).
__device__ __forceinline__ void store_group(float2* dst, const TravSmem& sm) {
    const float2 a = sm.grp[0], b = sm.grp[kTravThreads], c = sm.grp[2 * kTravThreads],
                 d = sm.grp[3 * kTravThreads];
    float4* p = reinterpret_cast<float4*>(dst);
    st_stream(p, __float_as_uint(a.x), __float_as_uint(a.y), __float_as_uint(b.x), __float_as_uint(b.y));
    st_stream(p + 1, __float_as_uint(c.x), __float_as_uint(c.y), __float_as_uint(d.x), __float_as_uint(d.y));
}

// The staged chunk of eight network ids as one 16-byte store at dst (16-byte aligned).
__device__ __forceinline__ void store_chunk(uint16_t* dst, const TravSmem& sm) {
    uint32_t v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        v[i] = reinterpret_cast<const uint32_t*>(sm.chk)[i * kTravThreads];
    st_stream(dst, v[0], v[1], v[2], v[3]);
}

// Emits node nd as the ray's next crossing (after the proposal and empty-space
// rules); returns false when the ray has reached maxc crossings.  kFVec: the crossings
// are collected in shared memory per group of four slots and written as one whole
// 32-byte sector, the network ids per chunk of eight slots (16 bytes), so that no
// sector of the crossing list is left partly written (see walk_flush).
template <int F>
__device__ __forceinline__ bool walk_emit(const TravArgs& t, RayWalk& w, const TravSmem& sm, uint32_t meta,
                                          int axis) {
    if ((F & kFMask) && w.masked && !overlaps_kept(w.kept_bins, w.r0, w.bw, w.e, w.x)) return true;
    if ((F & kFOcc) && !crossing_occupied(t.occ, w.o, w.d, w.key, w.e, w.x, w.cnt)) return true;
    const uint32_t net = (!(F & kFHier) || axis < 0) ? meta >> 2 : (uint32_t)__ldg(t.hier.node_net + w.nd);
    const size_t base = w.base;
    if (F & kFVec) {
        const int j = w.cnt & 3, k = w.cnt & 7;
        sm.grp[j * kTravThreads] = make_float2(w.e, w.x);
        sm.chk[2 * (k >> 1) * kTravThreads + (k & 1)] = (uint16_t)net;
        if (j == 3) store_group(t.xing + base + (w.cnt - 3), sm);
        if (k == 7) store_chunk(t.xleaf + base + (w.cnt - 7), sm);
    } else {
        t.xing[base + w.cnt] = make_float2(w.e, w.x);
        t.xleaf[base + w.cnt] = (uint16_t)net;
    }
    atomicAdd(&sm.cnt[net], 1u);
    return ++w.cnt < t.maxc;
}

// kFVec: writes the ray's last, partly filled group and chunk, and zero chunks of
// network ids to the end of its row: rows of ids are 16-byte aligned but share 32-byte
// sectors with the next ray's row, so each row is written whole.  Slots at and past
// the ray's crossing count hold no crossing (their contents are unspecified).
template <int F>
__device__ __forceinline__ void walk_flush(const TravArgs& t, const RayWalk& w, const TravSmem& sm) {
    if (!(F & kFVec) || w.cnt == 0) return;
    const size_t base = w.base;
    if (w.cnt & 3) store_group(t.xing + base + (w.cnt & ~3), sm);
    int c = w.cnt >> 3;
    if (w.cnt & 7) store_chunk(t.xleaf + base + 8 * c++, sm);
    uint4* q = reinterpret_cast<uint4*>(t.xleaf + base);
    for (; c < (t.maxc >> 3); ++c) st_stream(q + c, 0u, 0u, 0u, 0u);
}

// Moves to the children of inner node nd (split plane s on axis a).  The plane cuts
// (e, x) at ts = (s - o_a) * inv_a: the child the ray meets first is (e, min(x, ts)),
// the other (max(e, ts), x) -- the left child comes first for d_a >= +0, the right one
// for d_a <= -0 -- and a ts of NaN (a ray inside the plane) crosses neither.  These are
// the children's slab intervals (see the header).  As x > e, the first child is
// crossed iff ts > e and the other iff x > ts (a NaN fails both): when both are, the
// plane splits (e, x) at ts; when one is, its interval is (e, x) itself.  Enters the
// first crossed child and pushes the other when both are; returns false when neither is.
__device__ __forceinline__ bool walk_descend(const TravArgs& t, RayWalk& w, const TravSmem& sm, float split,
                                             uint32_t meta, int axis) {
    const float oa = sel3(axis, w.o), ia = sel3(axis, w.inv);
    const float ts = __fmul_rn(__fsub_rn(split, oa), ia);
    const bool ok1 = ts > w.e;
    const bool ok2 = w.x > ts;
    const bool neg = (__float_as_uint(ia) >> 31) != 0u;
    const int left = w.nd + 1, right = (int)(meta >> 2);
    const int c1 = neg ? right : left, c2 = neg ? left : right;
    if (ok1 && ok2) {
        if (w.sp >= t.depth) {  // unreachable: one entry per level at most; recorded, never trapped
            atomicCAS(t.err, 0, kDevErrStack);
            return false;
        }
        sm.nd[w.sp * kTravThreads] = (uint16_t)c2;
        sm.ex[w.sp * kTravThreads] = make_float2(ts, w.x);
        ++w.sp;
        w.x = ts;
    }
    w.nd = ok1 ? c1 : c2;
    return ok1 || ok2;
}

// Pops the next pending child; returns false when none is left.
__device__ __forceinline__ bool walk_pop(RayWalk& w, const TravSmem& sm) {
    if (w.sp == 0) return false;
    --w.sp;
    w.nd = sm.nd[w.sp * kTravThreads];
    const float2 ex = sm.ex[w.sp * kTravThreads];
    w.e = ex.x;
    w.x = ex.y;
    return true;
}

// Whether node nd is emitted rather than descended: a leaf, or (kFHier) an inner node
// whose extent along its split axis is not above lod x entry (HCheck).
template <int F>
__device__ __forceinline__ bool walk_stops(const TravArgs& t, const RayWalk& w, int axis) {
    if (axis < 0) return true;
    if (!(F & kFHier)) return false;
    const float* f = reinterpret_cast<const float*>(&t.nodes[w.nd]);
    const float lo_a = __ldg(f + axis);
    const float hi_a = __ldg(f + 3 + axis);
    return !(__fsub_rn(hi_a, lo_a) > __fmul_rn(t.hier.lod, w.e));
}

// One thread per ray; each loop iteration visits one node (emits it or moves to its
// children), then takes the next pending child when the walk below it is done.  With
// ray counters the CTAs are persistent (as many as fit on the SMs): each warp takes
// its next 32 consecutive rays from its counter when its current ones are done, so a
// CTA waits on its slowest ray once, at the end, instead of once per 256 rays (0.415
// against 0.463 ms at 800x800 x 8).  Six CTAs per SM (40 registers) when the shared
// memory allows it.
template <int F>
__global__ void __launch_bounds__(kTravThreads, 6) k_traverse(const TravArgs t, int n_leaves) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    TravSmem sm;
    unsigned char* p = s_raw;
    sm.cnt = reinterpret_cast<uint32_t*>(p);
    p += trav_hist_bytes(n_leaves);
    sm.grp = reinterpret_cast<float2*>(p) + threadIdx.x;
    if (F & kFVec) p += (size_t)4 * kTravThreads * sizeof(float2);
    sm.ex = reinterpret_cast<float2*>(p) + threadIdx.x;
    p += (size_t)t.depth * kTravThreads * sizeof(float2);
    sm.chk = reinterpret_cast<uint16_t*>(p) + 2 * threadIdx.x;
    if (F & kFVec) p += (size_t)8 * kTravThreads * sizeof(uint16_t);
    sm.nd = reinterpret_cast<uint16_t*>(p) + threadIdx.x;
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) sm.cnt[i] = 0u;
    __syncthreads();
    const bool pers = t.next_ray != nullptr;
    const uint32_t ctr = (threadIdx.x >> 5) % kRayCounters;  // this warp's counter
    while (true) {
        uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
        if (pers) {  // the next 32-ray block b of this warp's counter (b % kRayCounters == ctr)
            uint32_t v = 0;
            if ((threadIdx.x & 31) == 0) v = atomicAdd(t.next_ray + 32 * ctr, 1u);
            v = __shfl_sync(0xffffffffu, v, 0);
            const uint64_t r0 = ((uint64_t)v * kRayCounters + ctr) * 32u;
            if (r0 >= t.n) break;
            r = (uint32_t)r0 + (threadIdx.x & 31);
        }
        RayWalk w;
        if (r < t.n && walk_init<F>(t, w, r)) {
            while (true) {
                const float2 sm2 = __ldg(t.walk + w.nd);  // split, meta
                const uint32_t meta = __float_as_uint(sm2.y);
                const int axis = (int)(meta & 3u) - 1;
                bool next;
                if (walk_stops<F>(t, w, axis)) {
                    if (!walk_emit<F>(t, w, sm, meta, axis)) break;
                    next = walk_pop(w, sm);
                } else {
                    next = walk_descend(t, w, sm, sm2.x, meta, axis) || walk_pop(w, sm);
                }
                if (!next) break;
            }
            walk_flush<F>(t, w, sm);
            t.n_x[r] = (uint8_t)w.cnt;
        }
        if (!pers) break;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_leaves; i += blockDim.x) {
        const uint32_t c = sm.cnt[i];
        if (c) atomicAdd(&t.counts[i], c);
    }
}

using TravKernel = void (*)(const TravArgs, int);

// The sixteen feature combinations, indexed by their flags.
template <int... Fs>
struct TravTable {
    static constexpr TravKernel k[sizeof...(Fs)] = {k_traverse<Fs>...};
};
using Trav16 = TravTable<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15>;

}  // namespace

cudaError_t prepare_traverse() {
    const int smem = (int)trav_smem_bytes(kMaxNets, kMaxDepth, true);
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 16 && e == cudaSuccess; ++f)
        e = cudaFuncSetAttribute(Trav16::k[f], cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t launch_traverse(cudaStream_t s, const float* ro, const float* rd, uint32_t n, const DevNode* nodes,
                            const float2* walk, int maxc, uint8_t* n_x, float2* xing, uint16_t* xleaf,
                            uint32_t* counts, int n_leaves, int* err, const uint64_t* mask, const uint8_t* fallback,
                            float2* root_out, const OccArgs& occ, const HierArgs& hier, int depth,
                            uint32_t* ray_counter) {
    if (n == 0) return cudaSuccess;
    if (n_leaves < 1 || n_leaves > kMaxNets || depth < 0 || depth > kMaxDepth) return cudaErrorInvalidValue;
    TravArgs t{ro, rd, n, nodes, walk, maxc, n_x, xing, xleaf, counts, err, mask, fallback, root_out, occ, hier,
               depth > 0 ? depth : 1, ray_counter};
    const int f = ((hier.lod > 0.0f && hier.node_net) ? kFHier : 0) | (mask ? kFMask : 0) |
                  (occ.grid ? kFOcc : 0) | ((maxc & 7) == 0 ? kFVec : 0);
    const TravKernel kern = Trav16::k[f];
    unsigned blocks = (n + kTravThreads - 1) / kTravThreads;
    const size_t smem = trav_smem_bytes(n_leaves, t.depth, (f & kFVec) != 0);
    if (t.next_ray) {  // persistent: as many CTAs as are resident at once
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kTravThreads, (int)smem);
        if (e != cudaSuccess) return e;
        const unsigned cap = (unsigned)(sms * (per > 0 ? per : 1));
        blocks = blocks < cap ? blocks : cap;
    }
    kern<<<blocks, kTravThreads, smem, s>>>(t, n_leaves);
    return cudaGetLastError();
}

}  // namespace amnerf
