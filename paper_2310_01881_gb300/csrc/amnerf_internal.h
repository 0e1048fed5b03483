// amnerf_internal.h -- private declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/amnerf.h"

namespace amnerf {

// Device tree node: eight floats, (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z, split, meta)
// as two float4 (split and meta share one 8-byte load), meta bits: [0,2) axis + 1
// (0 = leaf), [2,32) right-child index (inner) or leaf id (leaf).  Left child = node + 1.
struct DevNode {
    float4 a, b;
};

constexpr int kTileRows = 128;   // samples per network tile (tcgen05 M)
constexpr int kMaxLeaves = 4096; // 2^12 leaves at depth 12
constexpr int kMaxNets = 2 * kMaxLeaves;  // one network per node: leaves, then inner nodes (< 8192)
constexpr int kMaxDepth = 12;
constexpr int kStackDepth = 16;  // traversal stack (depth + 1 entries suffice)
// Persistent kernels take their rays 32 at a time from kRayCounters counters, one per
// 128-byte line (warp w of a CTA uses counter w % kRayCounters, which hands out the
// 32-ray blocks b with b % kRayCounters == its index): a single counter's atomics
// limited large batches of short rays.
constexpr int kRayCounters = 8;
constexpr size_t kRayCounterBytes = 128 * kRayCounters;

#ifdef __CUDACC__
// ---- stratified jitter of the sample positions (Sec. 3.5: samples drawn at random within each interval) --
// u = (splitmix64 finaliser of key + 0x9e3779b97f4a7c15 (k steps + j + 1)) >> 40, over
// 2^24, for sample j of crossing k; the ray's key folds the bit patterns of (o.x, o.y),
// (o.z, d.x), (d.y, d.z) into the seed with three finalisations.  Seed 0: u = 1/2.
// The finaliser is splitmix64's (Steele, Lea and Flood, 2014).
__device__ __forceinline__ uint64_t jit_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t jit_ray_key(uint64_t seed, const float o[3], const float d[3]) {
    uint64_t k = jit_mix64(seed ^ ((uint64_t)__float_as_uint(o[0]) | ((uint64_t)__float_as_uint(o[1]) << 32)));
    k = jit_mix64(k ^ ((uint64_t)__float_as_uint(o[2]) | ((uint64_t)__float_as_uint(d[0]) << 32)));
    return jit_mix64(k ^ ((uint64_t)__float_as_uint(d[1]) | ((uint64_t)__float_as_uint(d[2]) << 32)));
}

// Fraction of its stratum at which sample j of crossing k sits (exact in FP32).
__device__ __forceinline__ float jit_fraction(uint64_t seed, uint64_t key, int k, int steps, int j) {
    if (seed == 0) return 0.5f;
    const uint64_t z = jit_mix64(key + 0x9e3779b97f4a7c15ull * (uint64_t)(k * steps + j + 1));
    return (float)(uint32_t)(z >> 40) * (1.0f / 16777216.0f);
}
#endif

// Error word values written by kernels (first error wins).
constexpr int kDevErrTimeout = 1;
constexpr int kDevErrStack = 2;
constexpr int kDevErrBounds = 3;

// ---- kernels (enqueue only; return cudaGetLastError) ------------------------------

// Empty-space skipping (grid == nullptr: off): the guidance grid (x fastest, G^3),
// the cell of p on axis a is floor((p - lo[a]) * sc[a]) clamped; occupied when the
// density > thr.  Samples are placed as in the sampling step (steps, jitter).
struct OccArgs {
    const float* grid = nullptr;
    int G = 0;
    float lo[3] = {0.f, 0.f, 0.f}, sc[3] = {0.f, 0.f, 0.f};
    float thr = 0.f;
    int steps = 8;
    uint64_t jitter = 0;
};

// Adaptive hierarchical sampling (lod <= 0 or node_net == nullptr: leaves only): an
// inner node is descended only while its extent along its split axis exceeds lod x the
// ray's entry distance into it; otherwise it is one crossing of network node_net[node].
struct HierArgs {
    float lod = 0.f;
    const uint16_t* node_net = nullptr;
};

// K-a: traversal + crossing list + per-network crossing histogram (n_nets counters);
// walk: (split, meta) of every node, the part of a node the walk below the root reads;
// depth: the tree's depth (0 .. kMaxDepth), which bounds the walk's stack;
// ray_counter: kRayCounterBytes zeroed before the launch, from which persistent CTAs
// take their rays (nullptr: one CTA per 256 rays).
cudaError_t launch_traverse(cudaStream_t s, const float* ro, const float* rd, uint32_t n, const DevNode* nodes,
                            const float2* walk, int maxc, uint8_t* n_x, float2* xing, uint16_t* xleaf, uint32_t* counts,
                            int n_nets, int* err, const uint64_t* mask = nullptr,
                            const uint8_t* fallback = nullptr, float2* root_out = nullptr,
                            const OccArgs& occ = OccArgs(), const HierArgs& hier = HierArgs(),
                            int depth = kMaxDepth, uint32_t* ray_counter = nullptr);

// K-b: exclusive scans (crossings and network tiles per leaf) and the grouped scatter.
// acc (may be NULL) accumulates (crossings, tiles) over the waves of one render.
cudaError_t launch_scan(cudaStream_t s, const uint32_t* counts, int n_leaves, int cpt, uint32_t* offsets,
                        uint32_t* tile_off, uint32_t* cursor, uint64_t* stats, uint64_t* acc = nullptr);
cudaError_t launch_scatter(cudaStream_t s, const uint8_t* n_x, const uint16_t* xleaf, uint32_t n_rays, int maxc,
                           uint32_t* cursor, uint32_t* order, int n_leaves);
// One wave: crossing k of ray r takes part when k_lo <= k < min(n_x[r], k_hi) and
// alive[r] (alive == NULL: every ray).  count: only the per-leaf totals, added to
// cursor (zeroed by the caller); else the grouped scatter from the scanned cursor.
cudaError_t launch_scatter_wave(cudaStream_t s, bool count, const uint8_t* n_x, const uint16_t* xleaf,
                                uint32_t n_rays, int maxc, int k_lo, int k_hi, const uint8_t* alive, uint32_t* cursor,
                                uint32_t* order, int n_leaves);
// Kernel attributes of the grouping kernels (their shared memory grows with the number
// of networks, up to kMaxNets); call once per device before a render.
cudaError_t prepare_group();
// Kernel attributes of the traversal (its shared memory holds a histogram over up to
// kMaxNets networks and the stack of pending far children); call once per device.
cudaError_t prepare_traverse();
// Crossings given by the caller instead of the traversal (render from crossings): copied
// into the crossing list, counted per network; bad ids / counts set kDevErrBounds.
cudaError_t launch_load_crossings(cudaStream_t s, const uint8_t* n_x_in, const uint16_t* leaf_in, const float* t_in,
                                  const float* t_out, uint32_t n_rays, int maxc, int n_nets, uint8_t* n_x,
                                  float2* xing, uint16_t* xleaf, uint32_t* counts, int* err);

// Tile schedules of the network kernels (values of amnerf_tuning.schedule).
constexpr int kSchedContiguous = 0;   // worker w takes tiles [w * per, (w + 1) * per)
constexpr int kSchedInterleaved = 1;  // worker w takes tiles w, w + workers, ...
constexpr int kSchedDynamic = 2;      // workers take the next tile from a device counter
constexpr int kSchedPerLeaf = 3;      // one launch per leaf (host loop; baseline)

// K-c: per-leaf networks over leaf-grouped tiles of 128 samples.
struct MlpArgs {
    const uint32_t* order;
    const uint32_t* offsets;
    const uint32_t* tile_off;
    const uint64_t* stats;  // [1] = total tiles
    uint32_t* tile_counter; // dynamic schedule: next free tile (zeroed before the launch)
    uint32_t t_begin, t_end;// tile range of this launch (t_end == 0xffffffff: up to stats[1])
    int schedule;           // kSched*
    int groups;             // tcgen05 kernel: warpgroups per CTA (1..4)
    int width_split;        // tcgen05 BF16: threads per sample row, each with width / split columns (1, 2)
    int n_leaves;
    const float2* xing;
    const float* ro;
    const float* rd;
    const void* weights;    // packed per leaf, layout depends on precision
    size_t leaf_stride;     // bytes per leaf
    int width, hidden, lx, ld, k0;
    int steps, maxc, cap;
    uint32_t maxc_magic;    // ceil(2^32 / maxc) (maxc >= 2): id / maxc by multiply-high (see div_maxc)
    int lg_steps;           // log2(steps)
    void* slot_out;         // per-sample outputs: float4 (FP32 path) or 4 x FP16 (tensor-core paths)
    int* err;
    float* amax;            // FP32 path, calibration: per leaf x hidden layer, max |input of layer l| (or NULL)
    int act_static;         // E4M3 path: static per-leaf, per-layer activation scales folded into the blob
    uint64_t jitter;        // sample placement: 0 = stratum midpoints, else the stratified jitter's seed
};
cudaError_t launch_mlp_simt(cudaStream_t s, const MlpArgs& a, int grid);
cudaError_t launch_mlp_tc(cudaStream_t s, const MlpArgs& a, int grid, int prec);
// Kernel attributes (dynamic shared memory) and the largest group count the tcgen05
// kernel supports for this shape; called at weight-load time, outside any capture.
cudaError_t prepare_mlp_tc(int width, int hidden, int k0, int prec, int* max_groups);
cudaError_t prepare_mlp_simt(int width, int hidden, int k0);
// Failure-detection self-test of the bounded device waits (see amnerf_selftest_wait).
cudaError_t launch_wait_selftest(cudaStream_t s, unsigned long long limit, int* err);
size_t tc_leaf_stride_bytes(int width, int hidden, int k0, int prec);
// act_max (E4M3 only, may be NULL): per hidden layer l, the largest |input of layer l|
// of this leaf; non-NULL folds static activation scales into the packed leaf.
void pack_tc_leaf(const float* src, uint8_t* dst, int width, int hidden, int k0, int prec, const float* act_max);
size_t simt_leaf_stride_floats(int width, int hidden, int k0);

// K-d: per-ray compositing.
// slot_half: slot_out holds 4 x FP16 per sample (sigma, r, g, b), else float4.
// jitter != 0: samples at the stratified jitter of that seed (ro, rd: the rays, for
// their keys); 0: stratum midpoints (ro, rd unused).
// Waves (st_c != NULL; 8 samples per crossing, no bins): crossings k_lo <= k < k_hi
// only, resuming from and storing the per-ray state (st_c: rgb, T; st_d: depth) and
// whether the ray goes on (alive).
cudaError_t launch_composite(cudaStream_t s, const uint8_t* n_x, const float2* xing, const void* slot_out,
                             int slot_half, uint32_t n, int steps, int maxc, int cap, float t_term, float bg0,
                             float bg1, float bg2, float* rgb, float* depth, float* opacity, uint64_t* stats,
                             uint64_t jitter, const float* ro, const float* rd,
                             const float2* root = nullptr, float* bins = nullptr, int k_lo = 0, int k_hi = 256,
                             float4* st_c = nullptr, float* st_d = nullptr, uint8_t* alive = nullptr,
                             uint32_t* ray_counters = nullptr);
// The generated slots (j < n_x[r] * steps) of 4 x FP16 per-sample outputs as float4.
cudaError_t launch_slots_to_f32(cudaStream_t s, const uint8_t* n_x, const void* slot_half, float4* out, uint32_t n,
                                int steps, int cap);

// Proposal sampler (k_proposal.cu).
int proposal_param_count();
// Kernel attributes on the current device; *infer_grid gets the resident CTAs of the
// inference kernel there (its persistent grid).
cudaError_t prepare_proposal(int* infer_grid);
cudaError_t launch_prop_infer(cudaStream_t s, int infer_grid, const float* params, const float root_box[6],
                              const float* ro, const float* rd, uint32_t n, float coverage, int max_bins,
                              uint64_t* mask, uint8_t* fallback, unsigned long long* n_fallback, float* q_out);
// The same selection for renders, the network on the tensor cores (BF16 operands).
// q_out (may be NULL): the probabilities [n][65] of every ray in a tile with at least
// one ray that hits the scene box (other rows untouched).
cudaError_t launch_prop_infer_tc(cudaStream_t s, const float* params, const float root_box[6], const float* ro,
                                 const float* rd, uint32_t n, float coverage, int max_bins, uint64_t* mask,
                                 uint8_t* fallback, unsigned long long* n_fallback, int* err,
                                 float* q_out = nullptr);
cudaError_t launch_prop_grad(cudaStream_t s, const float* params, const float* ro, const float* rd,
                             const float2* root, const float* targets, uint32_t n, uint32_t batch, uint64_t seed,
                             uint64_t step, float* grad, float* loss);
cudaError_t launch_prop_adam(cudaStream_t s, float* P, float* g, float* m, float* v, int t, float lr);

// ---- host tree builder -------------------------------------------------------------
// Returns false on invalid input (message in err).
bool build_kdtree(const float* grid, int G, const double bbox[6], int max_depth, double leaf_frac,
                  std::vector<amnerf_node>& out, int& n_leaves, std::string& err);

}  // namespace amnerf
