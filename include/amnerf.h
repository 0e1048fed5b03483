/*
 * amnerf.h -- C ABI of the GB300 (sm_103a) Adaptive Multi-NeRF rendering library.
 *
 * The library renders a batch of camera rays through a density-guided KD tree of
 * axis-aligned boxes, one small same-shaped MLP per leaf (arXiv 2310.01881):
 *   1. traversal   every ray is intersected with the tree front to back and one
 *                  interval is recorded per leaf crossed (Sec. 3.5, Algorithm 1
 *                  "Traverse");
 *   2. sampling    each interval gets the same number of samples at stratum
 *                  midpoints (Sec. 3.5, Algorithm 1 "Sampling", Fig. "prop");
 *   3. grouping    crossings are grouped by leaf so every leaf network runs as one
 *                  dense batch (Sec. 3.5, Fig. "parallel");
 *   4. network     frequency encoding + per-leaf MLP -> density and colour
 *                  (Sec. 3.1 F_Theta, Sec. 3.2 same-shaped networks);
 *   5. composite   front-to-back NeRF quadrature with early ray termination
 *                  (Sec. 3.1: classic volume rendering).
 * The tree comes from a guidance density grid (Sec. 3.3-3.4, BuildKDTree).
 *
 * Conventions
 *   - Every function returns an amnerf_status; no C++ exception crosses the ABI.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global
 *     memory of the context's device.  The caller owns every buffer it passes; the
 *     library owns the tree, the weights and its scratch memory.
 *   - Rendering is asynchronous on the context's stream unless stated otherwise;
 *     device-side failures (a bounded wait that ran out) are recorded in a sticky
 *     status word that amnerf_sync() returns.
 *   - Not thread-safe: one context must not be used from two host threads at once.
 */
#ifndef AMNERF_H
#define AMNERF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AMNERF_API __attribute__((visibility("default")))
#else
#define AMNERF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amnerf_ctx amnerf_ctx; /* opaque, owned by the library */

typedef enum {
    AMNERF_OK = 0,
    AMNERF_E_INVAL = 1,       /* an argument is out of range or NULL */
    AMNERF_E_NOMEM = 2,       /* device or host allocation failed; nothing was written */
    AMNERF_E_CUDA = 3,        /* a CUDA runtime call failed */
    AMNERF_E_NOTREE = 4,      /* amnerf_build_tree has not succeeded on this context */
    AMNERF_E_NOMLP = 5,       /* no networks loaded, or loaded for another tree */
    AMNERF_E_TIMEOUT = 6,     /* a bounded device-side wait ran out (sticky) */
    AMNERF_E_DEVICE = 7,      /* no usable sm_100-class device */
    AMNERF_E_UNSUPPORTED = 8  /* valid request that this build does not implement */
} amnerf_status;

typedef enum {
    AMNERF_FP32 = 0,     /* plain path: FP32 SIMT network */
    AMNERF_BF16 = 1,     /* tcgen05 tensor cores, BF16 operands, FP32 accumulation */
    AMNERF_FP8E4M3 = 2   /* tcgen05, E4M3 operands with per-channel scales, FP32 accumulation */
} amnerf_precision;

/* Subdivision rule (Sec. 3.4).  A node becomes a leaf when depth == max_depth, when
 * its guidance mass is <= leaf_mass_frac * total mass (leaf_mass_frac > 0), or when
 * it is one grid cell wide along its longest axis.  max_depth in [0, 12]. */
typedef struct {
    int max_depth;
    double leaf_mass_frac;
} amnerf_tree_params;

/* One tree node as returned by amnerf_get_tree (preorder: node, left subtree,
 * right subtree; the left child of an inner node i is node i + 1). */
typedef struct {
    float lo[3], hi[3];          /* axis-aligned box */
    int32_t cell_lo[3];          /* guidance-grid cell range, half-open, x y z */
    int32_t cell_hi[3];
    int32_t axis;                /* split axis 0..2, -1 for a leaf */
    float split;                 /* split coordinate (inner nodes) */
    int32_t left, right;         /* child node indices, -1 for a leaf */
    int32_t leaf_id;             /* dense leaf index in left-first order, -1 for inner */
    uint32_t code;               /* binary path code: root 1, children 2c and 2c+1 (Sec. 3.1) */
    int32_t depth;
    int32_t reserved;
    double mass;                 /* guidance mass of the node */
} amnerf_node;

/* Shape of every leaf network (all leaves share it, Sec. 3.2):
 * input gamma_lx(x) ++ gamma_ld(d), (3 + 6 lx) + (3 + 6 ld) wide; `hidden` ReLU
 * layers of `width`; a 4-wide head: sigma = softplus(z0), rgb = sigmoid(z1..3).
 * Supported: width in {32, 64}, hidden in [1, 8], lx in [0, 12], ld in [0, 6]. */
typedef struct {
    int lx, ld, hidden, width;
    amnerf_precision prec;
} amnerf_mlp_desc;

/* Sampling and compositing parameters (Sec. 3.5).
 * steps_per_leaf: samples per leaf crossing, a power of two in [1, 32].
 * max_samples:    cap per ray; whole crossings are kept while they fit, so at most
 *                 floor(max_samples / steps_per_leaf) <= 255 crossings per ray.
 * t_term:         a sample is composited only while transmittance >= t_term.
 * bg:             background colour added with the residual transmittance. */
typedef struct {
    int steps_per_leaf;
    int max_samples;
    float t_term;
    float bg[3];
    /* Learned proposal sampler (not in the paper; see amnerf_proposal_set): when
     * use_proposal != 0 a loaded proposal network predicts, per ray, the depth-bin
     * distribution of its compositing weight; bins are kept by decreasing predicted
     * mass until `coverage` is reached (the background bin counts toward it), and
     * only leaf crossings overlapping a kept bin are sampled.  Rays needing more than
     * max_bins depth bins fall back to the plain sampler. */
    int use_proposal;
    float coverage;   /* e.g. 0.99 */
    int max_bins;     /* in [1, 64], e.g. 16 */
    /* Sample placement (Sec. 3.5: the samples of an interval may be placed at random
     * within it): 0 = the midpoint of each of the steps_per_leaf equal
     * strata of a crossing; otherwise the seed of a stratified jitter, one uniform
     * point per stratum, t_j = t_in + (j + u_j) delta.  u_j = (splitmix64 finaliser
     * of key + 0x9e3779b97f4a7c15 * (k * steps_per_leaf + j + 1)) >> 40, over 2^24,
     * for sample j of crossing k; the ray's key folds the bit patterns of (o.x, o.y),
     * (o.z, d.x) and (d.y, d.z) into the seed with three finalisations, so a ray draws
     * the same points in any batch.  The quadrature widths are the strata either way. */
    uint64_t jitter_seed;
    /* Empty-space skipping (Sec. 4.1: the density grid also serves "empty space
     * detection"): when skip_empty != 0 a leaf crossing is sampled only if one of its
     * samples -- placed as it would be as the ray's next kept crossing -- lies in a
     * guidance-grid cell (the grid given to amnerf_build_tree) of density >
     * empty_threshold.  The cell of a coordinate p on axis a is floor((p - lo_a) *
     * (G / (hi_a - lo_a))) in FP32, clamped to [0, G - 1].  Skipped crossings do not
     * count toward max_samples. */
    int skip_empty;
    float empty_threshold;
    /* Early ray termination in waves: 0 = one pass (every generated sample goes
     * through the network; compositing stops at T < t_term).  W in [1, 255] (needs
     * steps_per_leaf = 8): crossings k in [0, W), [W, 2W), ... are grouped, evaluated
     * and composited wave by wave, each wave only for the rays whose transmittance
     * has not dropped below t_term, so samples behind an opaque part of the ray are
     * not evaluated.  Pixels are bit-identical to the one-pass render.  The number of
     * waves is ceil(floor(max_samples / 8) / W), fixed by the parameters (no host
     * synchronisation).  With debug output, counts, offsets and order describe the
     * last wave; stage times put the whole wave loop under the network step. */
    int ert_wave;
    /* Adaptive hierarchical sampling (Sec. 3.5, Algorithm 1's HCheck; Fig. 1 (c)):
     * 0 = leaves only.  lod > 0 (finite): an inner node is descended only while its
     * extent along its split axis exceeds lod x the ray's entry distance into it (FP32:
     * hi - lo > lod * t_in); otherwise the inner node is one crossing, sampled like a
     * leaf crossing and evaluated by the inner node's own network.  lod is the ray
     * footprint per unit distance (about the pixel angle) times the number of
     * footprints a node must span to be refined.  Needs one network per node
     * (amnerf_load_mlps with the tree's node count). */
    float lod;
} amnerf_render_params;

/* Schedule of the network step's tiles over the persistent workers (warpgroups). */
typedef enum {
    AMNERF_SCHED_CONTIGUOUS = 0,   /* each worker takes one contiguous range of tiles (default) */
    AMNERF_SCHED_INTERLEAVED = 1,  /* worker w takes tiles w, w + workers, ... */
    AMNERF_SCHED_DYNAMIC = 2,      /* workers take the next tile from a device counter */
    AMNERF_SCHED_PER_LEAF = 3      /* one kernel launch per leaf (a per-node baseline; the
                                      render then synchronises once to read tile offsets) */
} amnerf_schedule;

/* Launch configuration of the network step (tensor-core paths; the FP32 path ignores it).
 * groups:      warpgroup sets per CTA = tiles in flight per SM, 0 = the largest that fits.
 * schedule:    how the tiles are spread over the groups.
 * width_split: hidden-width tiling of the BF16 kernel: 1 = one thread per sample row
 *              holds all `width` accumulator columns; 2 = two threads per row, each
 *              with width / 2 columns and half of the layer-0 encoding (twice the warps
 *              per tile); 0 = the library's default.  E4M3 always uses 1.  Every setting
 *              gives the same pixels. */
typedef struct {
    int groups;
    amnerf_schedule schedule;
    int width_split;
} amnerf_tuning;

/* Filled by a render when a non-NULL pointer is passed (this synchronises). */
typedef struct {
    uint64_t rays;
    uint64_t crossings;           /* leaf crossings kept after the cap */
    uint64_t samples_generated;   /* steps_per_leaf x crossings */
    uint64_t samples_composited;  /* samples reached before early termination */
    uint64_t tiles;               /* network tiles of 128 samples launched (all waves) */
    uint64_t fallback_rays;       /* proposal sampler: rays that used the plain sampler */
    float ms[4];                  /* stage times: traverse, group, network, composite */
    float proposal_ms;            /* proposal inference (part of ms[0]); 0 without the proposal */
    uint64_t samples_evaluated;   /* samples through the network: samples_generated, or
                                     fewer with ert_wave */
} amnerf_stats;

/* Optional copies of the intermediate results of one render (all DEVICE pointers
 * owned by the caller; any may be NULL).  maxc = floor(max_samples / steps).
 * "Network" is the leaf id, or with lod > 0 the network id (leaves, then inner nodes).
 *   n_x      uint8  [n_rays]              crossings per ray
 *   leaf     uint16 [n_rays * maxc]       network of crossing k of ray r at r*maxc+k
 *   t_in     float  [n_rays * maxc]       crossing entry
 *   t_out    float  [n_rays * maxc]       crossing exit
 *   counts   uint32 [n_networks]          crossings per network (samples = steps x counts)
 *   offsets  uint32 [n_networks + 1]      exclusive scan of counts
 *   order    uint32 [n_rays * maxc]       crossing ids r*maxc+k grouped by network; the
 *                                         order inside a network is unspecified
 *   slot_out float  [n_rays * max_samples * 4]  sigma, r, g, b of sample j of ray r at
 *                                         slot r*max_samples+j (unused slots untouched)
 *   prop_mask, prop_fallback              the proposal sampler's per-ray decisions
 *   prop_q   float  [n_rays * 65]         the proposal network's softmax outputs as the
 *                                         render's tensor-core inference computed them
 *                                         (rows of rays in a 128-ray tile where no ray
 *                                         hits the scene box are left untouched)
 * Entries past the valid ones are left untouched. */
typedef struct {
    uint8_t *n_x;
    uint16_t *leaf;
    float *t_in;
    float *t_out;
    uint32_t *counts;
    uint32_t *offsets;
    uint32_t *order;
    float *slot_out;
    uint64_t *prop_mask;      /* [n_rays] kept depth bins (proposal renders only) */
    uint8_t *prop_fallback;   /* [n_rays] 1 = plain sampler used (proposal renders only) */
    float *prop_q;            /* [n_rays][65] proposal probabilities (proposal renders only) */
} amnerf_debug;

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *out receives the context.
 * Errors: E_INVAL (out NULL), E_DEVICE (device missing or not compute capability
 * 10.x), E_NOMEM. */
AMNERF_API amnerf_status amnerf_create(amnerf_ctx **out, int device, void *cuda_stream);

/* Change the stream later renders enqueue on. */
AMNERF_API amnerf_status amnerf_set_stream(amnerf_ctx *ctx, void *cuda_stream);

/* Build the density-guided KD tree (Sec. 3.4 BuildKDTree) on the host and upload it.
 * grid_host: HOST float32 [G][G][G] indexed [z][y][x] (x fastest), finite and >= 0,
 *            the guidance density at cell centres; G in [2, 1024].
 * bbox:      HOST double[6] = lo x, lo y, lo z, hi x, hi y, hi z, lo < hi.
 * Splits: axis = longest in cells (ties to x < y < z); position = the smallest cell
 * boundary k >= 1 whose prefix mass reaches half the node mass (k = n - 1 when none
 * does; k = n / 2 for an empty node).  Cell boundary i on axis a is
 * (float)(lo_a + (hi_a - lo_a) * (i / G)) computed in double.  Masses are double
 * sums: cells into their slice in z-major, x-minor order, slices in order.
 * Synchronous.  Replaces any previous tree and invalidates loaded networks.
 * Errors: E_INVAL (bad sizes, negative / non-finite density), E_NOMEM, E_CUDA. */
AMNERF_API amnerf_status amnerf_build_tree(amnerf_ctx *ctx, const float *grid_host, int G, const double bbox[6],
                                const amnerf_tree_params *params, int *n_leaves_out);

/* Copy the current tree into HOST nodes_out (capacity `cap` records); *n_nodes gets
 * the node count.  E_INVAL when cap is too small (*n_nodes still set). */
AMNERF_API amnerf_status amnerf_get_tree(amnerf_ctx *ctx, amnerf_node *nodes_out, int cap, int *n_nodes);

/* Load one network per leaf (Sec. 3.2: same shape for all leaves), or one per node
 * (Sec. 3.3: inner nodes carry networks too; used by adaptive hierarchical sampling).
 * n_leaves:     the tree's leaf count (leaf networks, by leaf id) or its node count
 *               (networks 0 .. L-1 are the leaves by leaf id, then the inner nodes in
 *               preorder: network L + r is the r-th inner node of amnerf_get_tree's
 *               order).
 * weights_host: HOST float32, network-major; per network, for each hidden layer W_l
 *               (width x fan_in, row = output, row-major) then b_l (width); then the
 *               head W_o (4 x width) and b_o (4).
 * The library repacks the weights into the layout of desc->prec (FP32 transposed
 * tiles, BF16 or E4M3 tcgen05 core-matrix tiles; E4M3 per-leaf, per-layer,
 * per-output-channel scales s = max|W_row| / 448).  Synchronous.
 * Errors: E_NOTREE, E_INVAL (shape unsupported or n_leaves neither count), E_NOMEM. */
AMNERF_API amnerf_status amnerf_load_mlps(amnerf_ctx *ctx, const amnerf_mlp_desc *desc, int n_leaves,
                               const float *weights_host);

/* E4M3 networks with static scales.  Same as amnerf_load_mlps with
 * desc->prec == AMNERF_FP8E4M3, except that the layer inputs are quantised with
 * fixed scales instead of the default per-row scale max|row| / 448: the encoded
 * input as it is (its features lie within +-448), and input channel n of hidden
 * layer l + 1 with the per-output-channel scale of layer l,
 * s_(l,n) = max(max_k |W_l[n,k] alpha_k|, act_max[leaf][l + 1]) / 448 (alpha_k:
 * the scales of layer l's own input channels, 1 for layer 0; the last hidden layer
 * without the second term).  Every scale is folded at load time into the stored
 * weights (the next layer's columns, the head's BF16 weights) and the bias, which
 * enters through one BF16 MMA, so the network epilogue is ReLU and the conversion.
 * act_max_host: HOST float32 [n_leaves][hidden], finite and >= 0: the largest
 * |input| of hidden layer l (l = 0: the encoded input, not used for a scale), e.g.
 * from amnerf_calibrate_fp8; zero entries drop their term (a scale that would be 0
 * is 1).  Inputs beyond act_max saturate at +-448 times their scale.  Synchronous.
 * Errors: as amnerf_load_mlps; E_INVAL when desc->prec is not E4M3 or act_max is bad. */
AMNERF_API amnerf_status amnerf_load_mlps_fp8_static(amnerf_ctx *ctx, const amnerf_mlp_desc *desc, int n_leaves,
                                          const float *weights_host, const float *act_max_host);

/* Calibration for amnerf_load_mlps_fp8_static: renders the rays with the loaded
 * FP32 networks (amnerf_load_mlps with AMNERF_FP32) and records, per leaf and hidden
 * layer l, the largest |input of layer l| over the samples of those rays.
 * rays_o, rays_d: DEVICE float32 [n_rays][3]; params: as amnerf_render (the plain
 * sampler).  act_max_host: HOST float32 [n_leaves][hidden] (leaves no sample reaches
 * get 0).  Allocates temporary device buffers; synchronous.
 * Errors: E_NOMLP, E_INVAL (not FP32, proposal requested, bad arguments), E_NOMEM, E_CUDA. */
AMNERF_API amnerf_status amnerf_calibrate_fp8(amnerf_ctx *ctx, const float *rays_o, const float *rays_d,
                                   int64_t n_rays, const amnerf_render_params *params, float *act_max_host);

/* Render n_rays rays (the whole hot path: traverse, sample, group, network,
 * composite; Sec. 3.5 and Algorithm 1).
 * rays_o, rays_d: DEVICE float32 [n_rays][3] (x y z per ray); d need not be unit
 *                 length (the encoding uses it as given).
 * rgb: DEVICE float32 [n_rays][3]; depth, opacity: DEVICE float32 [n_rays].
 *      rgb = sum w c + T bg, depth = sum w t (not normalised), opacity = 1 - T.
 * stats: HOST, may be NULL; when given the call synchronises and fills it.
 * Asynchronous on the context stream otherwise.  Rays with NaN components are
 * memory-safe and give NaN pixels.  n_rays * floor(max_samples / steps_per_leaf)
 * must be < 2^32 (crossing ids are 32-bit; sample slots are 64-bit).  Renders
 * contain no host synchronisation and no allocation once the scratch is large
 * enough (so they can be captured in a CUDA graph), except with the per-leaf
 * schedule or a non-NULL stats pointer.
 * Errors: E_NOTREE, E_NOMLP, E_INVAL, E_NOMEM (scratch growth), E_CUDA. */
AMNERF_API amnerf_status amnerf_render(amnerf_ctx *ctx, const float *rays_o, const float *rays_d, int64_t n_rays,
                            const amnerf_render_params *params, float *rgb, float *depth, float *opacity,
                            amnerf_stats *stats);

/* amnerf_render plus copies of the intermediate results into `dbg` (see
 * amnerf_debug).  For tests; slower. */
AMNERF_API amnerf_status amnerf_render_debug(amnerf_ctx *ctx, const float *rays_o, const float *rays_d, int64_t n_rays,
                                  const amnerf_render_params *params, float *rgb, float *depth,
                                  float *opacity, const amnerf_debug *dbg, amnerf_stats *stats);

/* The render from the grouping on (grouping, network, compositing; Sec. 3.5 Fig.
 * "parallel", Sec. 3.1) over crossings given by the caller instead of the traversal:
 * for ray r, n_x[r] <= floor(max_samples / steps_per_leaf) = maxc crossings k, each
 * with its network leaf[r maxc + k] (a leaf id, or with per-node networks a network
 * id) and its interval t_in / t_out at r maxc + k, sampled as the traversal's
 * crossings are.  DEVICE buffers in the layout of amnerf_debug (n_x uint8 [n_rays],
 * leaf uint16, t_in, t_out float [n_rays * maxc]); rays, outputs and stats as in
 * amnerf_render.  Crossings the traversal would produce render exactly as
 * amnerf_render does.  Used to drive the grouped network with arbitrary per-network
 * counts (e.g. Zipf-distributed), and by the tests.  params must not ask for the
 * proposal sampler, empty-space skipping or lod.  A network id >= the networks loaded
 * or a count above maxc is recorded in the sticky status word (amnerf_sync, or a
 * stats render, returns E_INVAL) and replaced by network 0 / maxc.
 * Errors: as amnerf_render. */
AMNERF_API amnerf_status amnerf_render_crossings(amnerf_ctx *ctx, const float *rays_o, const float *rays_d,
                                                 int64_t n_rays, const amnerf_render_params *params,
                                                 const uint8_t *n_x, const uint16_t *leaf, const float *t_in,
                                                 const float *t_out, float *rgb, float *depth, float *opacity,
                                                 amnerf_stats *stats);

/* amnerf_render with HOST inputs and outputs (same layouts): copies the rays to
 * library-owned device buffers, renders, copies the pixels back and synchronises.
 * Page-locked host buffers make the copies asynchronous DMA.  Without `stats`, a
 * batch of at least 2 M rays is rendered in up to 4 chunks whose uploads and
 * downloads run on a second stream, overlapping the other chunks' rendering; the
 * pixels are the same as one amnerf_render of the whole batch. */
AMNERF_API amnerf_status amnerf_render_host(amnerf_ctx *ctx, const float *rays_o_host, const float *rays_d_host,
                                 int64_t n_rays, const amnerf_render_params *params, float *rgb_host,
                                 float *depth_host, float *opacity_host, amnerf_stats *stats);

/* Wait for the context stream and return (then clear) the sticky device status:
 * E_TIMEOUT when a bounded device wait ran out, E_INVAL when given crossings were out
 * of range (amnerf_render_crossings), E_CUDA on an asynchronous CUDA error. */
AMNERF_API amnerf_status amnerf_sync(amnerf_ctx *ctx);

/* Failure-detection self-test (no counterpart in the paper): launches a kernel that
 * waits, with the same bounded-wait code as the tensor-core network kernel, on an
 * mbarrier phase that nothing completes.  The wait gives up after `cycles` SM clock
 * cycles (1 .. 4e9), records a timeout in the context's status word and returns, so
 * the call returns AMNERF_E_TIMEOUT and the context stays usable. */
AMNERF_API amnerf_status amnerf_selftest_wait(amnerf_ctx *ctx, uint64_t cycles);

/* Record per-stage CUDA-event timing in later renders (amnerf_stats.ms). */
AMNERF_API amnerf_status amnerf_set_timing(amnerf_ctx *ctx, int enable);

/* Group crossings by leaf without allocating anything (no counterpart in the paper;
 * a variant of the render's grouping step for callers that may not allocate device
 * memory when they call -- e.g. a frame loop with a fixed memory budget, or a render
 * thread where cudaMalloc/cudaFree are banned because they can synchronise the
 * device and stall other streams).
 * n_x:     DEVICE uint8  [n_rays]         crossings per ray (<= maxc)
 * leaf:    DEVICE uint16 [n_rays * maxc]  leaf id of crossing k of ray r at r*maxc+k
 * counts:  DEVICE uint32 [n_leaves]       out: crossings per leaf (cleared by the call)
 * offsets: DEVICE uint32 [n_leaves + 1]   out: exclusive scan of counts
 * order:   DEVICE uint32 [n_rays * maxc]  out: crossing ids r*maxc+k grouped by leaf,
 *                                          order inside a leaf unspecified
 * Leaf ids >= n_leaves are ignored.  Enqueued on cuda_stream of the current device;
 * asynchronous.  Scratch: one file-scope device array of about 33 KB per device,
 * resident until exit, sized for n_leaves <= 4096 (E_INVAL beyond).  The first call
 * on a device is a warm-up: it looks the array up with cudaGetSymbolAddress, which
 * with lazy module loading (the CUDA default) may load the library's device code and
 * data -- an allocation and a synchronisation of its own -- so make it once, outside
 * the region where allocation is banned and before any stream capture (e.g. with
 * n_rays = 0 right after amnerf_create).  Later calls only enqueue work.  The address
 * is kept per device for the life of the process: after cudaDeviceReset (or a reset
 * of the primary context) this entry point must not be called again.  Calls share
 * the array: calls that overlap on the GPU race.
 * Errors: E_INVAL (sizes, NULL buffers), E_CUDA. */
AMNERF_API amnerf_status amnerf_group_by_leaf_static(const uint8_t *n_x, const uint16_t *leaf, int64_t n_rays,
                                                     int maxc, int n_leaves, uint32_t *counts, uint32_t *offsets,
                                                     uint32_t *order, void *cuda_stream);

/* ---- learned proposal sampler (not in the paper) --------------------------------
 * Network: input gamma_10(o + t0 d) ++ gamma_4(d) (t0 = entry into the root box), two
 * ReLU layers of 32, 65 logits (64 uniform depth bins of the ray's root interval and a
 * background bin), softmax.  Parameters: FP32 W1 [32 x 90], b1 [32], W2 [32 x 32],
 * b2 [32], W3 [65 x 32], b3 [65] = AMNERF_PROPOSAL_PARAMS values.  Training minimises
 * the mean cross-entropy against the plain renderer's binned compositing weights with
 * Adam (beta 0.9 / 0.999, eps 1e-8). */
#define AMNERF_PROPOSAL_PARAMS 6113

/* Load proposal parameters (HOST FP32, AMNERF_PROPOSAL_PARAMS values) and, for a
 * resumed training run, the Adam moments m, v (HOST, same size; NULL = zero) and the
 * number of steps already taken.  Synchronous. */
AMNERF_API amnerf_status amnerf_proposal_set(amnerf_ctx *ctx, const float *params, const float *adam_m,
                                             const float *adam_v, int step);

/* Read back parameters, Adam moments (HOST, may be NULL) and the step count. */
AMNERF_API amnerf_status amnerf_proposal_get(amnerf_ctx *ctx, float *params, float *adam_m, float *adam_v,
                                             int *step);

/* Training targets from the plain renderer: renders (DEVICE rays, outputs as in
 * amnerf_render) and writes per ray the compositing weight of each depth bin plus
 * the residual transmittance (DEVICE float [n_rays][65], sums to 1) and the root
 * interval (DEVICE float [n_rays][2]; 0, 0 for rays that miss).  Synchronous. */
AMNERF_API amnerf_status amnerf_proposal_targets(amnerf_ctx *ctx, const float *rays_o, const float *rays_d,
                                                 int64_t n_rays, const amnerf_render_params *params, float *rgb,
                                                 float *depth, float *opacity, float *targets, float *root);

/* `steps` Adam steps with learning rate lr on minibatches of `batch` rays drawn
 * with a counter-based hash of (seed, step, index) from n_rays rays (DEVICE rays,
 * root intervals and targets as produced by amnerf_proposal_targets).  losses
 * (HOST, may be NULL) receives the minibatch loss of every step.  Synchronous. */
AMNERF_API amnerf_status amnerf_proposal_train(amnerf_ctx *ctx, const float *rays_o, const float *rays_d,
                                               const float *root, const float *targets, int64_t n_rays, int steps,
                                               int batch, float lr, uint64_t seed, float *losses);

/* Full-batch mean loss and gradient (HOST, AMNERF_PROPOSAL_PARAMS) without updating
 * anything (for checks).  Synchronous. */
AMNERF_API amnerf_status amnerf_proposal_grad(amnerf_ctx *ctx, const float *rays_o, const float *rays_d,
                                              const float *root, const float *targets, int64_t n_rays, float *grad,
                                              float *loss);

/* Inference only: softmax outputs (DEVICE float [n_rays][65], may be NULL), kept-bin
 * masks (DEVICE uint64 [n_rays]) and fallback flags (DEVICE uint8 [n_rays]).  A ray
 * that misses the scene box gets mask 0 and no fallback. */
AMNERF_API amnerf_status amnerf_proposal_predict(amnerf_ctx *ctx, const float *rays_o, const float *rays_d,
                                                 int64_t n_rays, float coverage, int max_bins, float *probs,
                                                 uint64_t *mask, uint8_t *fallback);

/* Set / read the network step's launch configuration (see amnerf_tuning).
 * amnerf_get_tuning also reports the largest group count the loaded shape allows. */
AMNERF_API amnerf_status amnerf_set_tuning(amnerf_ctx *ctx, const amnerf_tuning *tuning);
AMNERF_API amnerf_status amnerf_get_tuning(amnerf_ctx *ctx, amnerf_tuning *tuning, int *max_groups);

/* Autotuner: renders the caller's batch (DEVICE buffers as in amnerf_render) once
 * per candidate configuration to warm up, then `reps` times under CUDA events, for
 * every group count 1..max, the contiguous, interleaved and dynamic schedules and (BF16)
 * width splits 1 and 2 (FP32 path: one candidate), keeps the fastest in the context
 * and returns it with its time per render.  Synchronous; the outputs hold the last
 * render.
 * Errors: as amnerf_render, E_INVAL (reps < 1). */
AMNERF_API amnerf_status amnerf_autotune(amnerf_ctx *ctx, const float *rays_o, const float *rays_d, int64_t n_rays,
                                         const amnerf_render_params *params, float *rgb, float *depth,
                                         float *opacity, int reps, amnerf_tuning *best, float *best_ms);

/* Human-readable name of a status code (static string). */
AMNERF_API const char *amnerf_status_string(amnerf_status s);

/* Last error message recorded on this context (static until the next call). */
AMNERF_API const char *amnerf_last_error(amnerf_ctx *ctx);

/* Free everything the context owns.  NULL is accepted. */
AMNERF_API void amnerf_destroy(amnerf_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* AMNERF_H */
