// api.cu -- the C ABI (include/amnerf.h): context, tree and weight upload, scratch
// management and the render pipeline K-a -> K-b -> K-c -> K-d on one stream.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "amnerf_internal.h"

using namespace amnerf;

constexpr int kStatSlots = 10;  // device statistics words (see amnerf_ctx::d_stats)
constexpr int kDefaultWidthSplit = 1;  // BF16 hidden-width tiling when the caller sets none

struct amnerf_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    // tree
    std::vector<amnerf_node> nodes;
    int n_leaves = 0;
    int tree_depth = 0;  // depth of the deepest node (the traversal's stack size)
    DevNode* d_nodes = nullptr;
    uint16_t* d_node_net = nullptr;  // network id of every node (leaves: leaf id; inner: L + preorder rank)
    float2* d_walk = nullptr;        // (split, meta) of every node
    float* d_grid = nullptr;  // the guidance grid (empty-space skipping)
    int grid_G = 0;
    float grid_lo[3] = {0.f, 0.f, 0.f}, grid_sc[3] = {0.f, 0.f, 0.f};
    // networks
    bool mlp_loaded = false;
    int n_nets = 0;           // networks loaded: n_leaves, or one per node (hierarchical sampling)
    amnerf_mlp_desc desc{};
    int k0 = 0;
    size_t leaf_stride = 0;  // bytes
    void* d_weights = nullptr;
    // per-network scratch (sized for kMaxNets)
    uint32_t* d_counts = nullptr;
    uint32_t* d_offsets = nullptr;
    uint32_t* d_tile_off = nullptr;
    uint32_t* d_cursor = nullptr;
    // [0] crossings [1] tiles [2] composited [3] fallback rays [4] [5] one wave's
    // crossings and tiles [6] dynamic tile counter [8] [9] crossings and tiles over waves
    uint64_t* d_stats = nullptr;
    // ray counters of the persistent traversal and compositing (kRayCounters each, one
    // per 128-byte line), zeroed at the start of every render
    uint32_t* d_ray_ctr = nullptr;
    int* d_err = nullptr;
    // per-ray scratch
    size_t cap_slots = 0;   // n_rays * maxc capacity
    size_t cap_samples = 0; // n_rays * cap capacity
    size_t cap_rays = 0;
    uint8_t* d_nx = nullptr;
    float2* d_xing = nullptr;
    uint16_t* d_xleaf = nullptr;
    uint32_t* d_order = nullptr;
    float4* d_slot = nullptr;
    // host-buffer path
    size_t cap_host_rays = 0;
    float* d_hbuf = nullptr;  // o, d, rgb, depth, opacity
    // chunked host path: copies on their own stream, ordered by events
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_up[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_done[4] = {nullptr, nullptr, nullptr, nullptr};
    // network kernel schedule (autotuned or set by the caller)
    int max_groups = 1;
    amnerf_tuning tuning{0, AMNERF_SCHED_CONTIGUOUS, 0};
    std::vector<uint32_t> h_tile_off;  // per-leaf launches: host copy of tile offsets
    // proposal sampler
    bool prop_loaded = false;
    int prop_grid = 0;        // persistent grid of the inference kernel on this device
    int prop_step = 0;
    float* d_prop = nullptr;  // params | m | v | grad | loss (5 x NPAR floats + 1)
    size_t cap_prop_rays = 0;
    uint64_t* d_mask = nullptr;
    uint8_t* d_fallback = nullptr;
    float2* d_root = nullptr;
    // wave-by-wave rendering (early ray termination): per-ray state between waves
    size_t cap_wave_rays = 0;
    float4* d_wst_c = nullptr;  // rgb, T
    float* d_wst_d = nullptr;   // depth
    uint8_t* d_alive = nullptr;
    // E4M3 static activation scales; FP32-path calibration output while calibrating
    bool act_static = false;
    float* d_amax = nullptr;   // [n_leaves][hidden]
    bool calibrating = false;
    // timing
    bool timing = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace {

amnerf_status fail(amnerf_ctx* c, amnerf_status s, const std::string& msg) {
    if (c) c->last_error = msg;
    return s;
}

amnerf_status cuda_fail(amnerf_ctx* c, cudaError_t e, const char* what) {
    if (c) c->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? AMNERF_E_NOMEM : AMNERF_E_CUDA;
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void free_ray_scratch(amnerf_ctx* ctx) {
    dfree(ctx->d_nx);
    dfree(ctx->d_xing);
    dfree(ctx->d_xleaf);
    dfree(ctx->d_order);
    dfree(ctx->d_slot);
    ctx->cap_slots = ctx->cap_samples = ctx->cap_rays = 0;
}

// Grow the per-ray scratch to hold n rays x maxc crossings x cap slots.
amnerf_status ensure_scratch(amnerf_ctx* ctx, size_t n, int maxc, int cap) {
    const size_t slots = n * (size_t)maxc, samples = n * (size_t)cap;
    if (n <= ctx->cap_rays && slots <= ctx->cap_slots && samples <= ctx->cap_samples) return AMNERF_OK;
    free_ray_scratch(ctx);
    const size_t rn = std::max(n, ctx->cap_rays), rs = std::max(slots, ctx->cap_slots),
                 rm = std::max(samples, ctx->cap_samples);
    cudaError_t e;
    if ((e = cudaMalloc((void**)&ctx->d_nx, rn)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_xing, rs * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_xleaf, rs * sizeof(uint16_t))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_order, rs * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_slot, rm * sizeof(float4))) != cudaSuccess) {
        free_ray_scratch(ctx);
        cudaGetLastError();
        return cuda_fail(ctx, e, "scratch allocation");
    }
    ctx->cap_rays = rn;
    ctx->cap_slots = rs;
    ctx->cap_samples = rm;
    return AMNERF_OK;
}

amnerf_status check_params(amnerf_ctx* ctx, const amnerf_render_params* p, int64_t n, int& maxc) {
    if (!p) return fail(ctx, AMNERF_E_INVAL, "params is NULL");
    const int st = p->steps_per_leaf;
    if (st < 1 || st > 32 || (st & (st - 1)) != 0)
        return fail(ctx, AMNERF_E_INVAL, "steps_per_leaf must be a power of two in [1, 32]");
    if (p->max_samples < st) return fail(ctx, AMNERF_E_INVAL, "max_samples must be >= steps_per_leaf");
    maxc = p->max_samples / st;
    if (maxc > 255) return fail(ctx, AMNERF_E_INVAL, "max_samples / steps_per_leaf must be <= 255");
    if (!(p->t_term >= 0.0f) || !std::isfinite(p->t_term)) return fail(ctx, AMNERF_E_INVAL, "t_term must be >= 0");
    if (p->skip_empty && !std::isfinite(p->empty_threshold))
        return fail(ctx, AMNERF_E_INVAL, "empty_threshold must be finite");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(p->bg[c])) return fail(ctx, AMNERF_E_INVAL, "bg must be finite");
    if (n < 0) return fail(ctx, AMNERF_E_INVAL, "n_rays < 0");
    if (p->use_proposal) {
        if (!(p->coverage > 0.0f && p->coverage <= 1.0f)) return fail(ctx, AMNERF_E_INVAL, "coverage must be in (0, 1]");
        if (p->max_bins < 1 || p->max_bins > 64) return fail(ctx, AMNERF_E_INVAL, "max_bins must be in [1, 64]");
    }
    if ((uint64_t)n * (uint64_t)maxc >= (1ull << 32))
        return fail(ctx, AMNERF_E_INVAL, "n_rays * floor(max_samples / steps_per_leaf) must be < 2^32 (split the batch)");
    if (p->ert_wave < 0 || p->ert_wave > 255) return fail(ctx, AMNERF_E_INVAL, "ert_wave must be in [0, 255]");
    if (p->ert_wave > 0 && st != 8) return fail(ctx, AMNERF_E_INVAL, "ert_wave needs steps_per_leaf = 8");
    if (!(p->lod >= 0.0f) || !std::isfinite(p->lod)) return fail(ctx, AMNERF_E_INVAL, "lod must be finite and >= 0");
    return AMNERF_OK;
}

// Repack the FP32 master weights of one leaf into the FP32 SIMT layout (transposed).
void pack_simt(const float* src, float* dst, int width, int hidden, int k0) {
    const float* w = src;
    float* o = dst;
    int kin = k0;
    for (int l = 0; l < hidden; ++l) {
        for (int k = 0; k < kin; ++k)
            for (int n = 0; n < width; ++n) o[(size_t)k * width + n] = w[(size_t)n * kin + k];
        o += (size_t)kin * width;
        w += (size_t)kin * width;
        for (int n = 0; n < width; ++n) o[n] = w[n];
        o += width;
        w += width;
        kin = width;
    }
    for (int k = 0; k < width; ++k)
        for (int n = 0; n < 4; ++n) o[(size_t)k * 4 + n] = w[(size_t)n * width + k];
    o += 4 * width;
    w += 4 * width;
    for (int n = 0; n < 4; ++n) o[n] = w[n];
}

}  // namespace

// Per-ray proposal scratch (masks, fallback flags, root intervals).
static amnerf_status ensure_wave_scratch(amnerf_ctx* ctx, size_t n) {
    if (n <= ctx->cap_wave_rays) return AMNERF_OK;
    dfree(ctx->d_wst_c);
    dfree(ctx->d_wst_d);
    dfree(ctx->d_alive);
    ctx->cap_wave_rays = 0;
    cudaError_t e;
    if ((e = cudaMalloc((void**)&ctx->d_wst_c, n * sizeof(float4))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_wst_d, n * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_alive, n)) != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "wave scratch allocation");
    }
    ctx->cap_wave_rays = n;
    return AMNERF_OK;
}

static amnerf_status ensure_prop_scratch(amnerf_ctx* ctx, size_t n) {
    if (n <= ctx->cap_prop_rays) return AMNERF_OK;
    dfree(ctx->d_mask);
    dfree(ctx->d_fallback);
    dfree(ctx->d_root);
    ctx->cap_prop_rays = 0;
    cudaError_t e;
    if ((e = cudaMalloc((void**)&ctx->d_mask, n * 8)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_fallback, n)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_root, n * sizeof(float2))) != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "proposal scratch allocation");
    }
    ctx->cap_prop_rays = n;
    return AMNERF_OK;
}

extern "C" {

const char* amnerf_status_string(amnerf_status s) {
    switch (s) {
        case AMNERF_OK: return "ok";
        case AMNERF_E_INVAL: return "invalid argument";
        case AMNERF_E_NOMEM: return "out of memory";
        case AMNERF_E_CUDA: return "CUDA error";
        case AMNERF_E_NOTREE: return "no tree built";
        case AMNERF_E_NOMLP: return "no networks loaded";
        case AMNERF_E_TIMEOUT: return "device wait timed out";
        case AMNERF_E_DEVICE: return "no usable sm_100-class device";
        case AMNERF_E_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* amnerf_last_error(amnerf_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

amnerf_status amnerf_create(amnerf_ctx** out, int device, void* cuda_stream) {
    if (!out) return AMNERF_E_INVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return AMNERF_E_DEVICE;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess || prop.major != 10) return AMNERF_E_DEVICE;
    amnerf_ctx* ctx = new (std::nothrow) amnerf_ctx();
    if (!ctx) return AMNERF_E_NOMEM;
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if ((e = cudaSetDevice(device)) != cudaSuccess ||
        (e = prepare_group()) != cudaSuccess ||
        (e = prepare_traverse()) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_counts, sizeof(uint32_t) * kMaxNets)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_offsets, sizeof(uint32_t) * (kMaxNets + 1))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_tile_off, sizeof(uint32_t) * (kMaxNets + 1))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_cursor, sizeof(uint32_t) * kMaxNets)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_stats, sizeof(uint64_t) * kStatSlots)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_ray_ctr, kRayCounterBytes * 2)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ctx->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(ctx->d_err, 0, sizeof(int))) != cudaSuccess) {
        amnerf_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? AMNERF_E_NOMEM : AMNERF_E_CUDA;
    }
    for (int i = 0; i < 6; ++i) cudaEventCreate(&ctx->ev[i]);
    *out = ctx;
    return AMNERF_OK;
}

amnerf_status amnerf_set_stream(amnerf_ctx* ctx, void* cuda_stream) {
    if (!ctx) return AMNERF_E_INVAL;
    ctx->stream = (cudaStream_t)cuda_stream;
    return AMNERF_OK;
}

amnerf_status amnerf_set_timing(amnerf_ctx* ctx, int enable) {
    if (!ctx) return AMNERF_E_INVAL;
    ctx->timing = enable != 0;
    return AMNERF_OK;
}

void amnerf_destroy(amnerf_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    free_ray_scratch(ctx);
    dfree(ctx->d_nodes);
    dfree(ctx->d_node_net);
    dfree(ctx->d_walk);
    dfree(ctx->d_grid);
    dfree(ctx->d_weights);
    dfree(ctx->d_amax);
    dfree(ctx->d_counts);
    dfree(ctx->d_offsets);
    dfree(ctx->d_tile_off);
    dfree(ctx->d_cursor);
    dfree(ctx->d_stats);
    dfree(ctx->d_ray_ctr);
    dfree(ctx->d_err);
    dfree(ctx->d_hbuf);
    dfree(ctx->d_prop);
    dfree(ctx->d_mask);
    dfree(ctx->d_fallback);
    dfree(ctx->d_root);
    dfree(ctx->d_wst_c);
    dfree(ctx->d_wst_d);
    dfree(ctx->d_alive);
    for (int i = 0; i < 6; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    for (int i = 0; i < 4; ++i) {
        if (ctx->ev_up[i]) cudaEventDestroy(ctx->ev_up[i]);
        if (ctx->ev_done[i]) cudaEventDestroy(ctx->ev_done[i]);
    }
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    delete ctx;
}

amnerf_status amnerf_build_tree(amnerf_ctx* ctx, const float* grid_host, int G, const double bbox[6],
                                const amnerf_tree_params* params, int* n_leaves_out) {
    if (!ctx || !params || !bbox) return fail(ctx, AMNERF_E_INVAL, "NULL argument");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::vector<amnerf_node> nodes;
    int nl = 0;
    std::string err;
    if (!build_kdtree(grid_host, G, bbox, params->max_depth, params->leaf_mass_frac, nodes, nl, err))
        return fail(ctx, AMNERF_E_INVAL, err);
    std::vector<DevNode> dn(nodes.size());
    std::vector<float2> wk(nodes.size());
    std::vector<uint16_t> net(nodes.size());
    for (size_t i = 0, inner = 0; i < nodes.size(); ++i)
        net[i] = (uint16_t)(nodes[i].axis < 0 ? nodes[i].leaf_id : nl + (int)inner++);
    for (size_t i = 0; i < nodes.size(); ++i) {
        const amnerf_node& s = nodes[i];
        const uint32_t payload = s.axis < 0 ? (uint32_t)s.leaf_id : (uint32_t)s.right;
        const uint32_t meta = (uint32_t)(s.axis + 1) | (payload << 2);
        float fmeta;
        std::memcpy(&fmeta, &meta, sizeof fmeta);
        dn[i].a = make_float4(s.lo[0], s.lo[1], s.lo[2], s.hi[0]);
        dn[i].b = make_float4(s.hi[1], s.hi[2], s.split, fmeta);
        wk[i] = make_float2(s.split, fmeta);
    }
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    dfree(ctx->d_nodes);
    dfree(ctx->d_node_net);
    dfree(ctx->d_walk);
    dfree(ctx->d_grid);
    ctx->grid_G = 0;
    CK(cudaMalloc((void**)&ctx->d_nodes, sizeof(DevNode) * dn.size()), "tree allocation");
    CK(cudaMemcpy(ctx->d_nodes, dn.data(), sizeof(DevNode) * dn.size(), cudaMemcpyHostToDevice), "tree upload");
    CK(cudaMalloc((void**)&ctx->d_walk, sizeof(float2) * wk.size()), "tree allocation");
    CK(cudaMemcpy(ctx->d_walk, wk.data(), sizeof(float2) * wk.size(), cudaMemcpyHostToDevice), "tree upload");
    CK(cudaMalloc((void**)&ctx->d_node_net, sizeof(uint16_t) * net.size()), "tree allocation");
    CK(cudaMemcpy(ctx->d_node_net, net.data(), sizeof(uint16_t) * net.size(), cudaMemcpyHostToDevice),
       "tree upload");
    // the guidance grid stays resident for empty-space skipping
    const size_t cells = (size_t)G * G * G;
    CK(cudaMalloc((void**)&ctx->d_grid, sizeof(float) * cells), "grid allocation");
    CK(cudaMemcpy(ctx->d_grid, grid_host, sizeof(float) * cells, cudaMemcpyHostToDevice), "grid upload");
    ctx->grid_G = G;
    for (int a = 0; a < 3; ++a) {
        ctx->grid_lo[a] = (float)bbox[a];
        ctx->grid_sc[a] = (float)((double)G / (bbox[3 + a] - bbox[a]));
    }
    int depth = 0;
    for (const amnerf_node& s : nodes) depth = std::max(depth, (int)s.depth);
    ctx->nodes.swap(nodes);
    ctx->n_leaves = nl;
    ctx->tree_depth = depth;
    ctx->mlp_loaded = false;
    dfree(ctx->d_weights);
    if (n_leaves_out) *n_leaves_out = nl;
    return AMNERF_OK;
}

amnerf_status amnerf_get_tree(amnerf_ctx* ctx, amnerf_node* nodes_out, int cap, int* n_nodes) {
    if (!ctx || !n_nodes) return fail(ctx, AMNERF_E_INVAL, "NULL argument");
    if (ctx->nodes.empty()) return fail(ctx, AMNERF_E_NOTREE, "no tree");
    *n_nodes = (int)ctx->nodes.size();
    if (!nodes_out || cap < (int)ctx->nodes.size()) return fail(ctx, AMNERF_E_INVAL, "capacity too small");
    std::memcpy(nodes_out, ctx->nodes.data(), sizeof(amnerf_node) * ctx->nodes.size());
    return AMNERF_OK;
}

static amnerf_status load_impl(amnerf_ctx* ctx, const amnerf_mlp_desc* desc, int n_leaves,
                               const float* weights_host, const float* act_max) {
    if (!ctx || !desc || !weights_host) return fail(ctx, AMNERF_E_INVAL, "NULL argument");
    if (ctx->nodes.empty()) return fail(ctx, AMNERF_E_NOTREE, "build the tree first");
    if (n_leaves != ctx->n_leaves && n_leaves != (int)ctx->nodes.size())
        return fail(ctx, AMNERF_E_INVAL, "n_networks must be the tree's leaf count or its node count");
    const amnerf_mlp_desc& m = *desc;
    if ((m.width != 32 && m.width != 64) || m.hidden < 1 || m.hidden > 8 || m.lx < 0 || m.lx > 12 || m.ld < 0 ||
        m.ld > 6)
        return fail(ctx, AMNERF_E_INVAL, "unsupported network shape");
    if (m.prec != AMNERF_FP32 && m.prec != AMNERF_BF16 && m.prec != AMNERF_FP8E4M3)
        return fail(ctx, AMNERF_E_INVAL, "unknown precision");
    const int k0 = (3 + 6 * m.lx) + (3 + 6 * m.ld);
    const size_t per = (size_t)m.width * k0 + m.width + (size_t)(m.hidden - 1) * (m.width * m.width + m.width) +
                       4 * (size_t)m.width + 4;
    for (size_t i = 0; i < per * (size_t)n_leaves; ++i)
        if (!std::isfinite(weights_host[i])) return fail(ctx, AMNERF_E_INVAL, "non-finite weight");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    size_t stride;
    std::vector<uint8_t> blob;
    if (m.prec == AMNERF_FP32) {
        stride = simt_leaf_stride_floats(m.width, m.hidden, k0) * sizeof(float);
        blob.assign(stride * n_leaves, 0);
        for (int l = 0; l < n_leaves; ++l)
            pack_simt(weights_host + per * l, reinterpret_cast<float*>(blob.data() + stride * l), m.width, m.hidden,
                      k0);
    } else {
        stride = tc_leaf_stride_bytes(m.width, m.hidden, k0, (int)m.prec);
        if (stride == 0) return fail(ctx, AMNERF_E_UNSUPPORTED, "precision not built");
        blob.assign(stride * n_leaves, 0);
        for (int l = 0; l < n_leaves; ++l)
            pack_tc_leaf(weights_host + per * l, blob.data() + stride * l, m.width, m.hidden, k0, (int)m.prec,
                         act_max ? act_max + (size_t)l * m.hidden : nullptr);
    }
    int max_groups = 1;
    if (m.prec == AMNERF_FP32) {
        CK(prepare_mlp_simt(m.width, m.hidden, k0), "network kernel setup");
    } else {
        CK(prepare_mlp_tc(m.width, m.hidden, k0, (int)m.prec, &max_groups), "network kernel setup");
    }
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    dfree(ctx->d_weights);
    ctx->mlp_loaded = false;
    CK(cudaMalloc(&ctx->d_weights, blob.size()), "weight allocation");
    CK(cudaMemcpy(ctx->d_weights, blob.data(), blob.size(), cudaMemcpyHostToDevice), "weight upload");
    ctx->desc = m;
    ctx->n_nets = n_leaves;
    ctx->k0 = k0;
    ctx->leaf_stride = stride;
    ctx->max_groups = max_groups;
    ctx->act_static = act_max != nullptr;
    ctx->mlp_loaded = true;
    return AMNERF_OK;
}

amnerf_status amnerf_load_mlps(amnerf_ctx* ctx, const amnerf_mlp_desc* desc, int n_leaves,
                               const float* weights_host) {
    return load_impl(ctx, desc, n_leaves, weights_host, nullptr);
}

amnerf_status amnerf_load_mlps_fp8_static(amnerf_ctx* ctx, const amnerf_mlp_desc* desc, int n_leaves,
                                         const float* weights_host, const float* act_max_host) {
    if (!ctx || !desc || !act_max_host) return fail(ctx, AMNERF_E_INVAL, "NULL argument");
    if (desc->prec != AMNERF_FP8E4M3) return fail(ctx, AMNERF_E_INVAL, "static activation scales are for E4M3");
    if (desc->hidden < 1 || desc->hidden > 8 || n_leaves < 1 || n_leaves > kMaxNets)
        return fail(ctx, AMNERF_E_INVAL, "bad shape");
    for (size_t i = 0; i < (size_t)n_leaves * desc->hidden; ++i)
        if (!(act_max_host[i] >= 0.0f) || !std::isfinite(act_max_host[i]))
            return fail(ctx, AMNERF_E_INVAL, "act_max must be finite and >= 0");
    return load_impl(ctx, desc, n_leaves, weights_host, act_max_host);
}

// Crossings given by the caller (amnerf_render_crossings), in the debug layout.
struct CrossingsIn {
    const uint8_t* n_x;
    const uint16_t* leaf;
    const float* t_in;
    const float* t_out;
};

static amnerf_status device_status(int herr) {
    return herr == kDevErrTimeout ? AMNERF_E_TIMEOUT : (herr == kDevErrBounds ? AMNERF_E_INVAL : AMNERF_E_CUDA);
}

static amnerf_status render_impl(amnerf_ctx* ctx, const float* ro, const float* rd, int64_t n,
                                 const amnerf_render_params* p, float* rgb, float* depth, float* opacity,
                                 const amnerf_debug* dbg, amnerf_stats* stats, float* bins_out = nullptr,
                                 float2* root_out = nullptr, const CrossingsIn* cin = nullptr) {
    if (!ctx) return AMNERF_E_INVAL;
    if (ctx->nodes.empty()) return fail(ctx, AMNERF_E_NOTREE, "build the tree first");
    if (!ctx->mlp_loaded) return fail(ctx, AMNERF_E_NOMLP, "load the networks first");
    int maxc = 0;
    amnerf_status st = check_params(ctx, p, n, maxc);
    if (st != AMNERF_OK) return st;
    if (n > 0 && (!ro || !rd || !rgb || !depth || !opacity)) return fail(ctx, AMNERF_E_INVAL, "NULL buffer");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int steps = p->steps_per_leaf, cap = p->max_samples;
    if (n > 0) {
        st = ensure_scratch(ctx, (size_t)n, maxc, cap);
        if (st != AMNERF_OK) return st;
    }
    if (p->lod > 0.0f && ctx->n_nets != (int)ctx->nodes.size())
        return fail(ctx, AMNERF_E_INVAL, "lod > 0 needs one network per node");
    if (cin && (p->use_proposal || p->skip_empty || p->lod > 0.0f || bins_out || root_out))
        return fail(ctx, AMNERF_E_INVAL, "given crossings take no proposal, skipping, lod or targets");
    if (cin && n > 0 && (!cin->n_x || !cin->leaf || !cin->t_in || !cin->t_out))
        return fail(ctx, AMNERF_E_INVAL, "NULL crossing buffer");
    cudaStream_t s = ctx->stream;
    const int L = ctx->n_nets;  // networks: the grouping keys
    const uint32_t nn = (uint32_t)n;
    HierArgs hier;
    hier.lod = p->lod;
    hier.node_net = ctx->d_node_net;
    if (ctx->timing) cudaEventRecord(ctx->ev[0], s);
    CK(cudaMemsetAsync(ctx->d_counts, 0, sizeof(uint32_t) * L, s), "memset");
    CK(cudaMemsetAsync(ctx->d_stats, 0, sizeof(uint64_t) * kStatSlots, s), "memset");
    CK(cudaMemsetAsync(ctx->d_ray_ctr, 0, kRayCounterBytes * 2, s), "memset");
    const uint64_t* mask = nullptr;
    const uint8_t* fallback = nullptr;
    if (p->use_proposal && n > 0) {
        if (!ctx->prop_loaded) return fail(ctx, AMNERF_E_INVAL, "use_proposal set but no proposal network loaded");
        st = ensure_prop_scratch(ctx, (size_t)n);
        if (st != AMNERF_OK) return st;
        const amnerf_node& root = ctx->nodes[0];
        const float box[6] = {root.lo[0], root.lo[1], root.lo[2], root.hi[0], root.hi[1], root.hi[2]};
        // renders predict the kept bins with the proposal network on the tensor cores
        CK(launch_prop_infer_tc(s, ctx->d_prop, box, ro, rd, nn, p->coverage, p->max_bins, ctx->d_mask,
                                ctx->d_fallback, reinterpret_cast<unsigned long long*>(ctx->d_stats + 3), ctx->d_err,
                                dbg ? dbg->prop_q : nullptr),
           "proposal launch");
        if (ctx->timing) cudaEventRecord(ctx->ev[5], s);
        mask = ctx->d_mask;
        fallback = ctx->d_fallback;
    }
    OccArgs occ;
    if (p->skip_empty) {
        occ.grid = ctx->d_grid;
        occ.G = ctx->grid_G;
        for (int a = 0; a < 3; ++a) {
            occ.lo[a] = ctx->grid_lo[a];
            occ.sc[a] = ctx->grid_sc[a];
        }
        occ.thr = p->empty_threshold;
        occ.steps = steps;
        occ.jitter = p->jitter_seed;
    }
    if (cin) {
        CK(launch_load_crossings(s, cin->n_x, cin->leaf, cin->t_in, cin->t_out, nn, maxc, L, ctx->d_nx, ctx->d_xing,
                                 ctx->d_xleaf, ctx->d_counts, ctx->d_err),
           "crossing load launch");
    } else {
        CK(launch_traverse(s, ro, rd, nn, ctx->d_nodes, ctx->d_walk, maxc, ctx->d_nx, ctx->d_xing, ctx->d_xleaf,
                           ctx->d_counts, L, ctx->d_err, mask, fallback, root_out, occ, hier, ctx->tree_depth,
                           ctx->d_ray_ctr),
           "traverse launch");
    }
    if (ctx->timing) cudaEventRecord(ctx->ev[1], s);
    CK(launch_scan(s, ctx->d_counts, L, kTileRows / steps, ctx->d_offsets, ctx->d_tile_off, ctx->d_cursor,
                   ctx->d_stats),
       "scan launch");
    // waves: the rays' crossings in groups of ert_wave, each group only for the rays
    // that have not terminated, so that samples behind an opaque crossing are never
    // evaluated (the number of waves depends only on maxc: no host synchronisation)
    const bool waves = p->ert_wave > 0 && n > 0 && !bins_out;
    if (waves) {
        st = ensure_wave_scratch(ctx, (size_t)n);
        if (st != AMNERF_OK) return st;
    } else {
        CK(launch_scatter(s, ctx->d_nx, ctx->d_xleaf, nn, maxc, ctx->d_cursor, ctx->d_order, L), "scatter launch");
    }
    if (ctx->timing) cudaEventRecord(ctx->ev[2], s);
    // the network over the grouped crossings whose per-wave counts (crossings, tiles)
    // sit at wstats[0], wstats[1]
    auto run_network = [&](uint64_t* wstats) -> amnerf_status {
        MlpArgs a;
        a.order = ctx->d_order;
        a.offsets = ctx->d_offsets;
        a.tile_off = ctx->d_tile_off;
        a.stats = wstats;
        a.n_leaves = L;
        a.xing = ctx->d_xing;
        a.ro = ro;
        a.rd = rd;
        a.weights = ctx->d_weights;
        a.leaf_stride = ctx->leaf_stride;
        a.width = ctx->desc.width;
        a.hidden = ctx->desc.hidden;
        a.lx = ctx->desc.lx;
        a.ld = ctx->desc.ld;
        a.k0 = ctx->k0;
        a.steps = steps;
        a.maxc = maxc;
        a.maxc_magic = maxc > 1 ? (uint32_t)(((1ull << 32) + (uint64_t)maxc - 1ull) / (uint64_t)maxc) : 0u;
        a.lg_steps = 0;
        while ((1 << a.lg_steps) < steps) ++a.lg_steps;
        a.cap = cap;
        a.slot_out = ctx->d_slot;
        a.err = ctx->d_err;
        a.amax = ctx->calibrating ? ctx->d_amax : nullptr;
        a.act_static = ctx->act_static ? 1 : 0;
        a.jitter = p->jitter_seed;
        a.tile_counter = reinterpret_cast<uint32_t*>(ctx->d_stats + 6);
        a.t_begin = 0;
        a.t_end = 0xffffffffu;
        const bool tc = ctx->desc.prec != AMNERF_FP32;
        a.groups = ctx->tuning.groups > 0 ? std::min(ctx->tuning.groups, ctx->max_groups) : ctx->max_groups;
        a.width_split = ctx->desc.prec == AMNERF_BF16 ? (ctx->tuning.width_split > 0 ? ctx->tuning.width_split
                                                                                       : kDefaultWidthSplit)
                                                      : 1;
        int sched = ctx->tuning.schedule;
        if (!tc && sched != AMNERF_SCHED_PER_LEAF) sched = AMNERF_SCHED_CONTIGUOUS;
        a.schedule = sched == AMNERF_SCHED_PER_LEAF ? kSchedContiguous : sched;
        if (sched != AMNERF_SCHED_PER_LEAF) {
            cudaError_t e = tc ? launch_mlp_tc(s, a, ctx->sm_count, (int)ctx->desc.prec) : launch_mlp_simt(s, a, ctx->sm_count);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "network launch");
        } else {
            // baseline: one launch per leaf, as a per-node library call would do
            ctx->h_tile_off.resize((size_t)L + 1);
            CK(cudaMemcpyAsync(ctx->h_tile_off.data(), ctx->d_tile_off, 4 * ((size_t)L + 1), cudaMemcpyDeviceToHost, s),
               "tile offsets");
            CK(cudaStreamSynchronize(s), "stream sync");
            for (int l = 0; l < L; ++l) {
                const uint32_t tb = ctx->h_tile_off[l], te = ctx->h_tile_off[l + 1];
                if (te == tb) continue;
                a.t_begin = tb;
                a.t_end = te;
                const uint32_t per_cta = tc ? (uint32_t)a.groups : 1u;
                const int grid = (int)std::min<uint32_t>((uint32_t)ctx->sm_count, (te - tb + per_cta - 1) / per_cta);
                cudaError_t e = tc ? launch_mlp_tc(s, a, grid, (int)ctx->desc.prec) : launch_mlp_simt(s, a, grid);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "network launch");
            }
        }
        return AMNERF_OK;
    };
    if (!waves) {
        if (n > 0) {
            st = run_network(ctx->d_stats);
            if (st != AMNERF_OK) return st;
        }
        if (ctx->timing) cudaEventRecord(ctx->ev[3], s);
        CK(launch_composite(s, ctx->d_nx, ctx->d_xing, ctx->d_slot, ctx->desc.prec != AMNERF_FP32, nn, steps, maxc,
                            cap, p->t_term, p->bg[0], p->bg[1], p->bg[2], rgb, depth, opacity, ctx->d_stats,
                            p->jitter_seed, ro, rd, root_out, bins_out, 0, 256, nullptr, nullptr, nullptr,
                            ctx->d_ray_ctr + kRayCounterBytes / sizeof(uint32_t)),
           "composite launch");
    } else {
        const int W = p->ert_wave;
        for (int k_lo = 0; k_lo < maxc; k_lo += W) {
            const int k_hi = std::min(maxc, k_lo + W);
            const uint8_t* alive = k_lo > 0 ? ctx->d_alive : nullptr;
            CK(cudaMemsetAsync(ctx->d_counts, 0, sizeof(uint32_t) * L, s), "memset");
            CK(launch_scatter_wave(s, true, ctx->d_nx, ctx->d_xleaf, nn, maxc, k_lo, k_hi, alive, ctx->d_counts,
                                   nullptr, L),
               "wave count launch");
            CK(launch_scan(s, ctx->d_counts, L, kTileRows / steps, ctx->d_offsets, ctx->d_tile_off, ctx->d_cursor,
                           ctx->d_stats + 4, ctx->d_stats + 8),
               "scan launch");
            CK(launch_scatter_wave(s, false, ctx->d_nx, ctx->d_xleaf, nn, maxc, k_lo, k_hi, alive, ctx->d_cursor,
                                   ctx->d_order, L),
               "scatter launch");
            CK(cudaMemsetAsync(ctx->d_stats + 6, 0, sizeof(uint64_t), s), "memset");  // dynamic tile counter
            st = run_network(ctx->d_stats + 4);
            if (st != AMNERF_OK) return st;
            CK(launch_composite(s, ctx->d_nx, ctx->d_xing, ctx->d_slot, ctx->desc.prec != AMNERF_FP32, nn, steps,
                                maxc, cap, p->t_term, p->bg[0], p->bg[1], p->bg[2], rgb, depth, opacity, ctx->d_stats,
                                p->jitter_seed, ro, rd, nullptr, nullptr, k_lo, k_hi, ctx->d_wst_c, ctx->d_wst_d,
                                ctx->d_alive),
               "composite launch");
        }
        if (ctx->timing) cudaEventRecord(ctx->ev[3], s);
    }
    if (ctx->timing) cudaEventRecord(ctx->ev[4], s);

    if (dbg && n > 0) {
        const size_t slots = (size_t)n * maxc;
        if (dbg->n_x) CK(cudaMemcpyAsync(dbg->n_x, ctx->d_nx, (size_t)n, cudaMemcpyDeviceToDevice, s), "debug copy");
        if (dbg->leaf)
            CK(cudaMemcpyAsync(dbg->leaf, ctx->d_xleaf, slots * 2, cudaMemcpyDeviceToDevice, s), "debug copy");
        if (dbg->t_in)
            CK(cudaMemcpy2DAsync(dbg->t_in, sizeof(float), ctx->d_xing, sizeof(float2), sizeof(float), slots,
                                 cudaMemcpyDeviceToDevice, s),
               "debug copy");
        if (dbg->t_out)
            CK(cudaMemcpy2DAsync(dbg->t_out, sizeof(float), reinterpret_cast<const float*>(ctx->d_xing) + 1,
                                 sizeof(float2), sizeof(float), slots, cudaMemcpyDeviceToDevice, s),
               "debug copy");
        if (dbg->counts)
            CK(cudaMemcpyAsync(dbg->counts, ctx->d_counts, 4 * (size_t)L, cudaMemcpyDeviceToDevice, s), "debug copy");
        if (dbg->offsets)
            CK(cudaMemcpyAsync(dbg->offsets, ctx->d_offsets, 4 * (size_t)(L + 1), cudaMemcpyDeviceToDevice, s),
               "debug copy");
        if (dbg->order)
            CK(cudaMemcpyAsync(dbg->order, ctx->d_order, slots * 4, cudaMemcpyDeviceToDevice, s), "debug copy");
        if (dbg->slot_out) {
            if (ctx->desc.prec != AMNERF_FP32)  // the tensor-core paths keep 4 x FP16 per sample
                CK(launch_slots_to_f32(s, ctx->d_nx, ctx->d_slot, reinterpret_cast<float4*>(dbg->slot_out), (uint32_t)n,
                                       steps, cap),
                   "debug copy");
            else
                CK(cudaMemcpyAsync(dbg->slot_out, ctx->d_slot, (size_t)n * cap * 16, cudaMemcpyDeviceToDevice, s),
                   "debug copy");
        }
        if (dbg->prop_mask && mask)
            CK(cudaMemcpyAsync(dbg->prop_mask, mask, (size_t)n * 8, cudaMemcpyDeviceToDevice, s), "debug copy");
        if (dbg->prop_fallback && fallback)
            CK(cudaMemcpyAsync(dbg->prop_fallback, fallback, (size_t)n, cudaMemcpyDeviceToDevice, s), "debug copy");
    }
    if (stats) {
        uint64_t h[kStatSlots];
        CK(cudaMemcpyAsync(h, ctx->d_stats, sizeof h, cudaMemcpyDeviceToHost, s), "stats copy");
        CK(cudaStreamSynchronize(s), "stream sync");
        stats->rays = (uint64_t)n;
        stats->crossings = h[0];
        stats->samples_generated = h[0] * (uint64_t)steps;
        stats->tiles = waves ? h[9] : h[1];
        stats->samples_evaluated = (waves ? h[8] : h[0]) * (uint64_t)steps;
        stats->samples_composited = h[2];
        stats->fallback_rays = h[3];
        for (int i = 0; i < 4; ++i) {
            float ms = 0.f;
            if (ctx->timing) cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]);
            stats->ms[i] = ms;
        }
        stats->proposal_ms = 0.f;
        if (ctx->timing && mask) cudaEventElapsedTime(&stats->proposal_ms, ctx->ev[0], ctx->ev[5]);
        int herr = 0;
        CK(cudaMemcpy(&herr, ctx->d_err, sizeof herr, cudaMemcpyDeviceToHost), "status copy");
        if (herr) {
            cudaMemset(ctx->d_err, 0, sizeof(int));
            return fail(ctx, device_status(herr), "device status word set");
        }
    }
    return AMNERF_OK;
}

amnerf_status amnerf_render_crossings(amnerf_ctx* ctx, const float* rays_o, const float* rays_d, int64_t n_rays,
                                      const amnerf_render_params* params, const uint8_t* n_x, const uint16_t* leaf,
                                      const float* t_in, const float* t_out, float* rgb, float* depth, float* opacity,
                                      amnerf_stats* stats) {
    const CrossingsIn cin{n_x, leaf, t_in, t_out};
    return render_impl(ctx, rays_o, rays_d, n_rays, params, rgb, depth, opacity, nullptr, stats, nullptr, nullptr,
                       &cin);
}

amnerf_status amnerf_render(amnerf_ctx* ctx, const float* rays_o, const float* rays_d, int64_t n_rays,
                            const amnerf_render_params* params, float* rgb, float* depth, float* opacity,
                            amnerf_stats* stats) {
    return render_impl(ctx, rays_o, rays_d, n_rays, params, rgb, depth, opacity, nullptr, stats);
}

amnerf_status amnerf_calibrate_fp8(amnerf_ctx* ctx, const float* rays_o, const float* rays_d, int64_t n_rays,
                                   const amnerf_render_params* params, float* act_max_host) {
    if (!ctx || !act_max_host) return fail(ctx, AMNERF_E_INVAL, "NULL argument");
    if (!ctx->mlp_loaded) return fail(ctx, AMNERF_E_NOMLP, "load the FP32 networks first");
    if (ctx->desc.prec != AMNERF_FP32) return fail(ctx, AMNERF_E_INVAL, "calibration runs the FP32 networks");
    if (params && params->use_proposal) return fail(ctx, AMNERF_E_INVAL, "calibrate with the plain sampler");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t cnt = (size_t)ctx->n_nets * ctx->desc.hidden;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    dfree(ctx->d_amax);
    CK(cudaMalloc((void**)&ctx->d_amax, sizeof(float) * cnt), "calibration allocation");
    CK(cudaMemsetAsync(ctx->d_amax, 0, sizeof(float) * cnt, ctx->stream), "memset");
    float *rgb = nullptr, *aux = nullptr;
    if (n_rays > 0) {
        CK(cudaMalloc((void**)&rgb, sizeof(float) * 3 * (size_t)n_rays), "calibration allocation");
        if (cudaMalloc((void**)&aux, sizeof(float) * 2 * (size_t)n_rays) != cudaSuccess) {
            cudaFree(rgb);
            cudaGetLastError();
            return fail(ctx, AMNERF_E_NOMEM, "calibration allocation");
        }
    }
    ctx->calibrating = true;
    amnerf_status st = render_impl(ctx, rays_o, rays_d, n_rays, params, rgb, aux, aux + (n_rays > 0 ? n_rays : 0),
                                   nullptr, nullptr);
    ctx->calibrating = false;
    if (st == AMNERF_OK) st = amnerf_sync(ctx);
    if (st == AMNERF_OK &&
        cudaMemcpy(act_max_host, ctx->d_amax, sizeof(float) * cnt, cudaMemcpyDeviceToHost) != cudaSuccess)
        st = fail(ctx, AMNERF_E_CUDA, "calibration copy");
    cudaFree(rgb);
    cudaFree(aux);
    return st;
}

amnerf_status amnerf_render_debug(amnerf_ctx* ctx, const float* rays_o, const float* rays_d, int64_t n_rays,
                                  const amnerf_render_params* params, float* rgb, float* depth, float* opacity,
                                  const amnerf_debug* dbg, amnerf_stats* stats) {
    return render_impl(ctx, rays_o, rays_d, n_rays, params, rgb, depth, opacity, dbg, stats);
}

amnerf_status amnerf_render_host(amnerf_ctx* ctx, const float* ro, const float* rd, int64_t n,
                                 const amnerf_render_params* p, float* rgb, float* depth, float* opacity,
                                 amnerf_stats* stats) {
    if (!ctx) return AMNERF_E_INVAL;
    if (n < 0) return fail(ctx, AMNERF_E_INVAL, "n_rays < 0");
    if (n > 0 && (!ro || !rd || !rgb || !depth || !opacity)) return fail(ctx, AMNERF_E_INVAL, "NULL buffer");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t nn = (size_t)n;
    if (nn > ctx->cap_host_rays) {
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        dfree(ctx->d_hbuf);
        ctx->cap_host_rays = 0;
        CK(cudaMalloc((void**)&ctx->d_hbuf, nn * 11 * sizeof(float)), "host-path buffers");
        ctx->cap_host_rays = nn;
    }
    float* dro = ctx->d_hbuf;
    float* drd = dro + 3 * ctx->cap_host_rays;
    float* drgb = drd + 3 * ctx->cap_host_rays;
    float* ddep = drgb + 3 * ctx->cap_host_rays;
    float* dop = ddep + ctx->cap_host_rays;
    cudaStream_t s = ctx->stream;
    // Large batches without statistics go in up to 4 chunks of >= 1 M rays: the copy
    // stream uploads every chunk up front and downloads chunk i once it is rendered,
    // so the copies overlap the rendering of the other chunks.
    constexpr size_t kChunkMin = (size_t)1 << 20;
    const int chunks = stats ? 1 : (int)std::min<size_t>(4, nn / kChunkMin);
    if (chunks >= 2) {
        if (!ctx->copy_stream) {
            CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "copy stream");
            for (int i = 0; i < 4; ++i) {
                CK(cudaEventCreateWithFlags(&ctx->ev_up[i], cudaEventDisableTiming), "event");
                CK(cudaEventCreateWithFlags(&ctx->ev_done[i], cudaEventDisableTiming), "event");
            }
        }
        cudaStream_t cs = ctx->copy_stream;
        // the buffers are free: the previous call synchronised before returning
        size_t b[5];
        for (int i = 0; i <= chunks; ++i) b[i] = nn * (size_t)i / (size_t)chunks;
        for (int i = 0; i < chunks; ++i) {
            const size_t m = b[i + 1] - b[i];
            CK(cudaMemcpyAsync(dro + 3 * b[i], ro + 3 * b[i], m * 12, cudaMemcpyHostToDevice, cs), "ray upload");
            CK(cudaMemcpyAsync(drd + 3 * b[i], rd + 3 * b[i], m * 12, cudaMemcpyHostToDevice, cs), "ray upload");
            CK(cudaEventRecord(ctx->ev_up[i], cs), "event");
        }
        for (int i = 0; i < chunks; ++i) {
            const size_t m = b[i + 1] - b[i];
            CK(cudaStreamWaitEvent(s, ctx->ev_up[i], 0), "event wait");
            amnerf_status st = render_impl(ctx, dro + 3 * b[i], drd + 3 * b[i], (int64_t)m, p, drgb + 3 * b[i],
                                           ddep + b[i], dop + b[i], nullptr, nullptr);
            if (st != AMNERF_OK) {
                cudaStreamSynchronize(cs);
                return st;
            }
            CK(cudaEventRecord(ctx->ev_done[i], s), "event");
            CK(cudaStreamWaitEvent(cs, ctx->ev_done[i], 0), "event wait");
            CK(cudaMemcpyAsync(rgb + 3 * b[i], drgb + 3 * b[i], m * 12, cudaMemcpyDeviceToHost, cs), "pixel download");
            CK(cudaMemcpyAsync(depth + b[i], ddep + b[i], m * 4, cudaMemcpyDeviceToHost, cs), "pixel download");
            CK(cudaMemcpyAsync(opacity + b[i], dop + b[i], m * 4, cudaMemcpyDeviceToHost, cs), "pixel download");
        }
        CK(cudaStreamSynchronize(cs), "stream sync");  // it waited for the last chunk's render
        return AMNERF_OK;
    }
    if (nn) {
        CK(cudaMemcpyAsync(dro, ro, nn * 12, cudaMemcpyHostToDevice, s), "ray upload");
        CK(cudaMemcpyAsync(drd, rd, nn * 12, cudaMemcpyHostToDevice, s), "ray upload");
    }
    amnerf_status st = render_impl(ctx, dro, drd, n, p, drgb, ddep, dop, nullptr, stats);
    if (st != AMNERF_OK) return st;
    if (nn) {
        CK(cudaMemcpyAsync(rgb, drgb, nn * 12, cudaMemcpyDeviceToHost, s), "pixel download");
        CK(cudaMemcpyAsync(depth, ddep, nn * 4, cudaMemcpyDeviceToHost, s), "pixel download");
        CK(cudaMemcpyAsync(opacity, dop, nn * 4, cudaMemcpyDeviceToHost, s), "pixel download");
    }
    CK(cudaStreamSynchronize(s), "stream sync");
    return AMNERF_OK;
}

static float* prop_params(amnerf_ctx* c) { return c->d_prop; }
static float* prop_m(amnerf_ctx* c) { return c->d_prop + proposal_param_count(); }
static float* prop_v(amnerf_ctx* c) { return c->d_prop + 2 * proposal_param_count(); }
static float* prop_g(amnerf_ctx* c) { return c->d_prop + 3 * proposal_param_count(); }
static float* prop_loss(amnerf_ctx* c) { return c->d_prop + 4 * proposal_param_count(); }

amnerf_status amnerf_proposal_set(amnerf_ctx* ctx, const float* params, const float* m, const float* v, int step) {
    if (!ctx || !params || step < 0) return fail(ctx, AMNERF_E_INVAL, "bad arguments");
    const int np = proposal_param_count();
    for (int i = 0; i < np; ++i)
        if (!std::isfinite(params[i])) return fail(ctx, AMNERF_E_INVAL, "non-finite proposal parameter");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (!ctx->d_prop) {
        CK(cudaMalloc((void**)&ctx->d_prop, sizeof(float) * (5 * (size_t)np + 1)), "proposal allocation");
        CK(prepare_proposal(&ctx->prop_grid), "proposal kernel setup");
    }
    CK(cudaMemset(ctx->d_prop, 0, sizeof(float) * (5 * (size_t)np + 1)), "memset");
    CK(cudaMemcpy(prop_params(ctx), params, sizeof(float) * np, cudaMemcpyHostToDevice), "proposal upload");
    if (m) CK(cudaMemcpy(prop_m(ctx), m, sizeof(float) * np, cudaMemcpyHostToDevice), "proposal upload");
    if (v) CK(cudaMemcpy(prop_v(ctx), v, sizeof(float) * np, cudaMemcpyHostToDevice), "proposal upload");
    ctx->prop_step = step;
    ctx->prop_loaded = true;
    return AMNERF_OK;
}

amnerf_status amnerf_proposal_get(amnerf_ctx* ctx, float* params, float* m, float* v, int* step) {
    if (!ctx) return AMNERF_E_INVAL;
    if (!ctx->prop_loaded) return fail(ctx, AMNERF_E_INVAL, "no proposal network loaded");
    const int np = proposal_param_count();
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize(), "stream sync");
    if (params) CK(cudaMemcpy(params, prop_params(ctx), sizeof(float) * np, cudaMemcpyDeviceToHost), "download");
    if (m) CK(cudaMemcpy(m, prop_m(ctx), sizeof(float) * np, cudaMemcpyDeviceToHost), "download");
    if (v) CK(cudaMemcpy(v, prop_v(ctx), sizeof(float) * np, cudaMemcpyDeviceToHost), "download");
    if (step) *step = ctx->prop_step;
    return AMNERF_OK;
}

amnerf_status amnerf_proposal_targets(amnerf_ctx* ctx, const float* ro, const float* rd, int64_t n,
                                      const amnerf_render_params* p, float* rgb, float* depth, float* opacity,
                                      float* targets, float* root) {
    if (!ctx || !p) return AMNERF_E_INVAL;
    if (n > 0 && (!targets || !root)) return fail(ctx, AMNERF_E_INVAL, "NULL buffer");
    amnerf_render_params q = *p;
    q.use_proposal = 0;  // targets come from the plain sampler
    amnerf_status st = render_impl(ctx, ro, rd, n, &q, rgb, depth, opacity, nullptr, nullptr, targets,
                                   reinterpret_cast<float2*>(root));
    if (st != AMNERF_OK) return st;
    return amnerf_sync(ctx);
}

amnerf_status amnerf_proposal_train(amnerf_ctx* ctx, const float* ro, const float* rd, const float* root,
                                    const float* targets, int64_t n, int steps, int batch, float lr, uint64_t seed,
                                    float* losses) {
    if (!ctx || n <= 0 || steps < 0 || batch < 1 || !(lr > 0.0f) || seed == 0 || !ro || !rd || !root || !targets)
        return fail(ctx, AMNERF_E_INVAL, "bad arguments (seed must be nonzero)");
    if (!ctx->prop_loaded) return fail(ctx, AMNERF_E_INVAL, "no proposal network loaded");
    if (n >= (1ll << 32)) return fail(ctx, AMNERF_E_INVAL, "n_rays must be < 2^32");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = ctx->stream;
    std::vector<float> h_loss((size_t)steps);
    float* d_losses = nullptr;
    if (steps > 0) CK(cudaMalloc((void**)&d_losses, sizeof(float) * (size_t)steps), "loss buffer");
    CK(cudaMemsetAsync(prop_g(ctx), 0, sizeof(float) * proposal_param_count(), s), "memset");
    if (steps > 0) CK(cudaMemsetAsync(d_losses, 0, sizeof(float) * (size_t)steps, s), "memset");
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < steps && e == cudaSuccess; ++i) {
        const uint64_t step = (uint64_t)ctx->prop_step + 1;
        e = launch_prop_grad(s, prop_params(ctx), ro, rd, reinterpret_cast<const float2*>(root), targets, (uint32_t)n,
                             (uint32_t)batch, seed, step, prop_g(ctx), d_losses + i);
        if (e == cudaSuccess) e = launch_prop_adam(s, prop_params(ctx), prop_g(ctx), prop_m(ctx), prop_v(ctx), (int)step, lr);
        ctx->prop_step += 1;
    }
    if (e == cudaSuccess && steps > 0)
        e = cudaMemcpyAsync(h_loss.data(), d_losses, sizeof(float) * (size_t)steps, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (d_losses) cudaFree(d_losses);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "proposal training");
    if (losses) std::memcpy(losses, h_loss.data(), sizeof(float) * (size_t)steps);
    return AMNERF_OK;
}

amnerf_status amnerf_proposal_grad(amnerf_ctx* ctx, const float* ro, const float* rd, const float* root,
                                   const float* targets, int64_t n, float* grad, float* loss) {
    if (!ctx || n <= 0 || !grad || !loss || !ro || !rd || !root || !targets) return fail(ctx, AMNERF_E_INVAL, "bad arguments");
    if (!ctx->prop_loaded) return fail(ctx, AMNERF_E_INVAL, "no proposal network loaded");
    if (n >= (1ll << 32)) return fail(ctx, AMNERF_E_INVAL, "n_rays must be < 2^32");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = ctx->stream;
    const int np = proposal_param_count();
    CK(cudaMemsetAsync(prop_g(ctx), 0, sizeof(float) * np, s), "memset");
    CK(cudaMemsetAsync(prop_loss(ctx), 0, sizeof(float), s), "memset");
    CK(launch_prop_grad(s, prop_params(ctx), ro, rd, reinterpret_cast<const float2*>(root), targets, (uint32_t)n,
                        (uint32_t)n, 0, 0, prop_g(ctx), prop_loss(ctx)),
       "proposal gradient");
    CK(cudaMemcpyAsync(grad, prop_g(ctx), sizeof(float) * np, cudaMemcpyDeviceToHost, s), "download");
    CK(cudaMemcpyAsync(loss, prop_loss(ctx), sizeof(float), cudaMemcpyDeviceToHost, s), "download");
    CK(cudaMemsetAsync(prop_g(ctx), 0, sizeof(float) * np, s), "memset");
    CK(cudaStreamSynchronize(s), "stream sync");
    return AMNERF_OK;
}

amnerf_status amnerf_proposal_predict(amnerf_ctx* ctx, const float* ro, const float* rd, int64_t n, float coverage,
                                      int max_bins, float* probs, uint64_t* mask, uint8_t* fallback) {
    if (!ctx || n < 0 || !(coverage > 0.0f && coverage <= 1.0f) || max_bins < 1 || max_bins > 64)
        return fail(ctx, AMNERF_E_INVAL, "bad arguments");
    if (n > 0 && (!ro || !rd || !mask || !fallback)) return fail(ctx, AMNERF_E_INVAL, "NULL buffer");
    if (!ctx->prop_loaded) return fail(ctx, AMNERF_E_INVAL, "no proposal network loaded");
    if (ctx->nodes.empty()) return fail(ctx, AMNERF_E_NOTREE, "build the tree first");
    if (n >= (1ll << 32)) return fail(ctx, AMNERF_E_INVAL, "n_rays must be < 2^32");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const amnerf_node& r = ctx->nodes[0];
    const float box[6] = {r.lo[0], r.lo[1], r.lo[2], r.hi[0], r.hi[1], r.hi[2]};
    CK(cudaMemsetAsync(ctx->d_stats + 3, 0, 8, ctx->stream), "memset");
    CK(launch_prop_infer(ctx->stream, ctx->prop_grid, prop_params(ctx), box, ro, rd, (uint32_t)n, coverage, max_bins, mask, fallback,
                         reinterpret_cast<unsigned long long*>(ctx->d_stats + 3), probs),
       "proposal launch");
    return AMNERF_OK;
}

amnerf_status amnerf_set_tuning(amnerf_ctx* ctx, const amnerf_tuning* t) {
    if (!ctx || !t) return AMNERF_E_INVAL;
    if (t->groups < 0 || t->groups > 4 || t->schedule < AMNERF_SCHED_CONTIGUOUS || t->schedule > AMNERF_SCHED_PER_LEAF ||
        t->width_split < 0 || t->width_split > 2)
        return fail(ctx, AMNERF_E_INVAL, "tuning out of range");
    ctx->tuning = *t;
    return AMNERF_OK;
}

amnerf_status amnerf_get_tuning(amnerf_ctx* ctx, amnerf_tuning* t, int* max_groups) {
    if (!ctx || !t) return AMNERF_E_INVAL;
    *t = ctx->tuning;
    if (max_groups) *max_groups = ctx->max_groups;
    return AMNERF_OK;
}

amnerf_status amnerf_autotune(amnerf_ctx* ctx, const float* ro, const float* rd, int64_t n,
                              const amnerf_render_params* p, float* rgb, float* depth, float* opacity, int reps,
                              amnerf_tuning* best_out, float* best_ms_out) {
    if (!ctx || reps < 1) return fail(ctx, AMNERF_E_INVAL, "bad arguments");
    if (!ctx->mlp_loaded) return fail(ctx, AMNERF_E_NOMLP, "load the networks first");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const bool tc = ctx->desc.prec != AMNERF_FP32;
    std::vector<amnerf_tuning> cand;
    if (tc) {
        const int max_split = ctx->desc.prec == AMNERF_BF16 ? 2 : 1;
        for (int ws = 1; ws <= max_split; ++ws)
            for (int g = 1; g <= ctx->max_groups; ++g)
                for (int sc = AMNERF_SCHED_CONTIGUOUS; sc <= AMNERF_SCHED_DYNAMIC; ++sc)
                    cand.push_back(amnerf_tuning{g, (amnerf_schedule)sc, ws});
    } else {
        cand.push_back(amnerf_tuning{0, AMNERF_SCHED_CONTIGUOUS, 1});
    }
    const amnerf_tuning saved = ctx->tuning;
    const bool saved_timing = ctx->timing;
    ctx->timing = false;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    float best = 1e30f;
    amnerf_tuning best_t = cand[0];
    amnerf_status st = AMNERF_OK;
    for (const amnerf_tuning& c : cand) {
        ctx->tuning = c;
        st = render_impl(ctx, ro, rd, n, p, rgb, depth, opacity, nullptr, nullptr);  // warm-up
        if (st != AMNERF_OK) break;
        cudaEventRecord(e0, ctx->stream);
        for (int r = 0; r < reps && st == AMNERF_OK; ++r)
            st = render_impl(ctx, ro, rd, n, p, rgb, depth, opacity, nullptr, nullptr);
        cudaEventRecord(e1, ctx->stream);
        if (st != AMNERF_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = fail(ctx, AMNERF_E_CUDA, "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        if (ms < best) {
            best = ms;
            best_t = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->timing = saved_timing;
    if (st != AMNERF_OK) {
        ctx->tuning = saved;
        return st;
    }
    ctx->tuning = best_t;
    if (best_out) *best_out = best_t;
    if (best_ms_out) *best_ms_out = best;
    return amnerf_sync(ctx);
}

amnerf_status amnerf_selftest_wait(amnerf_ctx* ctx, uint64_t cycles) {
    if (!ctx || cycles == 0 || cycles > 4000000000ull) return fail(ctx, AMNERF_E_INVAL, "cycles must be in [1, 4e9]");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(launch_wait_selftest(ctx->stream, (unsigned long long)cycles, ctx->d_err), "self-test launch");
    return amnerf_sync(ctx);
}

amnerf_status amnerf_sync(amnerf_ctx* ctx) {
    if (!ctx) return AMNERF_E_INVAL;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize(), "stream sync");
    int herr = 0;
    CK(cudaMemcpy(&herr, ctx->d_err, sizeof herr, cudaMemcpyDeviceToHost), "status copy");
    if (herr) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        return fail(ctx, device_status(herr), "device status word set");
    }
    return AMNERF_OK;
}

}  // extern "C"
