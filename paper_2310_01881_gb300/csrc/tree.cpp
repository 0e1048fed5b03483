// tree.cpp -- host-side density-guided KD-tree construction (Sec. 3.4, BuildKDTree).
//
// The scene box is split recursively: along the node's longest axis (in grid cells,
// ties to x < y < z), at the cell boundary where the cumulative guidance density
// first reaches half of the node's mass (the density-weighted median).  TestLeaf in
// the paper compares distillation PSNR against a trained teacher; without a teacher
// a node becomes a leaf at the depth limit, when its mass is at most a fraction of
// the total, or when it is one cell wide.  Nodes are emitted in preorder (left child
// of node i is i + 1) and leaves are numbered in left-first order; node codes are
// the binary path code of Sec. 3.1 (root 1, children 2c, 2c + 1).
#include <cmath>
#include <cstring>

#include "amnerf_internal.h"

namespace amnerf {
namespace {

struct Builder {
    const float* grid;
    int G;
    double lo[3], hi[3];
    int max_depth;
    double leaf_frac;
    double total = 0.0;
    int n_leaves = 0;
    std::vector<amnerf_node>* nodes;
    std::vector<double> slice;

    float boundary(int axis, int i) const {
        double v = lo[axis] + (hi[axis] - lo[axis]) * ((double)i / (double)G);
        return (float)v;
    }

    // Mass per slice along `axis`; cells are visited z-major, x-minor and each is
    // added to its slice; the node mass is the in-order sum of the slices.
    double slice_mass(const int c0[3], const int c1[3], int axis) {
        const int n = c1[axis] - c0[axis];
        std::fill(slice.begin(), slice.begin() + n, 0.0);
        for (int z = c0[2]; z < c1[2]; ++z) {
            for (int y = c0[1]; y < c1[1]; ++y) {
                const float* row = grid + ((size_t)z * G + y) * G;
                for (int x = c0[0]; x < c1[0]; ++x) {
                    const int at = axis == 0 ? x : (axis == 1 ? y : z);
                    slice[at - c0[axis]] += (double)row[x];
                }
            }
        }
        double m = 0.0;
        for (int i = 0; i < n; ++i) m += slice[i];
        return m;
    }

    int node(const int c0[3], const int c1[3], int depth, uint32_t code) {
        int axis = 0;
        for (int k = 1; k < 3; ++k)
            if (c1[k] - c0[k] > c1[axis] - c0[axis]) axis = k;
        const int n = c1[axis] - c0[axis];
        const double m = slice_mass(c0, c1, axis);
        if (depth == 0) total = m;

        const int id = (int)nodes->size();
        amnerf_node rec;
        std::memset(&rec, 0, sizeof rec);
        for (int k = 0; k < 3; ++k) {
            rec.lo[k] = boundary(k, c0[k]);
            rec.hi[k] = boundary(k, c1[k]);
            rec.cell_lo[k] = c0[k];
            rec.cell_hi[k] = c1[k];
        }
        rec.code = code;
        rec.depth = depth;
        rec.mass = m;
        rec.left = rec.right = -1;
        rec.leaf_id = -1;
        rec.axis = -1;
        nodes->push_back(rec);

        const bool stop = depth >= max_depth || n <= 1 || (leaf_frac > 0.0 && m <= leaf_frac * total);
        if (stop) {
            (*nodes)[id].leaf_id = n_leaves++;
            return id;
        }
        int k_split = n - 1;
        if (m == 0.0) {
            k_split = n / 2;
        } else {
            const double half = 0.5 * m;
            double acc = 0.0;
            for (int k = 1; k < n; ++k) {
                acc += slice[k - 1];
                if (acc >= half) {
                    k_split = k;
                    break;
                }
            }
        }
        int l0[3] = {c0[0], c0[1], c0[2]}, l1[3] = {c1[0], c1[1], c1[2]};
        int r0[3] = {c0[0], c0[1], c0[2]}, r1[3] = {c1[0], c1[1], c1[2]};
        l1[axis] = c0[axis] + k_split;
        r0[axis] = c0[axis] + k_split;
        (*nodes)[id].axis = axis;
        (*nodes)[id].split = boundary(axis, c0[axis] + k_split);
        const int left = node(l0, l1, depth + 1, code << 1);
        const int right = node(r0, r1, depth + 1, (code << 1) | 1u);
        (*nodes)[id].left = left;
        (*nodes)[id].right = right;
        return id;
    }
};

}  // namespace

bool build_kdtree(const float* grid, int G, const double bbox[6], int max_depth, double leaf_frac,
                  std::vector<amnerf_node>& out, int& n_leaves, std::string& err) {
    if (!grid || G < 2 || G > 1024) {
        err = "grid must be non-NULL with G in [2, 1024]";
        return false;
    }
    if (max_depth < 0 || max_depth > kMaxDepth) {
        err = "max_depth must be in [0, 12]";
        return false;
    }
    if (!(leaf_frac >= 0.0 && leaf_frac <= 1.0)) {
        err = "leaf_mass_frac must be in [0, 1]";
        return false;
    }
    for (int k = 0; k < 3; ++k) {
        if (!std::isfinite(bbox[k]) || !std::isfinite(bbox[3 + k]) || !(bbox[k] < bbox[3 + k])) {
            err = "bbox must be finite with lo < hi";
            return false;
        }
    }
    const size_t cells = (size_t)G * G * G;
    for (size_t i = 0; i < cells; ++i) {
        if (!(grid[i] >= 0.0f) || !std::isfinite(grid[i])) {
            err = "guidance density must be finite and >= 0";
            return false;
        }
    }
    Builder b;
    b.grid = grid;
    b.G = G;
    for (int k = 0; k < 3; ++k) {
        b.lo[k] = bbox[k];
        b.hi[k] = bbox[3 + k];
    }
    b.max_depth = max_depth;
    b.leaf_frac = leaf_frac;
    b.nodes = &out;
    b.slice.assign((size_t)G, 0.0);
    out.clear();
    const int c0[3] = {0, 0, 0}, c1[3] = {G, G, G};
    b.node(c0, c1, 0, 1u);
    n_leaves = b.n_leaves;
    return true;
}

}  // namespace amnerf
