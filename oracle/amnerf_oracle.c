/*
 * amnerf_oracle.c -- plain, slow CPU oracle of the Adaptive Multi-NeRF rendering
 * hot path (arXiv 2310.01881).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header, table
 * or helper with the CUDA library; both sides only consume the seeded arrays built
 * by the input generator.
 *
 * Every function exists in two modes:
 *   mode 0 (FP64): the definition, evaluated in double precision;
 *   mode 1 (FP32): the same steps in float, in a fixed operation order with no
 *                  fused multiply-add (the file is compiled with -ffp-contract=off),
 *                  so that tree, leaf ids, crossings and sample positions can be
 *                  compared bit for bit against a GPU path that follows the order.
 *
 * Steps and where they come from (paper sections):
 *   tree       Sec. 3.4 (BuildKDTree: split at the median of the cumulative density,
 *              recurse left then right; node index = binary path code, Sec. 3.1).
 *              TestLeaf (Sec. 3.4) needs a trained teacher; here a node is a leaf
 *              when it reaches the depth limit, when its mass is at most a fraction
 *              of the total, or when it is one cell wide.
 *   traversal  Sec. 3.5, Algorithm 1 (Traverse), read as ordered front-to-back
 *              KD-tree traversal that records one interval per leaf crossed.
 *   sampling   Sec. 3.5, Algorithm 1 (Sampling) and Fig. "prop": every interval is
 *              normalised and gets the same number of samples, stored per ray at
 *              ray * max_cell_count + j; placed at stratum midpoints, or (the paper's
 *              random placement within an interval) at one uniform point per stratum drawn
 *              from a counter-based generator keyed by the ray (see or_jitter_u).
 *   grouping   Sec. 3.5 and Fig. "parallel": samples sorted by node id so that each
 *              node's network runs as one batch.
 *   network    Sec. 3.1 (F_Theta(x, d) -> (c, sigma)), Sec. 3.2 and 4.1 (one small
 *              same-shaped MLP per node), sinusoidal positional encoding (Fig.
 *              "complex" caption).
 *   composite  Sec. 3.1 (classic volume rendering): NeRF quadrature with
 *              early ray termination.
 *   proposal   not in the paper (related work, Sec. 2.1: sampling networks);
 *              defined in the proposal section of this file.
 *
 * Parity pins live in the test suite (brute-force ray/box classification, closed
 * forms, invariants, library matmul chains, finite differences).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_STACK 128

/* ======================================================================== */
/* Tree build (Sec. 3.4)                                                     */
/* ======================================================================== */

/* Flat node record used by every oracle entry point.
 *   box[6]   = lo x, lo y, lo z, hi x, hi y, hi z   (float)
 *   cells[6] = cell range x0, y0, z0, x1, y1, z1     (half-open)
 *   info[6]  = axis (-1 for a leaf), left, right, leaf id (-1 inner), code, depth
 *   split    = split coordinate (float), mass = node mass (double)
 * Nodes are stored in preorder (node, left subtree, right subtree). */
typedef struct {
    const float *grid;
    int G;
    double blo[3], bhi[3];
    int max_depth;
    double leaf_frac;
    double total;
    int cap, n, n_leaves, err;
    float *box;
    int *cells, *info;
    float *split;
    double *mass;
    double *slice; /* scratch, G doubles */
} or_build;

static float or_coord(const or_build *b, int a, int i)
{
    /* cell boundary i along axis a, rounded once from double */
    double v = b->blo[a] + (b->bhi[a] - b->blo[a]) * ((double)i / (double)b->G);
    return (float)v;
}

/* longest axis in cells, ties to the lowest index */
static int or_longest(const int lo[3], const int hi[3])
{
    int a = 0;
    for (int k = 1; k < 3; k++)
        if (hi[k] - lo[k] > hi[a] - lo[a]) a = k;
    return a;
}

/* slice[i] = sum of the node's cells whose index along a is lo[a] + i; cells are
 * added in z-major, x-minor order.  Node mass = slice[0] + slice[1] + ... in order. */
static double or_slices(const or_build *b, const int lo[3], const int hi[3], int a, double *slice)
{
    int n = hi[a] - lo[a];
    for (int i = 0; i < n; i++) slice[i] = 0.0;
    for (int z = lo[2]; z < hi[2]; z++)
        for (int y = lo[1]; y < hi[1]; y++)
            for (int x = lo[0]; x < hi[0]; x++) {
                int idx = (a == 0) ? x : (a == 1) ? y : z;
                slice[idx - lo[a]] += (double)b->grid[((size_t)z * b->G + y) * b->G + x];
            }
    double m = 0.0;
    for (int i = 0; i < n; i++) m += slice[i];
    return m;
}

static int or_build_rec(or_build *b, const int lo[3], const int hi[3], int depth, uint32_t code)
{
    if (b->n >= b->cap) { b->err = 1; return -1; }
    int id = b->n++;
    int a = or_longest(lo, hi);
    int n = hi[a] - lo[a];
    double m = or_slices(b, lo, hi, a, b->slice);
    if (depth == 0) b->total = m;
    for (int k = 0; k < 3; k++) {
        b->box[6 * id + k] = or_coord(b, k, lo[k]);
        b->box[6 * id + 3 + k] = or_coord(b, k, hi[k]);
        b->cells[6 * id + k] = lo[k];
        b->cells[6 * id + 3 + k] = hi[k];
    }
    b->mass[id] = m;
    int *inf = b->info + 6 * id;
    inf[4] = (int)code;
    inf[5] = depth;
    int leaf = depth >= b->max_depth || n <= 1 || (b->leaf_frac > 0.0 && m <= b->leaf_frac * b->total);
    if (leaf) {
        inf[0] = -1; inf[1] = -1; inf[2] = -1; inf[3] = b->n_leaves++;
        b->split[id] = 0.0f;
        return id;
    }
    /* density-weighted median: the smallest k in [1, n-1] whose prefix mass reaches
     * half of the node mass; an empty node is halved */
    int ks;
    if (m == 0.0) {
        ks = n / 2;
    } else {
        double half = 0.5 * m, pre = 0.0;
        ks = n - 1;
        for (int k = 1; k <= n - 1; k++) {
            pre += b->slice[k - 1];
            if (pre >= half) { ks = k; break; }
        }
    }
    inf[0] = a; inf[3] = -1;
    b->split[id] = or_coord(b, a, lo[a] + ks);
    int llo[3] = {lo[0], lo[1], lo[2]}, lhi[3] = {hi[0], hi[1], hi[2]};
    int rlo[3] = {lo[0], lo[1], lo[2]}, rhi[3] = {hi[0], hi[1], hi[2]};
    lhi[a] = lo[a] + ks;
    rlo[a] = lo[a] + ks;
    int l = or_build_rec(b, llo, lhi, depth + 1, 2u * code);
    int r = or_build_rec(b, rlo, rhi, depth + 1, 2u * code + 1u);
    inf = b->info + 6 * id;
    inf[1] = l; inf[2] = r;
    return id;
}

/* Returns the node count (>0), or -1 when max_nodes is too small / input invalid. */
int or_build_tree(const float *grid, int G, const double *bbox6, int max_depth, double leaf_frac,
                  int max_nodes, float *box, int *cells, int *info, float *split, double *mass,
                  int *n_leaves)
{
    if (G < 1 || max_depth < 0) return -1;
    or_build b;
    memset(&b, 0, sizeof b);
    b.grid = grid; b.G = G; b.max_depth = max_depth; b.leaf_frac = leaf_frac; b.cap = max_nodes;
    for (int k = 0; k < 3; k++) { b.blo[k] = bbox6[k]; b.bhi[k] = bbox6[3 + k]; }
    b.box = box; b.cells = cells; b.info = info; b.split = split; b.mass = mass;
    b.slice = (double *)malloc(sizeof(double) * (size_t)G);
    int lo[3] = {0, 0, 0}, hi[3] = {G, G, G};
    or_build_rec(&b, lo, hi, 0, 1u);
    free(b.slice);
    if (b.err) return -1;
    *n_leaves = b.n_leaves;
    return b.n;
}

/* ======================================================================== */
/* Ray / box slab test and traversal (Sec. 3.5, Algorithm 1 Traverse)       */
/* ======================================================================== */

/* FP32: t0 = (lo - o) * inv, t1 = (hi - o) * inv per axis (subtract, round, multiply,
 * round); entry = max over x, y, z of min(t0, t1), exit = min of max(t0, t1), with
 * NaN-ignoring min/max; entry clamped at 0; a crossing exists iff exit > entry. */
static int or_slab32(const float *box, const float o[3], const float inv[3], float *tin, float *tout)
{
    float tmin[3], tmax[3];
    for (int a = 0; a < 3; a++) {
        float s0 = box[a] - o[a];
        float s1 = box[3 + a] - o[a];
        float t0 = s0 * inv[a];
        float t1 = s1 * inv[a];
        tmin[a] = fminf(t0, t1);
        tmax[a] = fmaxf(t0, t1);
    }
    float e = fmaxf(fmaxf(tmin[0], tmin[1]), tmin[2]);
    float x = fminf(fminf(tmax[0], tmax[1]), tmax[2]);
    e = fmaxf(e, 0.0f);
    *tin = e; *tout = x;
    return x > e;
}

static int or_slab64(const float *box, const double o[3], const double inv[3], double *tin, double *tout)
{
    double tmin[3], tmax[3];
    for (int a = 0; a < 3; a++) {
        double t0 = ((double)box[a] - o[a]) * inv[a];
        double t1 = ((double)box[3 + a] - o[a]) * inv[a];
        tmin[a] = fmin(t0, t1);
        tmax[a] = fmax(t0, t1);
    }
    double e = fmax(fmax(tmin[0], tmin[1]), tmin[2]);
    double x = fmin(fmin(tmax[0], tmax[1]), tmax[2]);
    e = fmax(e, 0.0);
    *tin = e; *tout = x;
    return x > e;
}

/* Adaptive hierarchical sampling (Sec. 3.5, Algorithm 1's HCheck; Fig. 1 (c)): the
 * paper leaves HCheck undefined beyond naming its inputs: the scene density and the camera distance.
 * Reading: a ray's footprint grows linearly with the distance travelled, so a node
 * whose subdivision is finer than the footprint cannot be resolved and its own
 * network takes the whole crossing.  An inner node is descended (HCheck true) iff
 * its extent along its split axis exceeds lod times the ray's entry distance into it
 * (lod = the footprint per unit distance times the number of footprints a node must
 * span to be refined); otherwise the inner node is emitted as one crossing with its
 * own network.  The density enters through the tree: density-median splits make
 * nodes small where the scene is dense, so dense distant parts stop early.  lod <= 0
 * descends everywhere (leaves only).  In FP32 mode the test is size > lod * entry
 * with the size hi - lo of the box along the axis (exact for dyadic boxes) and the
 * product rounded to float.  Networks: leaves 0 .. L-1 by leaf id, then the inner
 * nodes in preorder, L + rank. */
typedef struct or_hier_s {
    double lod;
    const int *net;   /* network id of every node */
    const int *parent;
} or_hier;

static int or_descends(const or_hier *H, int mode, const float *bx, int ax, double tin)
{
    if (!H || !(H->lod > 0.0)) return 1;
    if (mode == 1) {
        float size = bx[3 + ax] - bx[ax];
        float thr = (float)H->lod * (float)tin;
        return size > thr;
    }
    return ((double)bx[3 + ax] - (double)bx[ax]) > H->lod * tin;
}

/* Network ids and parents of every node (net: L + preorder rank for inner nodes). */
static void or_hier_tables(const int *info, int n_nodes, int *net, int *parent)
{
    int nl = 0, ni = 0;
    for (int i = 0; i < n_nodes; i++) if (info[6 * i] < 0) nl++;
    for (int i = 0; i < n_nodes; i++) parent[i] = -1;
    for (int i = 0; i < n_nodes; i++) {
        if (info[6 * i] < 0) { net[i] = info[6 * i + 3]; continue; }
        net[i] = nl + ni++;
        parent[info[6 * i + 1]] = i;
        parent[info[6 * i + 2]] = i;
    }
}

/* One ray: ordered list of crossings (network id, entry, exit), at most maxc.
 * method 0 = stack traversal (near child first: the child on the origin's side of the
 * split plane; an origin on the plane goes left when d <= 0 along the axis), method 1 =
 * the definition the stack form must reproduce: every leaf with a positive crossing
 * sorted by entry; with hierarchical sampling (H, lod > 0) every node with a positive
 * crossing whose strict ancestors all have positive crossings and descend, and which
 * is a leaf or does not descend, sorted by entry. */
static int or_trav_ray(const float *box, const int *info, const float *split, int n_nodes,
                       const float of[3], const float df[3], int maxc, int mode, int method,
                       const or_hier *H, int *leaf, double *tin, double *tout)
{
    float inv32[3];
    double o64[3], inv64[3];
    for (int a = 0; a < 3; a++) {
        inv32[a] = 1.0f / df[a];
        o64[a] = (double)of[a];
        inv64[a] = 1.0 / (double)df[a];
    }
    int cnt = 0;
    const int hier = H && H->lod > 0.0;
    if (method == 1 && hier) {
        int nl = 0;
        for (int i = 0; i < n_nodes; i++) {
            double a0 = 0.0, a1 = 0.0;
            int ok = 1;
            /* the node itself, then its ancestors up to the root */
            for (int j = i, first = 1; j >= 0 && ok; j = H->parent[j], first = 0) {
                double e, x;
                int hit;
                if (mode == 1) {
                    float ef, xf;
                    hit = or_slab32(box + 6 * j, of, inv32, &ef, &xf);
                    e = ef; x = xf;
                } else {
                    hit = or_slab64(box + 6 * j, o64, inv64, &e, &x);
                }
                if (!hit) { ok = 0; break; }
                const int ax = info[6 * j];
                const int desc = ax >= 0 && or_descends(H, mode, box + 6 * j, ax, e);
                if (first) {
                    if (desc) ok = 0;          /* an inner node that descends emits nothing */
                    a0 = e; a1 = x;
                } else if (!desc) {
                    ok = 0;                    /* an ancestor stopped above this node */
                }
            }
            if (!ok) continue;
            int p = nl;
            while (p > 0 && tin[p - 1] > a0) {
                if (p < maxc) { leaf[p] = leaf[p - 1]; tin[p] = tin[p - 1]; tout[p] = tout[p - 1]; }
                p--;
            }
            if (p < maxc) { leaf[p] = H->net[i]; tin[p] = a0; tout[p] = a1; }
            if (nl < maxc) nl++;
        }
        return nl;
    }
    if (method == 1) {
        int nl = 0;
        for (int i = 0; i < n_nodes; i++) {
            if (info[6 * i] != -1) continue;
            double a0, a1;
            int hit;
            if (mode == 1) {
                float e, x;
                hit = or_slab32(box + 6 * i, of, inv32, &e, &x);
                a0 = e; a1 = x;
            } else {
                hit = or_slab64(box + 6 * i, o64, inv64, &a0, &a1);
            }
            if (!hit) continue;
            /* insertion into the entry-sorted list (stable for equal entries) */
            int p = nl;
            while (p > 0 && tin[p - 1] > a0) {
                if (p < maxc) { leaf[p] = leaf[p - 1]; tin[p] = tin[p - 1]; tout[p] = tout[p - 1]; }
                p--;
            }
            if (p < maxc) { leaf[p] = info[6 * i + 3]; tin[p] = a0; tout[p] = a1; }
            if (nl < maxc) nl++;
        }
        return nl;
    }
    int stack[OR_MAX_STACK], sp = 0;
    stack[sp++] = 0;
    while (sp > 0 && cnt < maxc) {
        int nd = stack[--sp];
        double a0, a1;
        int hit;
        if (mode == 1) {
            float e, x;
            hit = or_slab32(box + 6 * nd, of, inv32, &e, &x);
            a0 = e; a1 = x;
        } else {
            hit = or_slab64(box + 6 * nd, o64, inv64, &a0, &a1);
        }
        if (!hit) continue;
        const int *inf = info + 6 * nd;
        if (inf[0] < 0) {
            leaf[cnt] = inf[3]; tin[cnt] = a0; tout[cnt] = a1; cnt++;
            continue;
        }
        int ax = inf[0];
        if (hier && !or_descends(H, mode, box + 6 * nd, ax, a0)) {
            leaf[cnt] = H->net[nd]; tin[cnt] = a0; tout[cnt] = a1; cnt++;
            continue;
        }
        int near_left = of[ax] < split[nd] || (of[ax] == split[nd] && df[ax] <= 0.0f);
        int nearc = near_left ? inf[1] : inf[2];
        int farc = near_left ? inf[2] : inf[1];
        if (sp + 2 > OR_MAX_STACK) return -1;
        stack[sp++] = farc;
        stack[sp++] = nearc;
    }
    return cnt;
}

/* Hierarchical-sampling context for lod > 0 (NULL otherwise); free with free(). */
static or_hier *or_hier_new(const int *info, int n_nodes, double lod)
{
    if (!(lod > 0.0)) return NULL;
    or_hier *H = (or_hier *)malloc(sizeof(or_hier) + 2 * sizeof(int) * (size_t)n_nodes);
    int *net = (int *)(H + 1);
    int *parent = net + n_nodes;
    or_hier_tables(info, n_nodes, net, parent);
    H->lod = lod; H->net = net; H->parent = parent;
    return H;
}

int or_traverse(const float *box, const int *info, const float *split, int n_nodes,
                const float *o, const float *d, int64_t n, int maxc, int mode, int method,
                int *n_x, int *leaf, double *tin, double *tout, double lod)
{
    or_hier *H = or_hier_new(info, n_nodes, lod);
    int rc = 0;
    for (int64_t r = 0; r < n && rc == 0; r++) {
        int c = or_trav_ray(box, info, split, n_nodes, o + 3 * r, d + 3 * r, maxc, mode, method, H,
                            leaf + r * maxc, tin + r * maxc, tout + r * maxc);
        if (c < 0) rc = -1;
        else n_x[r] = c;
    }
    free(H);
    return rc;
}

/* ======================================================================== */
/* Sampling (Sec. 3.5, Algorithm 1 Sampling; Fig. "prop")                   */
/* ======================================================================== */

/* Stratified jitter (Sec. 3.5: the samples of an interval may be placed at random
 * within it): sample j of crossing k of a ray sits at fraction u of its
 * stratum, u = (splitmix64 output >> 40) / 2^24 in [0, 1).  splitmix64 (Steele, Lea
 * and Flood, 2014) finalises z: z ^= z >> 30, z *= 0xbf58476d1ce4e5b9, z ^= z >> 27,
 * z *= 0x94d049bb133111eb, z ^= z >> 31.  The ray's key folds the bit patterns of its
 * origin and direction into the seed with three finalisations (so a ray draws the
 * same points whatever batch it is rendered in); the sample's input is the key plus
 * the golden gamma 0x9e3779b97f4a7c15 times (k * steps + j + 1).  Seed 0 means
 * midpoints (u = 1/2). */
static uint64_t or_mix64(uint64_t z)
{
    z ^= z >> 30; z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27; z *= 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return z;
}

static uint64_t or_ray_key(uint64_t seed, const float o[3], const float d[3])
{
    uint32_t b[6];
    memcpy(b, o, 12);
    memcpy(b + 3, d, 12);
    uint64_t k = or_mix64(seed ^ ((uint64_t)b[0] | ((uint64_t)b[1] << 32)));
    k = or_mix64(k ^ ((uint64_t)b[2] | ((uint64_t)b[3] << 32)));
    k = or_mix64(k ^ ((uint64_t)b[4] | ((uint64_t)b[5] << 32)));
    return k;
}

static float or_jitter_u(uint64_t seed, uint64_t key, int k, int steps, int j)
{
    if (seed == 0) return 0.5f;
    uint64_t z = or_mix64(key + 0x9e3779b97f4a7c15ULL * (uint64_t)(k * steps + j + 1));
    return (float)(z >> 40) * (1.0f / 16777216.0f);
}

/* The generator's pieces, for the pins: the finaliser, and sample j's fraction. */
uint64_t or_splitmix64_mix(uint64_t z) { return or_mix64(z); }

float or_jitter_fraction(uint64_t seed, const float *o, const float *d, int k, int steps, int j)
{
    return or_jitter_u(seed, or_ray_key(seed, o, d), k, steps, j);
}

/* Sample j of a crossing at fraction u of its stratum: delta = (exit - entry) / steps,
 * t_j = entry + (j + u) delta, x_j = o + t_j d per component (multiply, round, add,
 * round). */
static void or_sample32(float e, float x, int steps, int j, float u, const float o[3], const float d[3],
                        float *t, float *dl, float p[3])
{
    float len = x - e;
    float delta = len / (float)steps;
    float fj = (float)j + u;
    float off = fj * delta;
    float tj = e + off;
    for (int a = 0; a < 3; a++) {
        float m = tj * d[a];
        p[a] = o[a] + m;
    }
    *t = tj; *dl = delta;
}

static void or_sample64(double e, double x, int steps, int j, double u, const double o[3], const double d[3],
                        double *t, double *dl, double p[3])
{
    double delta = (x - e) / (double)steps;
    double tj = e + ((double)j + u) * delta;
    for (int a = 0; a < 3; a++) p[a] = o[a] + tj * d[a];
    *t = tj; *dl = delta;
}

/* Samples of every ray in slot layout (slot = ray * cap + k * steps + j). */
int or_samples(const float *o, const float *d, int64_t n, const int *n_x, const double *tin,
               const double *tout, int maxc, int steps, int cap, int mode, uint64_t jitter,
               double *t_out, double *delta_out, double *x_out)
{
    for (int64_t r = 0; r < n; r++) {
        const uint64_t key = or_ray_key(jitter, o + 3 * r, d + 3 * r);
        for (int k = 0; k < n_x[r]; k++) {
            for (int j = 0; j < steps; j++) {
                int64_t s = r * cap + (int64_t)k * steps + j;
                const float u = or_jitter_u(jitter, key, k, steps, j);
                if (mode == 1) {
                    float t, dl, p[3];
                    or_sample32((float)tin[r * maxc + k], (float)tout[r * maxc + k], steps, j, u,
                                o + 3 * r, d + 3 * r, &t, &dl, p);
                    t_out[s] = t; delta_out[s] = dl;
                    for (int a = 0; a < 3; a++) x_out[3 * s + a] = p[a];
                } else {
                    double o64[3] = {o[3 * r], o[3 * r + 1], o[3 * r + 2]};
                    double d64[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
                    double t, dl, p[3];
                    or_sample64(tin[r * maxc + k], tout[r * maxc + k], steps, j, (double)u, o64, d64, &t, &dl, p);
                    t_out[s] = t; delta_out[s] = dl;
                    for (int a = 0; a < 3; a++) x_out[3 * s + a] = p[a];
                }
            }
        }
    }
    return 0;
}

/* ======================================================================== */
/* Empty-space skipping (Sec. 4.1: the finer density grid also serves "empty */
/* space detection")                                                         */
/* ======================================================================== */

/* The guidance grid as an occupancy grid: a cell is occupied when its density
 * exceeds thr.  The cell of a coordinate p on axis a is floor((p - lo_a) * sc_a),
 * sc_a = G / (hi_a - lo_a), clamped to [0, G - 1] (in the mode's precision, the
 * FP32 product rounded once). */
typedef struct {
    const float *grid; int G; float thr;
    float lo32[3], sc32[3]; double lo64[3], sc64[3];
    int steps; uint64_t jitter;
} or_occ;

static int or_clampc(long long c, int G) { return c < 0 ? 0 : (c > G - 1 ? G - 1 : (int)c); }

/* 1 when a sample of crossing [tin, tout], placed as the k-th kept crossing of the
 * ray (its jitter depends on k), lies in an occupied cell. */
static int or_crossing_occupied(const or_occ *oc, int mode, uint64_t key, const float of[3], const float df[3],
                                double tin, double tout, int k)
{
    const int G = oc->G;
    for (int j = 0; j < oc->steps; j++) {
        const float u = or_jitter_u(oc->jitter, key, k, oc->steps, j);
        int c[3];
        if (mode == 1) {
            float t, dl, p[3];
            or_sample32((float)tin, (float)tout, oc->steps, j, u, of, df, &t, &dl, p);
            for (int a = 0; a < 3; a++) {
                float q = p[a] - oc->lo32[a];
                float f = q * oc->sc32[a];
                c[a] = or_clampc((long long)floorf(f), G);
            }
        } else {
            double o64[3] = {of[0], of[1], of[2]}, d64[3] = {df[0], df[1], df[2]};
            double t, dl, p[3];
            or_sample64(tin, tout, oc->steps, j, (double)u, o64, d64, &t, &dl, p);
            for (int a = 0; a < 3; a++) c[a] = or_clampc((long long)floor((p[a] - oc->lo64[a]) * oc->sc64[a]), G);
        }
        if (oc->grid[(size_t)c[0] + (size_t)G * ((size_t)c[1] + (size_t)G * (size_t)c[2])] > oc->thr) return 1;
    }
    return 0;
}

static void or_occ_init(or_occ *oc, const float *grid, int G, const double *bbox6, double thr, int steps,
                        uint64_t jitter)
{
    oc->grid = grid; oc->G = G; oc->thr = (float)thr; oc->steps = steps; oc->jitter = jitter;
    for (int a = 0; a < 3; a++) {
        oc->lo64[a] = bbox6[a];
        oc->sc64[a] = (double)G / (bbox6[3 + a] - bbox6[a]);
        oc->lo32[a] = (float)bbox6[a];
        oc->sc32[a] = (float)oc->sc64[a];
    }
}

/* ======================================================================== */
/* Grouping by leaf (Sec. 3.5, Fig. "parallel")                             */
/* ======================================================================== */

/* counts[l] = samples whose crossing lies in leaf l (= steps x crossings);
 * offsets = exclusive scan of counts (n_leaves + 1 entries);
 * order = crossing ids (ray * maxc + k) grouped by leaf, ascending inside a leaf. */
int or_group(const int *n_x, const int *leaf, int64_t n, int maxc, int steps, int n_leaves,
             int64_t *counts, int64_t *offsets, int64_t *order)
{
    int64_t *cur = (int64_t *)calloc((size_t)n_leaves + 1, sizeof(int64_t));
    for (int l = 0; l < n_leaves; l++) counts[l] = 0;
    for (int64_t r = 0; r < n; r++)
        for (int k = 0; k < n_x[r]; k++) {
            int l = leaf[r * maxc + k];
            if (l < 0 || l >= n_leaves) { free(cur); return -1; }
            counts[l] += steps;
        }
    offsets[0] = 0;
    for (int l = 0; l < n_leaves; l++) offsets[l + 1] = offsets[l] + counts[l];
    for (int l = 0; l < n_leaves; l++) cur[l] = offsets[l] / steps;
    for (int64_t r = 0; r < n; r++)
        for (int k = 0; k < n_x[r]; k++) {
            int l = leaf[r * maxc + k];
            order[cur[l]++] = r * maxc + k;
        }
    free(cur);
    return 0;
}

/* ======================================================================== */
/* Frequency positional encoding and the per-leaf MLP (Sec. 3.1, 3.3, 4.1)   */
/* ======================================================================== */

/* gamma_L(p) = [p, sin(pi 2^0 p), cos(pi 2^0 p), ..., sin(pi 2^(L-1) p), cos(pi 2^(L-1) p)],
 * each term a 3-vector.  2^k p is exact; it is reduced exactly to r in [-1, 1]
 * (remainder by 2) before sin(pi r), cos(pi r) are taken in double. */
static void or_encode64(const double p[3], int L, double *out)
{
    for (int a = 0; a < 3; a++) out[a] = p[a];
    for (int k = 0; k < L; k++)
        for (int a = 0; a < 3; a++) {
            double r = remainder(ldexp(p[a], k), 2.0);
            out[3 + 6 * k + a] = sin(M_PI * r);
            out[3 + 6 * k + 3 + a] = cos(M_PI * r);
        }
}

static void or_encode32(const float p[3], int L, float *out)
{
    for (int a = 0; a < 3; a++) out[a] = p[a];
    for (int k = 0; k < L; k++)
        for (int a = 0; a < 3; a++) {
            float r = remainderf(ldexpf(p[a], k), 2.0f);
            out[3 + 6 * k + a] = (float)sin(M_PI * (double)r);
            out[3 + 6 * k + 3 + a] = (float)cos(M_PI * (double)r);
        }
}

void or_encode(const double *p, int L, int mode, double *out)
{
    if (mode == 1) {
        float pf[3] = {(float)p[0], (float)p[1], (float)p[2]};
        float tmp[3 + 6 * 32];
        or_encode32(pf, L, tmp);
        for (int i = 0; i < 3 + 6 * L; i++) out[i] = tmp[i];
    } else {
        or_encode64(p, L, out);
    }
}

static double or_softplus64(double z) { return z > 20.0 ? z : log1p(exp(z)); }
static double or_sigmoid64(double z) { return 1.0 / (1.0 + exp(-z)); }
static float or_softplus32(float z) { return z > 20.0f ? z : log1pf(expf(z)); }
static float or_sigmoid32(float z) { return 1.0f / (1.0f + expf(-z)); }

#define OR_MAXW 256
#define OR_MAXK 512

/* h_0 = input (k0 wide); h_{l+1} = ReLU(W_l h_l + b_l) for `hidden` layers of `width`;
 * raw = W_o h_H + b_o (4 wide); sigma = softplus(raw_0), rgb = sigmoid(raw_1..3).
 * Each dot product is summed over the input index in ascending order, then the bias
 * is added.  out = sigma, r, g, b; raw (may be NULL) = pre-activation head. */
static void or_mlp64(const float *P, int width, int hidden, int k0, const double *in, double *out, double *raw,
                     double *in_absmax)
{
    double h[OR_MAXK], g[OR_MAXW];
    int kin = k0;
    for (int i = 0; i < k0; i++) h[i] = in[i];
    const float *w = P;
    for (int l = 0; l < hidden; l++) {
        if (in_absmax)  /* largest |input| of layer l (the E4M3 activation scale's range) */
            for (int i = 0; i < kin; i++) in_absmax[l] = fabs(h[i]) > in_absmax[l] ? fabs(h[i]) : in_absmax[l];
        const float *b = w + (size_t)width * kin;
        for (int o = 0; o < width; o++) {
            double acc = 0.0;
            for (int i = 0; i < kin; i++) acc += (double)w[(size_t)o * kin + i] * h[i];
            acc += (double)b[o];
            g[o] = acc > 0.0 ? acc : 0.0;
        }
        for (int o = 0; o < width; o++) h[o] = g[o];
        w = b + width;
        kin = width;
    }
    const float *b = w + 4 * width;
    double z[4];
    for (int o = 0; o < 4; o++) {
        double acc = 0.0;
        for (int i = 0; i < width; i++) acc += (double)w[o * width + i] * h[i];
        z[o] = acc + (double)b[o];
    }
    if (raw) for (int o = 0; o < 4; o++) raw[o] = z[o];
    out[0] = or_softplus64(z[0]);
    for (int o = 1; o < 4; o++) out[o] = or_sigmoid64(z[o]);
}

static void or_mlp32(const float *P, int width, int hidden, int k0, const float *in, float *out, float *raw)
{
    float h[OR_MAXK], g[OR_MAXW];
    int kin = k0;
    for (int i = 0; i < k0; i++) h[i] = in[i];
    const float *w = P;
    for (int l = 0; l < hidden; l++) {
        const float *b = w + (size_t)width * kin;
        for (int o = 0; o < width; o++) {
            float acc = 0.0f;
            for (int i = 0; i < kin; i++) {
                float m = w[(size_t)o * kin + i] * h[i];
                acc = acc + m;
            }
            acc = acc + b[o];
            g[o] = acc > 0.0f ? acc : 0.0f;
        }
        for (int o = 0; o < width; o++) h[o] = g[o];
        w = b + width;
        kin = width;
    }
    const float *b = w + 4 * width;
    float z[4];
    for (int o = 0; o < 4; o++) {
        float acc = 0.0f;
        for (int i = 0; i < width; i++) {
            float m = w[o * width + i] * h[i];
            acc = acc + m;
        }
        z[o] = acc + b[o];
    }
    if (raw) for (int o = 0; o < 4; o++) raw[o] = z[o];
    out[0] = or_softplus32(z[0]);
    for (int o = 1; o < 4; o++) out[o] = or_sigmoid32(z[o]);
}

/* Network of one leaf on n (x, d) pairs: encodes gamma_lx(x) ++ gamma_ld(d) and runs the
 * MLP.  out is (n, 4): sigma, r, g, b; raw (may be NULL) is (n, 4) pre-activations. */
int or_mlp_eval(const float *P, int width, int hidden, int lx, int ld, const double *x, const double *d,
                int64_t n, int mode, double *out, double *raw)
{
    int kx = 3 + 6 * lx, kd = 3 + 6 * ld, k0 = kx + kd;
    if (width > OR_MAXW || k0 > OR_MAXK || lx > 32 || ld > 32) return -1;
    for (int64_t s = 0; s < n; s++) {
        if (mode == 1) {
            float px[3] = {(float)x[3 * s], (float)x[3 * s + 1], (float)x[3 * s + 2]};
            float pd[3] = {(float)d[3 * s], (float)d[3 * s + 1], (float)d[3 * s + 2]};
            float in[OR_MAXK], o4[4], r4[4];
            or_encode32(px, lx, in);
            or_encode32(pd, ld, in + kx);
            or_mlp32(P, width, hidden, k0, in, o4, r4);
            for (int i = 0; i < 4; i++) { out[4 * s + i] = o4[i]; if (raw) raw[4 * s + i] = r4[i]; }
        } else {
            double in[OR_MAXK];
            or_encode64(x + 3 * s, lx, in);
            or_encode64(d + 3 * s, ld, in + kx);
            or_mlp64(P, width, hidden, k0, in, out + 4 * s, raw ? raw + 4 * s : NULL, NULL);
        }
    }
    return 0;
}

/* Largest |input| of every hidden layer over n samples of one leaf's network (FP64):
 * amax[l] for l < hidden, l = 0 being the encoded input.  The range an E4M3
 * activation scale a_l = amax[l] / 448 must cover (a quantisation choice; the paper
 * uses half-precision networks, Sec. 4.1). */
int or_mlp_input_absmax(const float *P, int width, int hidden, int lx, int ld, const double *x, const double *d,
                        int64_t n, double *amax)
{
    int kx = 3 + 6 * lx, kd = 3 + 6 * ld, k0 = kx + kd;
    if (width > OR_MAXW || k0 > OR_MAXK || lx > 32 || ld > 32) return -1;
    for (int l = 0; l < hidden; l++) amax[l] = 0.0;
    for (int64_t s = 0; s < n; s++) {
        double in[OR_MAXK], o4[4];
        or_encode64(x + 3 * s, lx, in);
        or_encode64(d + 3 * s, ld, in + kx);
        or_mlp64(P, width, hidden, k0, in, o4, NULL, amax);
    }
    return 0;
}

/* ======================================================================== */
/* Full render: traversal, sampling, network, compositing (Sec. 3.1, 3.5)   */
/* ======================================================================== */

typedef struct {
    /* tree */
    const float *box; const int *info; const float *split; int n_nodes;
    /* networks */
    const float *params; int64_t per_leaf; int width, hidden, lx, ld;
    /* rays */
    const float *o, *d; int64_t n;
    /* render params */
    int steps, cap; double t_term; double bg[3]; int mode; uint64_t jitter;
    const or_occ *occ;  /* empty-space skipping (NULL: off) */
    /* outputs */
    double *rgb, *depth, *opacity; int *n_gen, *n_eval; double *ert_margin;
    double *slot_out; /* (n, cap, 4) sigma rgb; may be NULL */
    double *slot_w;   /* (n, cap) compositing weight; may be NULL */
    double *t_final;  /* (n) final transmittance; may be NULL */
    /* proposal: per-ray kept-bin mask and fallback flag (both NULL = plain) */
    const uint64_t *mask; const int *fallback;
    double *bins;     /* (n, 65) compositing weight per depth bin + residual T; may be NULL */
    /* FP64 mode only: round each sample's (sigma, r, g, b) to binary16 before it is
     * composited (sigma first limited to the largest binary16 value), to measure the
     * effect of a half-precision per-sample store on its own */
    int slot_f16;
    /* adaptive hierarchical sampling (NULL: leaves only); crossings then carry
     * network ids, leaves first, inner nodes after them in preorder */
    const struct or_hier_s *hier;
    /* threading */
    int64_t r0, r1; int err;
} or_job;

/* Round to the nearest IEEE binary16 value (11 significant bits, ties to even;
 * subnormal spacing 2^-24 below 2^-14).  Inputs are finite with |x| <= 65504. */
static double or_f16(double x)
{
    if (x == 0.0) return x;
    if (fabs(x) < ldexp(1.0, -14)) return ldexp(nearbyint(ldexp(x, 24)), -24);
    int e;
    double m = frexp(x, &e);
    return ldexp(nearbyint(ldexp(m, 11)), e - 11);
}

int or_f16_round_n(const double *x, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = or_f16(x[i]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Proposal sampler support (not in the paper; a learned sampler in the      */
/* spirit of the sampling networks of the related work, Sec. 2.1).  Depth    */
/* bins: the ray's root interval [t0, t1] cut into 64 equal bins; bin k is    */
/* [t0 + k w, t0 + (k + 1) w) with w = (t1 - t0) / 64, evaluated in the       */
/* mode's precision in that operation order.                                 */
/* ------------------------------------------------------------------------ */

/* Root interval of one ray (the slab test of node 0); 0 when the ray misses. */
static int or_root(const float *box, const float *of, const float *df, int mode, double *t0, double *t1)
{
    if (mode == 1) {
        float inv[3] = {1.0f / df[0], 1.0f / df[1], 1.0f / df[2]};
        float e, x;
        int hit = or_slab32(box, of, inv, &e, &x);
        *t0 = hit ? e : 0.0; *t1 = hit ? x : 0.0;
        return hit;
    }
    double o64[3] = {of[0], of[1], of[2]};
    double inv[3] = {1.0 / (double)df[0], 1.0 / (double)df[1], 1.0 / (double)df[2]};
    double e, x;
    int hit = or_slab64(box, o64, inv, &e, &x);
    *t0 = hit ? e : 0.0; *t1 = hit ? x : 0.0;
    return hit;
}

/* Bin of a sample at t (training targets; clamped to [0, 63]): floor((t - t0) / w),
 * in the mode's precision (FP32: w = (t1 - t0) * 2^-6, then subtract, divide, floor). */
static int or_bin_of(int mode, double t0, double t1, double t)
{
    int k;
    if (mode == 1) {
        float w = ((float)t1 - (float)t0) * 0.015625f;
        float q = ((float)t - (float)t0) / w;
        k = w > 0.0f ? (int)floorf(q) : 0;
    } else {
        double w = (t1 - t0) / 64.0;
        k = w > 0.0 ? (int)floor((t - t0) / w) : 0;
    }
    return k < 0 ? 0 : (k > 63 ? 63 : k);
}

/* Bins of n samples (training-target binning, exported for its pins). */
int or_bin_indices(int mode, const double *t0, const double *t1, const double *t, int64_t n, int *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = or_bin_of(mode, t0[i], t1[i], t[i]);
    return 0;
}

/* Does crossing [a, b] overlap bin k?  a < hi_k and b > lo_k. */
static int or_overlaps(int mode, double t0, double t1, int k, double a, double b)
{
    if (mode == 1) {
        float w = ((float)t1 - (float)t0) * 0.015625f;
        float lo = (float)t0 + (float)k * w;
        float hi = (float)t0 + (float)(k + 1) * w;
        return (float)a < hi && (float)b > lo;
    }
    double w = (t1 - t0) / 64.0;
    return a < t0 + (k + 1) * w && b > t0 + k * w;
}

/* Keep, in order and at most maxc, the crossings that overlap a bin of *mask (when
 * mask != NULL) and have a sample in an occupied cell (when oc != NULL; the sample
 * placed as the crossing's index among the kept ones). */
static int or_keep(int mode, const uint64_t *mask, double t0, double t1, const or_occ *oc, uint64_t key,
                   const float *of, const float *df, int *leaf, double *tin, double *tout, int n, int maxc)
{
    int m = 0;
    for (int i = 0; i < n && m < maxc; i++) {
        if (mask) {
            int keep = 0;
            for (int k = 0; k < 64 && !keep; k++)
                if ((*mask >> k) & 1ull) keep = or_overlaps(mode, t0, t1, k, tin[i], tout[i]);
            if (!keep) continue;
        }
        if (oc && !or_crossing_occupied(oc, mode, key, of, df, tin[i], tout[i], m)) continue;
        leaf[m] = leaf[i]; tin[m] = tin[i]; tout[m] = tout[i]; m++;
    }
    return m;
}

/* Traversal with empty-space skipping: every crossing in order, then the occupied
 * ones kept (at most maxc), each tested with its samples placed as the kept index. */
int or_traverse_skip(const float *box, const int *info, const float *split, int n_nodes,
                     const float *o, const float *d, int64_t n, int maxc, int mode, int method, int steps,
                     uint64_t jitter, const float *occ_grid, int occ_G, const double *occ_bbox, double occ_thr,
                     int *n_x, int *leaf, double *tin, double *tout, double lod)
{
    or_occ oc;
    or_occ_init(&oc, occ_grid, occ_G, occ_bbox, occ_thr, steps, jitter);
    or_hier *H = or_hier_new(info, n_nodes, lod);
    for (int64_t r = 0; r < n; r++) {
        int lf[256];
        double a[256], b[256];
        int c = or_trav_ray(box, info, split, n_nodes, o + 3 * r, d + 3 * r, 256, mode, method, H, lf, a, b);
        if (c < 0) { free(H); return -1; }
        c = or_keep(mode, NULL, 0.0, 0.0, &oc, or_ray_key(jitter, o + 3 * r, d + 3 * r), o + 3 * r, d + 3 * r, lf, a,
                    b, c, maxc);
        for (int i = 0; i < c; i++) {
            leaf[r * maxc + i] = lf[i]; tin[r * maxc + i] = a[i]; tout[r * maxc + i] = b[i];
        }
        n_x[r] = c;
    }
    free(H);
    return 0;
}

/* Compositing (NeRF quadrature, Sec. 3.1): T = 1; per sample in ray order, stop once
 * T < t_term; tau = sigma * delta, e = exp(-tau), alpha = 1 - e, w = T alpha,
 * C += w c, D += w t, T = T e.  rgb = C + T bg, depth = D, opacity = 1 - T. */
static void or_render_ray(const or_job *J, int64_t r)
{
    int maxc = J->cap / J->steps;
    int leaf[256];
    double tin[256], tout[256];
    int kx = 3 + 6 * J->lx, k0 = kx + 3 + 6 * J->ld;
    int nx;
    double root0 = 0.0, root1 = 0.0;
    int root_hit = or_root(J->box, J->o + 3 * r, J->d + 3 * r, J->mode, &root0, &root1);
    const int masked = J->mask && !J->fallback[r];
    if (masked || J->occ) {
        nx = or_trav_ray(J->box, J->info, J->split, J->n_nodes, J->o + 3 * r, J->d + 3 * r,
                         256, J->mode, 0, J->hier, leaf, tin, tout);
        if (nx < 0) nx = 0;
        nx = or_keep(J->mode, masked ? J->mask + r : NULL, root0, root1, J->occ,
                     or_ray_key(J->jitter, J->o + 3 * r, J->d + 3 * r), J->o + 3 * r, J->d + 3 * r, leaf, tin,
                     tout, nx, maxc);
    } else {
        nx = or_trav_ray(J->box, J->info, J->split, J->n_nodes, J->o + 3 * r, J->d + 3 * r,
                         maxc, J->mode, 0, J->hier, leaf, tin, tout);
        if (nx < 0) nx = 0;
    }
    double *bins = J->bins ? J->bins + r * 65 : NULL;
    if (bins) for (int b = 0; b < 65; b++) bins[b] = 0.0;
    const float *of = J->o + 3 * r, *df = J->d + 3 * r;
    int full = J->slot_out != NULL || J->slot_w != NULL;
    int nev = 0, stopped = 0;
    double margin = INFINITY;
    double lt = log(J->t_term);
    const uint64_t key = or_ray_key(J->jitter, J->o + 3 * r, J->d + 3 * r);
    if (J->slot_w) for (int s = 0; s < J->cap; s++) J->slot_w[r * J->cap + s] = 0.0;
    if (J->mode == 1) {
        float T = 1.0f, C[3] = {0, 0, 0}, D = 0.0f;
        float tterm = (float)J->t_term;
        float din[OR_MAXK];
        or_encode32(df, J->ld, din + kx);
        for (int k = 0; k < nx && !(stopped && !full); k++) {
            const float *P = J->params + (size_t)leaf[k] * J->per_leaf;
            for (int j = 0; j < J->steps; j++) {
                int s = k * J->steps + j;
                if (!stopped) {
                    double m = fabs(log((double)T) - lt);
                    if (m < margin) margin = m;
                    if (T < tterm) stopped = 1;
                }
                if (stopped && !full) break;
                float t, dl, p[3], o4[4];
                or_sample32((float)tin[k], (float)tout[k], J->steps, j, or_jitter_u(J->jitter, key, k, J->steps, j), of,
                            df, &t, &dl, p);
                or_encode32(p, J->lx, din);
                or_mlp32(P, J->width, J->hidden, k0, din, o4, NULL);
                if (J->slot_out) for (int i = 0; i < 4; i++) J->slot_out[(r * J->cap + s) * 4 + i] = o4[i];
                if (stopped) continue;
                float tau = o4[0] * dl;
                float e = expf(-tau);
                float al = 1.0f - e;
                float w = T * al;
                for (int c = 0; c < 3; c++) { float wc = w * o4[1 + c]; C[c] = C[c] + wc; }
                float wt = w * t;
                D = D + wt;
                T = T * e;
                nev++;
                if (J->slot_w) J->slot_w[r * J->cap + s] = w;
                if (bins && root_hit) bins[or_bin_of(J->mode, root0, root1, t)] += w;
            }
        }
        if (bins) bins[64] = T;
        for (int c = 0; c < 3; c++) { float tb = T * (float)J->bg[c]; J->rgb[3 * r + c] = C[c] + tb; }
        J->depth[r] = D;
        J->opacity[r] = 1.0f - T;
        if (J->t_final) J->t_final[r] = T;
    } else {
        double T = 1.0, C[3] = {0, 0, 0}, D = 0.0;
        double o64[3] = {of[0], of[1], of[2]}, d64[3] = {df[0], df[1], df[2]};
        double din[OR_MAXK];
        or_encode64(d64, J->ld, din + kx);
        for (int k = 0; k < nx && !(stopped && !full); k++) {
            const float *P = J->params + (size_t)leaf[k] * J->per_leaf;
            for (int j = 0; j < J->steps; j++) {
                int s = k * J->steps + j;
                if (!stopped) {
                    double m = fabs(log(T) - lt);
                    if (m < margin) margin = m;
                    if (T < J->t_term) stopped = 1;
                }
                if (stopped && !full) break;
                double t, dl, p[3], o4[4];
                or_sample64(tin[k], tout[k], J->steps, j, (double)or_jitter_u(J->jitter, key, k, J->steps, j), o64,
                            d64, &t, &dl, p);
                or_encode64(p, J->lx, din);
                or_mlp64(P, J->width, J->hidden, k0, din, o4, NULL, NULL);
                if (J->slot_f16) {
                    if (o4[0] > 65504.0) o4[0] = 65504.0;
                    for (int i = 0; i < 4; i++) o4[i] = or_f16(o4[i]);
                }
                if (J->slot_out) for (int i = 0; i < 4; i++) J->slot_out[(r * J->cap + s) * 4 + i] = o4[i];
                if (stopped) continue;
                double e = exp(-o4[0] * dl);
                double w = T * (1.0 - e);
                for (int c = 0; c < 3; c++) C[c] += w * o4[1 + c];
                D += w * t;
                T *= e;
                nev++;
                if (J->slot_w) J->slot_w[r * J->cap + s] = w;
                if (bins && root_hit) bins[or_bin_of(J->mode, root0, root1, t)] += w;
            }
        }
        if (bins) bins[64] = T;
        for (int c = 0; c < 3; c++) J->rgb[3 * r + c] = C[c] + T * J->bg[c];
        J->depth[r] = D;
        J->opacity[r] = 1.0 - T;
        if (J->t_final) J->t_final[r] = T;
    }
    J->n_gen[r] = nx * J->steps;
    J->n_eval[r] = nev;
    J->ert_margin[r] = margin;
}

static void *or_render_worker(void *arg)
{
    or_job *J = (or_job *)arg;
    for (int64_t r = J->r0; r < J->r1; r++) or_render_ray(J, r);
    return NULL;
}

int or_render(const float *box, const int *info, const float *split, int n_nodes,
              const float *params, int width, int hidden, int lx, int ld,
              const float *o, const float *d, int64_t n,
              int steps, int cap, double t_term, const double *bg, int mode, uint64_t jitter,
              const float *occ_grid, int occ_G, const double *occ_bbox, double occ_thr, int n_threads,
              double *rgb, double *depth, double *opacity, int *n_gen, int *n_eval, double *ert_margin,
              double *slot_out, double *slot_w, double *t_final, const uint64_t *mask, const int *fallback,
              double *bins, int slot_f16, double lod)
{
    if (steps < 1 || cap < steps || cap / steps > 256 || width > OR_MAXW || lx > 32 || ld > 32) return -1;
    if (n_threads < 1) n_threads = 1;
    int k0 = 3 + 6 * lx + 3 + 6 * ld;
    or_job base;
    memset(&base, 0, sizeof base);
    base.box = box; base.info = info; base.split = split; base.n_nodes = n_nodes;
    base.params = params; base.width = width; base.hidden = hidden; base.lx = lx; base.ld = ld;
    base.per_leaf = (int64_t)width * k0 + width + (int64_t)(hidden - 1) * (width * width + width) + 4 * width + 4;
    base.o = o; base.d = d; base.n = n; base.steps = steps; base.cap = cap; base.t_term = t_term;
    for (int c = 0; c < 3; c++) base.bg[c] = bg[c];
    base.mode = mode;
    base.jitter = jitter;
    or_occ oc;
    if (occ_grid) {
        or_occ_init(&oc, occ_grid, occ_G, occ_bbox, occ_thr, steps, jitter);
        base.occ = &oc;
    }
    base.rgb = rgb; base.depth = depth; base.opacity = opacity; base.n_gen = n_gen; base.n_eval = n_eval;
    base.ert_margin = ert_margin; base.slot_out = slot_out; base.slot_w = slot_w; base.t_final = t_final;
    base.mask = mask; base.fallback = fallback; base.bins = bins;
    base.slot_f16 = mode == 0 ? slot_f16 : 0;
    or_hier *H = or_hier_new(info, n_nodes, lod);
    base.hier = H;
    if (n_threads == 1 || n < 64) {
        base.r0 = 0; base.r1 = n;
        or_render_worker(&base);
        free(H);
        return 0;
    }
    or_job *jobs = (or_job *)malloc(sizeof(or_job) * (size_t)n_threads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    int64_t chunk = (n + n_threads - 1) / n_threads;
    int started = 0;
    for (int i = 0; i < n_threads; i++) {
        jobs[i] = base;
        jobs[i].r0 = (int64_t)i * chunk;
        jobs[i].r1 = jobs[i].r0 + chunk < n ? jobs[i].r0 + chunk : n;
        if (jobs[i].r0 >= n) break;
        if (pthread_create(&th[i], NULL, or_render_worker, &jobs[i]) != 0) {
            or_render_worker(&jobs[i]);
            th[i] = 0;
        }
        started = i + 1;
    }
    for (int i = 0; i < started; i++) if (th[i]) pthread_join(th[i], NULL);
    free(jobs); free(th); free(H);
    return 0;
}

/* ======================================================================== */
/* Proposal network (not in the paper; see the proposal sampler section).   */
/* Input: gamma_10(entry point o + t0 d) ++ gamma_4(d) (90); two ReLU layers */
/* of 32; 65 logits (64 depth bins + background); softmax.                   */
/* Parameters, FP32 flat: W1 [32 x 90], b1 [32], W2 [32 x 32], b2 [32],      */
/* W3 [65 x 32], b3 [65] (6113 values).  Loss: mean over rays of the cross-  */
/* entropy -sum_b p_b log q_b against the binned compositing weights p.      */
/* ======================================================================== */

#define OR_PIN 90
#define OR_PH 32
#define OR_PO 65
#define OR_PNPAR (OR_PH * OR_PIN + OR_PH + OR_PH * OR_PH + OR_PH + OR_PO * OR_PH + OR_PO)

/* The entry point is an FP32 quantity like the rays and the root interval it comes
 * from: e = o + t0 d with the product and the sum each rounded to float; its
 * encoding is then evaluated in double. */
static void or_prop_input(const float *of, const float *df, double t0, double *in)
{
    double e[3], d[3];
    for (int a = 0; a < 3; a++) {
        float m = (float)t0 * df[a];
        float ef = of[a] + m;
        d[a] = df[a];
        e[a] = ef;
    }
    or_encode64(e, 10, in);
    or_encode64(d, 4, in + 63);
}

/* Round to the nearest bfloat16 value (8 significant bits, ties to even); the
 * operand precision of a tensor-core evaluation.  Finite inputs in the normal range
 * of bfloat16; zero stays zero.  x = m 2^e with m in [0.5, 1): m 2^8 is rounded to
 * an integer in [128, 256] (nearbyint rounds ties to even in the default mode). */
static double or_bf16(double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    double m = frexp(x, &e);
    return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

double or_bf16_round(double x) { return or_bf16(x); }

int or_bf16_round_n(const double *x, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = or_bf16(x[i]);
    return 0;
}

/* Forward pass of one ray; h1, h2: post-ReLU activations, q: softmax output.
 * bf != 0: every operand of the three affine maps -- inputs, weights, biases and
 * the post-ReLU activations fed to the next layer -- is first rounded to bfloat16;
 * products and sums stay in double (the operand rounding of a BF16 tensor-core
 * evaluation of the same network, with exact accumulation). */
static void or_prop_forward(const double *P, const double *in, double *h1, double *h2, double *z, double *q, int bf)
{
    const double *W1 = P, *b1 = W1 + OR_PH * OR_PIN, *W2 = b1 + OR_PH, *b2 = W2 + OR_PH * OR_PH;
    const double *W3 = b2 + OR_PH, *b3 = W3 + OR_PO * OR_PH;
#define OR_OP(v) (bf ? or_bf16(v) : (v))
    for (int o = 0; o < OR_PH; o++) {
        double acc = 0.0;
        for (int i = 0; i < OR_PIN; i++) acc += OR_OP(W1[o * OR_PIN + i]) * OR_OP(in[i]);
        acc += OR_OP(b1[o]);
        h1[o] = acc > 0.0 ? acc : 0.0;
    }
    for (int o = 0; o < OR_PH; o++) {
        double acc = 0.0;
        for (int i = 0; i < OR_PH; i++) acc += OR_OP(W2[o * OR_PH + i]) * OR_OP(h1[i]);
        acc += OR_OP(b2[o]);
        h2[o] = acc > 0.0 ? acc : 0.0;
    }
    double m = -INFINITY;
    for (int o = 0; o < OR_PO; o++) {
        double acc = 0.0;
        for (int i = 0; i < OR_PH; i++) acc += OR_OP(W3[o * OR_PH + i]) * OR_OP(h2[i]);
        z[o] = acc + OR_OP(b3[o]);
        if (z[o] > m) m = z[o];
    }
#undef OR_OP
    double s = 0.0;
    for (int o = 0; o < OR_PO; o++) { q[o] = exp(z[o] - m); s += q[o]; }
    for (int o = 0; o < OR_PO; o++) q[o] /= s;
}

/* Softmax outputs of n rays (q: n x 65).  t0: root entry per ray.  bf != 0: the
 * operands rounded to bfloat16 (see or_prop_forward). */
int or_prop_predict(const double *P, const float *o, const float *d, const double *t0, int64_t n, double *q, int bf)
{
    double in[OR_PIN], h1[OR_PH], h2[OR_PH], z[OR_PO];
    for (int64_t r = 0; r < n; r++) {
        or_prop_input(o + 3 * r, d + 3 * r, t0[r], in);
        or_prop_forward(P, in, h1, h2, z, q + r * OR_PO, bf);
    }
    return 0;
}

/* Mean cross-entropy of n rays against targets p (n x 65) and its exact gradient
 * (backpropagation through softmax, the two ReLU layers and the affine maps). */
int or_prop_loss_grad(const double *P, const float *o, const float *d, const double *t0, const double *p,
                      int64_t n, double *loss, double *grad)
{
    const double *W2 = P + OR_PH * OR_PIN + OR_PH, *W3 = W2 + OR_PH * OR_PH + OR_PH;
    double *gW1 = grad, *gb1 = gW1 + OR_PH * OR_PIN, *gW2 = gb1 + OR_PH, *gb2 = gW2 + OR_PH * OR_PH;
    double *gW3 = gb2 + OR_PH, *gb3 = gW3 + OR_PO * OR_PH;
    double in[OR_PIN], h1[OR_PH], h2[OR_PH], z[OR_PO], q[OR_PO], dz[OR_PO], dh2[OR_PH], dh1[OR_PH];
    for (int i = 0; i < OR_PNPAR; i++) grad[i] = 0.0;
    double L = 0.0;
    for (int64_t r = 0; r < n; r++) {
        const double *pr = p + r * OR_PO;
        or_prop_input(o + 3 * r, d + 3 * r, t0[r], in);
        or_prop_forward(P, in, h1, h2, z, q, 0);
        double ps = 0.0;
        for (int b = 0; b < OR_PO; b++) {
            if (pr[b] > 0.0) L -= pr[b] * log(q[b]);
            ps += pr[b];
        }
        /* d/dz_b of -sum_c p_c log softmax(z)_c = q_b sum_c p_c - p_b */
        for (int b = 0; b < OR_PO; b++) dz[b] = q[b] * ps - pr[b];
        for (int b = 0; b < OR_PO; b++) {
            gb3[b] += dz[b] / (double)n;
            for (int i = 0; i < OR_PH; i++) gW3[b * OR_PH + i] += dz[b] * h2[i] / (double)n;
        }
        for (int i = 0; i < OR_PH; i++) {
            double acc = 0.0;
            for (int b = 0; b < OR_PO; b++) acc += W3[b * OR_PH + i] * dz[b];
            dh2[i] = h2[i] > 0.0 ? acc : 0.0;
        }
        for (int o2 = 0; o2 < OR_PH; o2++) {
            gb2[o2] += dh2[o2] / (double)n;
            for (int i = 0; i < OR_PH; i++) gW2[o2 * OR_PH + i] += dh2[o2] * h1[i] / (double)n;
        }
        for (int i = 0; i < OR_PH; i++) {
            double acc = 0.0;
            for (int o2 = 0; o2 < OR_PH; o2++) acc += W2[o2 * OR_PH + i] * dh2[o2];
            dh1[i] = h1[i] > 0.0 ? acc : 0.0;
        }
        for (int o1 = 0; o1 < OR_PH; o1++) {
            gb1[o1] += dh1[o1] / (double)n;
            for (int i = 0; i < OR_PIN; i++) gW1[o1 * OR_PIN + i] += dh1[o1] * in[i] / (double)n;
        }
    }
    *loss = L / (double)n;
    return 0;
}

/* One Adam step (Kingma and Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * P -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps); t counts from 1. */
int or_prop_adam(double *P, const double *g, double *m, double *v, int n_par, int t, double lr, double b1, double b2,
                 double eps)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int i = 0; i < n_par; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        P[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
    return 0;
}

/* Kept depth bins of one ray: bins are visited by decreasing predicted mass (ties
 * to the lower index); their mass is added until it reaches `coverage`; the
 * background bin counts toward coverage but is not a depth bin.  When more than
 * max_bins depth bins would be needed the ray falls back to the plain sampler.
 * single != 0: the running sum is kept in binary32 (each partial sum rounded to
 * float, compared with the float coverage), the precision in which the GPU
 * kernels take this decision; q must then hold float values. */
int or_prop_select(const double *q, int64_t n, double coverage, int max_bins, uint64_t *mask, int *fallback,
                   int single)
{
    const double cov = single ? (double)(float)coverage : coverage;
    for (int64_t r = 0; r < n; r++) {
        const double *qr = q + r * OR_PO;
        int used[OR_PO] = {0};
        double cum = 0.0;
        int kept = 0;
        uint64_t mk = 0;
        int fb = 0;
        while (cum < cov) {
            int best = -1;
            for (int b = 0; b < OR_PO; b++)
                if (!used[b] && (best < 0 || qr[b] > qr[best])) best = b;
            if (best < 0) break;
            used[best] = 1;
            cum += qr[best];
            if (single) cum = (double)(float)cum;   /* a float sum of two floats, rounded once */
            if (best < 64) {
                if (kept == max_bins) { fb = 1; break; }
                mk |= 1ull << best;
                kept++;
            }
        }
        mask[r] = fb ? ~0ull : mk;
        fallback[r] = fb;
    }
    return 0;
}
