"""A CPU model of the traversal kernel's walk (Sec. 3.5, Algorithm 1 "Traverse")
checked against the oracle's FP32-mode crossings, bit for bit.

The kernel does not slab-test every box it visits: it slab-tests the root and carries
(entry, exit) down, cutting it at each inner node's split plane ts = (s - o_a) * inv_a
into (e, min(x, ts)) for the child the ray meets first (left for d_a >= +0, right for
d_a <= -0) and (max(e, ts), x) for the other, with no child when ts is NaN; only
children with exit > entry are entered or pushed.  As x > e, that is ts > e for the
first child and x > ts for the other (a NaN fails both), and a child crossed alone
keeps (e, x).  The claim that these are the
children's slab intervals, bit for bit, rests on face values being monotone in the
face coordinate.  This model replays the walk in float32 scalar arithmetic (numpy
scalars: correctly rounded, no fused multiply-add) and compares its crossings with the
oracle's set definition (every leaf with a positive slab crossing, sorted by entry) on
camera rays, rays starting on split planes with axis-parallel directions of both signs
(zero and negative-zero components: the NaN and infinite cases), and origins inside
the scene; with adaptive hierarchical sampling the HCheck runs on the carried entry.
The GPU tests compare the kernel itself with the oracle."""
import math

import numpy as np

import oracle as O
from paper_2310_01881_gb300 import scenes as S

F32 = np.float32


def _fmin(a, b):  # NaN-ignoring, as fminf
    if math.isnan(a):
        return b
    if math.isnan(b):
        return a
    return a if a < b else b


def _fmax(a, b):
    if math.isnan(a):
        return b
    if math.isnan(b):
        return a
    return a if a > b else b


def _walk(tree, o, d, maxc, lod=0.0, net=None):
    """The kernel's walk for one ray: list of (network, entry, exit)."""
    box, info, split = tree.box, tree.info, tree.split
    with np.errstate(all="ignore"):
        inv = [F32(F32(1) / d[a]) for a in range(3)]
        lo_t = [F32(F32(box[0][a] - o[a]) * inv[a]) for a in range(3)]
        hi_t = [F32(F32(box[0][3 + a] - o[a]) * inv[a]) for a in range(3)]
    e = _fmax(_fmax(_fmax(_fmin(lo_t[0], hi_t[0]), _fmin(lo_t[1], hi_t[1])), _fmin(lo_t[2], hi_t[2])), F32(0))
    x = _fmin(_fmin(_fmax(lo_t[0], hi_t[0]), _fmax(lo_t[1], hi_t[1])), _fmax(lo_t[2], hi_t[2]))
    out = []
    if not x > e:
        return out
    stack, nd = [], 0
    while True:
        ax = int(info[nd, 0])
        emit = ax < 0
        if not emit and lod > 0:
            emit = not (F32(box[nd][3 + ax] - box[nd][ax]) > F32(F32(lod) * e))
        if emit:
            out.append((int(info[nd, 3]) if ax < 0 else int(net[nd]), e, x))
            if len(out) >= maxc or not stack:
                break
            nd, e, x = stack.pop()
            continue
        with np.errstate(all="ignore"):
            ts = F32(F32(split[nd] - o[ax]) * inv[ax])
        ok1, ok2 = ts > e, x > ts          # (e, min(x, ts)) and (max(e, ts), x) non-empty
        left, right = int(info[nd, 1]), int(info[nd, 2])
        c1, c2 = (right, left) if math.copysign(1.0, inv[ax]) < 0 else (left, right)
        if ok1 and ok2:
            stack.append((c2, ts, x))
            nd, x = c1, ts
        elif ok1 or ok2:
            nd = c1 if ok1 else c2
        elif stack:
            nd, e, x = stack.pop()
        else:
            break
    return out


def _rays(tree, seed):
    cfg = S.CONFIGS["c1"]
    o, d = S.view_rays(cfg, seed, 0)
    idx = S.ray_subset(len(o), 240, seed)
    rng = np.random.default_rng(seed)
    po, pd = [], []
    for j in rng.choice(np.nonzero(tree.info[:, 0] >= 0)[0], 120):
        ax = tree.info[j, 0]
        p = rng.uniform(tree.box[j][:3], tree.box[j][3:]).astype(F32)
        p[ax] = tree.split[j]                      # the origin on the node's split plane
        q = np.zeros(3, F32)
        q[rng.integers(3)] = rng.choice([-1.0, 1.0])
        if rng.random() < 0.5:                     # a direction inside the plane
            q = rng.normal(size=3).astype(F32)
            q[ax] = 0.0
        if rng.random() < 0.3:
            q = -q                                 # negative zeros
        po.append(p)
        pd.append(q)
    io = rng.uniform(-0.9, 0.9, (60, 3)).astype(F32)
    idr = rng.normal(size=(60, 3))
    idr = (idr / np.linalg.norm(idr, axis=1, keepdims=True)).astype(F32)
    return (np.concatenate([o[idx], np.array(po, F32), io]), np.concatenate([d[idx], np.array(pd, F32), idr]))


def _check(tree, o, d, maxc, lod=0.0):
    nx, net, tin, tout = O.traverse(tree, o, d, maxc, mode=1, method=1, lod=lod)
    ids = None
    if lod > 0:  # network ids: leaves by leaf id, then the inner nodes in preorder
        ids = np.zeros(tree.n_nodes, np.int64)
        n_leaves, k = int((tree.info[:, 0] < 0).sum()), 0
        for i in range(tree.n_nodes):
            if tree.info[i, 0] < 0:
                ids[i] = tree.info[i, 3]
            else:
                ids[i] = n_leaves + k
                k += 1
    for r in range(len(o)):
        got = _walk(tree, [F32(v) for v in o[r]], [F32(v) for v in d[r]], maxc, lod, ids)
        assert len(got) == nx[r], r
        for k, (n, e, x) in enumerate(got):
            assert n == net[r, k] and e == F32(tin[r, k]) and x == F32(tout[r, k]), (r, k)


def test_split_plane_walk_reproduces_slab_crossings():
    cfg = S.CONFIGS["c1"]
    for seed in (0, 3):
        tree = O.build_tree(S.density_grid(S.scene_for(cfg.scene, seed), cfg.G), cfg.max_depth, cfg.leaf_mass_frac)
        o, d = _rays(tree, seed)
        _check(tree, o, d, cfg.cap // cfg.steps)


def test_split_plane_walk_with_hierarchical_sampling():
    cfg = S.CONFIGS["c1"]
    tree = O.build_tree(S.density_grid(S.scene_for(cfg.scene, 1), cfg.G), cfg.max_depth, cfg.leaf_mass_frac)
    o, d = _rays(tree, 1)
    for lod in (0.1, 0.5):
        _check(tree, o, d, cfg.cap // cfg.steps, lod)
