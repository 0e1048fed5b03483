"""Pins of the CPU oracle to things other than itself.

Each test checks the oracle against what the paper and the mathematics fix:
hand-derived trees (Sec. 3.4), brute-force point-in-box classification along rays
(Algorithm 1), closed forms of the volume-rendering quadrature (Sec. 3.1), exact
values and identities of the frequency encoding, and a library matmul chain for the
MLP.  None of them calls the CUDA library.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2310_01881_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------------
# helpers (independent of the oracle's arithmetic)
# ----------------------------------------------------------------------------------

def _fixture_grid(case):
    G = case["G"]
    g = np.full((G, G, G), case["density"]["default"], np.float32)
    col = case["density"].get("x_column")
    if col:
        g[:, :, col["x"]] = col["value"]
    for x, y, z, v in case["density"]["cells"]:
        g[z, y, x] = v
    return g


@pytest.fixture(scope="module")
def c1_scene():
    cfg = S.CONFIGS["c1"]
    grid = S.density_grid(S.scene_for("c1", 0), cfg.G)
    tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    return cfg, grid, tree


@pytest.fixture(scope="module")
def mass_scene():
    """A c2-style scene on a small grid with a mass threshold (uneven leaves)."""
    grid = S.density_grid(S.scene_for("c2", 3), 32)
    tree = O.build_tree(grid, 6, 1.0 / 48.0)
    return grid, tree


def _leaf_boxes(tree):
    lv = tree.leaves()
    return tree.box[lv].astype(np.float64)


def _classify(points, boxes, eps):
    """Leaf index of each point when it lies inside exactly one box by more than eps
    from every face of that box; -1 when outside all boxes, -2 when ambiguous."""
    lo = boxes[None, :, :3]
    hi = boxes[None, :, 3:]
    p = points[:, None, :]
    inside = np.all((p > lo + eps) & (p < hi - eps), axis=2)
    near = np.all((p >= lo - eps) & (p <= hi + eps), axis=2)
    out = np.full(len(points), -1, np.int64)
    one = inside.sum(1) == 1
    out[one] = np.argmax(inside[one], axis=1)
    amb = (~one) & (near.sum(1) > 0)
    out[amb] = -2
    return out


def _camera_rays(n, seed, radius=3.0, spread=0.9):
    rng = np.random.default_rng(seed)
    u = rng.normal(size=(n, 3)); u /= np.linalg.norm(u, axis=1, keepdims=True)
    o = radius * u
    tgt = rng.uniform(-spread, spread, size=(n, 3))
    d = tgt - o; d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


# ----------------------------------------------------------------------------------
# tree (Sec. 3.4)
# ----------------------------------------------------------------------------------

def test_tree_matches_hand_derived_fixtures():
    with open(os.path.join(GOLDEN, "tree_g4.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        t = O.build_tree(_fixture_grid(case), case["max_depth"], case["leaf_frac"])
        exp = case["nodes"]
        assert t.n_nodes == len(exp), case["name"]
        for i, e in enumerate(exp):
            np.testing.assert_array_equal(t.box[i], np.asarray(e["box"], np.float32), err_msg=case["name"])
            assert t.info[i, 0] == e["axis"], (case["name"], i)
            assert t.info[i, 3] == e["leaf"], (case["name"], i)
            assert t.info[i, 4] == e["code"], (case["name"], i)
            assert t.info[i, 5] == e["depth"], (case["name"], i)
            assert t.mass[i] == e["mass"], (case["name"], i)
            if e["axis"] >= 0:
                assert t.split[i] == np.float32(e["split"]), (case["name"], i)


@pytest.mark.parametrize("which", ["c1", "mass"])
def test_tree_leaves_tile_the_root(which, c1_scene, mass_scene):
    grid, tree = (c1_scene[1], c1_scene[2]) if which == "c1" else mass_scene
    G = grid.shape[0]
    cover = np.zeros((G, G, G), np.int32)
    vol = 0.0
    for x0, y0, z0, x1, y1, z1 in tree.leaf_cells():
        cover[z0:z1, y0:y1, x0:x1] += 1
    for b in _leaf_boxes(tree):
        vol += np.prod(b[3:] - b[:3])
    assert np.all(cover == 1)
    assert vol == pytest.approx(8.0, abs=1e-12)
    # children partition their parent exactly
    for i in range(tree.n_nodes):
        a, l, r = tree.info[i, 0], tree.info[i, 1], tree.info[i, 2]
        if a < 0:
            continue
        assert tree.box[l, 3 + a] == tree.split[i] == tree.box[r, a]
        assert tree.box[l, a] == tree.box[i, a] and tree.box[r, 3 + a] == tree.box[i, 3 + a]


@pytest.mark.parametrize("which", ["c1", "mass"])
def test_tree_split_is_density_median_by_brute_force(which, c1_scene, mass_scene):
    grid, tree = (c1_scene[1], c1_scene[2]) if which == "c1" else mass_scene
    g64 = grid.astype(np.float64)
    total = g64.sum()
    for i in range(tree.n_nodes):
        x0, y0, z0, x1, y1, z1 = tree.cells[i]
        blk = g64[z0:z1, y0:y1, x0:x1]
        ext = [x1 - x0, y1 - y0, z1 - z0]
        a = int(np.argmax(ext))                          # longest, ties to lowest index
        m = blk.sum()
        assert tree.mass[i] == pytest.approx(m, rel=1e-12, abs=1e-12)
        if tree.info[i, 0] < 0:
            # leaf rule: depth limit, mass threshold or one cell wide
            assert (tree.info[i, 5] == (4 if which == "c1" else 6)) or max(ext) <= 1 or \
                (which == "mass" and m <= total / 48.0 * (1 + 1e-12))
            continue
        assert tree.info[i, 0] == a
        assert which == "c1" or m > total / 48.0 * (1 - 1e-12)
        slices = blk.sum(axis=tuple(ax for ax in (0, 1, 2) if ax != 2 - a))
        n = ext[a]
        pre = np.cumsum(slices)[:-1]                     # prefix(k) for k = 1..n-1
        if m == 0:
            k_exp = n // 2
        else:
            if np.any(np.abs(pre - 0.5 * m) <= 1e-9 * m):
                continue                                 # rounding-order tie: both answers valid
            hit = np.nonzero(pre >= 0.5 * m)[0]
            k_exp = int(hit[0]) + 1 if len(hit) else n - 1
        lo = (x0, y0, z0)[a]
        k_got = round((float(tree.split[i]) + 1.0) / 2.0 * grid.shape[0]) - lo
        assert k_got == k_exp, (i, a, k_got, k_exp)


# ----------------------------------------------------------------------------------
# traversal (Algorithm 1) and sampling
# ----------------------------------------------------------------------------------

def _check_against_point_classification(tree, o, d, nx, leaf, tin, tout, dt=1e-3, eps=1e-9):
    boxes = _leaf_boxes(tree)
    for r in range(len(o)):
        ts = np.arange(dt / 2, 8.0, dt)
        pts = o[r].astype(np.float64)[None] + ts[:, None] * d[r].astype(np.float64)[None]
        cls = _classify(pts, boxes, eps)
        # every point strictly inside a reported crossing is in that leaf
        for k in range(nx[r]):
            sel = (ts > tin[r, k] + 4 * dt) & (ts < tout[r, k] - 4 * dt)
            got = cls[sel]
            assert np.all((got == leaf[r, k]) | (got == -2)), (r, k)
        # every run of points in some leaf longer than a few steps is a reported crossing
        seq = [c for c in cls if c >= 0]
        runs = []
        for c in seq:
            if not runs or runs[-1][0] != c:
                runs.append([c, 1])
            else:
                runs[-1][1] += 1
        long_runs = [c for c, m in runs if m > 8]
        rep = list(leaf[r, :nx[r]])
        it = iter(rep)
        assert all(c in it for c in long_runs), (r, long_runs, rep)     # ordered subsequence
        # nothing outside the root box is reported
        inroot = np.all((pts >= -1 - 1e-9) & (pts <= 1 + 1e-9), axis=1)
        if nx[r]:
            assert np.all(inroot[(ts > tin[r, 0] + dt) & (ts < tout[r, nx[r] - 1] - dt)])
        else:
            assert inroot.sum() <= 2


@pytest.mark.parametrize("mode", [0, 1])
def test_traversal_matches_point_classification(mode, c1_scene, mass_scene):
    for tree in (c1_scene[2], mass_scene[1]):
        o, d = _camera_rays(60, 11)
        o2 = np.random.default_rng(5).uniform(-0.9, 0.9, (20, 3)).astype(np.float32)   # origins inside
        d2 = _camera_rays(20, 12)[1]
        o = np.concatenate([o, o2]); d = np.concatenate([d, d2])
        nx, leaf, tin, tout = O.traverse(tree, o, d, 64, mode=mode)
        _check_against_point_classification(tree, o, d, nx, leaf, tin, tout)


@pytest.mark.parametrize("mode", [0, 1])
def test_stack_traversal_equals_sorted_all_leaves(mode, c1_scene, mass_scene):
    for tree in (c1_scene[2], mass_scene[1]):
        o, d = _camera_rays(400, 21)
        a = O.traverse(tree, o, d, 64, mode=mode, method=0)
        b = O.traverse(tree, o, d, 64, mode=mode, method=1)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_crossings_are_contiguous_and_cover_root(c1_scene):
    tree = c1_scene[2]
    o, d = _camera_rays(300, 31)
    nx, leaf, tin, tout = O.traverse(tree, o, d, 64, mode=0)
    for r in range(len(o)):
        if nx[r] == 0:
            continue
        # consecutive crossings share their boundary (same plane, same arithmetic)
        for k in range(nx[r] - 1):
            assert tout[r, k] == pytest.approx(tin[r, k + 1], abs=1e-12)
        # union = root interval, which for a ray starting outside is where |o + t d|_inf <= 1
        t0, t1 = tin[r, 0], tout[r, nx[r] - 1]
        for t, inside in ((t0 + 1e-7, True), (t1 - 1e-7, True), (t0 - 1e-6, False), (t1 + 1e-6, False)):
            p = o[r].astype(np.float64) + t * d[r].astype(np.float64)
            assert (np.max(np.abs(p)) <= 1.0) == inside


def test_fp32_mode_agrees_with_fp64_on_leaf_sequences(c1_scene):
    tree = c1_scene[2]
    o, d = _camera_rays(2000, 41)
    a = O.traverse(tree, o, d, 64, mode=0)
    b = O.traverse(tree, o, d, 64, mode=1)
    same = np.all(a[1] == b[1], axis=1) & (a[0] == b[0])
    assert same.mean() > 0.995
    ok = same[:, None] & (np.arange(64)[None] < a[0][:, None])
    assert np.max(np.abs(a[2] - b[2])[ok]) < 1e-5


def test_adversarial_rays_documented_behaviour():
    with open(os.path.join(GOLDEN, "tree_g4.json")) as f:
        case = json.load(f)["cases"][0]
    tree = O.build_tree(_fixture_grid(case), case["max_depth"], case["leaf_frac"])
    f32 = np.float32
    rays = [
        # axis-parallel along +x at y=-0.5, z=0.3: leaves 0 (x<0.5) then 2 (x>0.5), split at t=3.5
        ((-3, -0.5, 0.3), (1, 0, 0), [0, 2], [(2.0, 3.5), (3.5, 4.0)]),
        # axis-parallel along -y at x=0.75: leaves 3 then 2 (split y=0 at t=3)
        ((0.75, 3, 0.1), (0, -1, 0), [3, 2], [(2.0, 3.0), (3.0, 4.0)]),
        # ray lying in the split plane x=0.5 (d_x = 0): NaN slab terms, no child is entered
        ((0.5, -3, 0.2), (0, 1, 0), [], []),
        # grazing the root's edge y=1, z=1 along x: zero-length slab -> nothing
        ((-3, 1, 1), (1, 0, 0), [], []),
        # miss
        ((-3, 2, 0), (1, 0, 0), [], []),
        # origin inside leaf 1, heading +y: one crossing from t=0
        ((0, 0.5, 0), (0, 1, 0), [1], [(0.0, 0.5)]),
    ]
    o = np.array([r[0] for r in rays], f32); d = np.array([r[1] for r in rays], f32)
    for mode in (0, 1):
        nx, leaf, tin, tout = O.traverse(tree, o, d, 8, mode=mode)
        for i, (_, _, lv, iv) in enumerate(rays):
            assert list(leaf[i, :nx[i]]) == lv, (mode, i)
            for k, (a, b) in enumerate(iv):
                assert tin[i, k] == a and tout[i, k] == b, (mode, i, k)


def test_cap_truncates_whole_crossings(c1_scene):
    tree = c1_scene[2]
    o, d = _camera_rays(200, 51)
    full = O.traverse(tree, o, d, 64, mode=1)
    cut = O.traverse(tree, o, d, 2, mode=1)
    assert np.all(cut[0] == np.minimum(full[0], 2))
    np.testing.assert_array_equal(cut[1], full[1][:, :2] * (np.arange(2)[None] < cut[0][:, None]) +
                                  -1 * (np.arange(2)[None] >= cut[0][:, None]))


@pytest.mark.parametrize("mode", [0, 1])
def test_samples_lie_in_their_leaf_and_fill_the_hit(mode, c1_scene):
    cfg, _, tree = c1_scene
    o, d = _camera_rays(300, 61)
    maxc = cfg.cap // cfg.steps
    nx, leaf, tin, tout = O.traverse(tree, o, d, maxc, mode=mode)
    t, dl, x = O.samples(o, d, nx, tin, tout, maxc, cfg.steps, cfg.cap, mode=mode)
    boxes = _leaf_boxes(tree)
    tol = 1e-12 if mode == 0 else 4e-7
    for r in range(len(o)):
        n = nx[r] * cfg.steps
        assert n <= cfg.cap
        lv = np.repeat(leaf[r, :nx[r]], cfg.steps)
        b = boxes[lv]
        assert np.all(x[r, :n] >= b[:, :3] - tol) and np.all(x[r, :n] <= b[:, 3:] + tol)
        assert np.all(np.diff(t[r, :n]) > 0)
        # the strata tile each crossing: sum of deltas = sum of crossing lengths
        assert dl[r, :n].sum() == pytest.approx(float((tout[r, :nx[r]] - tin[r, :nx[r]]).sum()), rel=1e-6)


def test_splitmix64_finaliser_matches_published_sequence():
    """splitmix64 (Steele, Lea and Flood, 2014) from state 0 -- the state advanced by the
    golden gamma 0x9e3779b97f4a7c15 before each finalisation -- starts with these
    outputs in its reference implementation."""
    gamma = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [O.splitmix64_mix((k * gamma) & ((1 << 64) - 1)) for k in (1, 2, 3)]
    assert got == want


@pytest.mark.parametrize("mode", [0, 1])
def test_jittered_samples_stay_in_their_strata_and_are_uniform(mode, c1_scene):
    """Sec. 3.5 random placement: one sample per stratum, uniform within it."""
    cfg, _, tree = c1_scene
    o, d = _camera_rays(800, 67)
    maxc = cfg.cap // cfg.steps
    nx, leaf, tin, tout = O.traverse(tree, o, d, maxc, mode=mode)
    t, dl, x = O.samples(o, d, nx, tin, tout, maxc, cfg.steps, cfg.cap, mode=mode, jitter=12345)
    tm, dlm, _ = O.samples(o, d, nx, tin, tout, maxc, cfg.steps, cfg.cap, mode=mode, jitter=0)
    us = []
    for r in range(len(o)):
        n = nx[r] * cfg.steps
        e = np.repeat(tin[r, :nx[r]], cfg.steps)
        j = np.tile(np.arange(cfg.steps), nx[r])
        np.testing.assert_array_equal(dl[r, :n], dlm[r, :n])          # the strata are unchanged
        u = (t[r, :n] - e) / dl[r, :n] - j
        # FP32: t is rounded to its ulp, which is a larger fraction of short strata
        tol = 1e-9 if mode == 0 else 4.0 * 2.0 ** -24 * np.maximum(np.abs(t[r, :n]), np.abs(e)) / dl[r, :n] + 1e-6
        assert np.all(u >= -tol) and np.all(u < 1 + tol)
        # midpoints for seed 0
        assert np.all(np.abs((tm[r, :n] - e) / dlm[r, :n] - j - 0.5) <= tol)
        us.append(u)
    u = np.concatenate(us)
    assert len(u) > 20000
    assert abs(u.mean() - 0.5) < 0.01
    # Kolmogorov-Smirnov distance to U[0, 1)
    s = np.sort(np.clip(u, 0.0, 1.0))
    ks = np.max(np.abs(s - (np.arange(len(s)) + 0.5) / len(s)))
    assert ks < 1.6 / np.sqrt(len(s))


def test_jitter_is_keyed_by_the_ray_not_its_batch_position(c1_scene):
    cfg, _, tree = c1_scene
    o, d = _camera_rays(64, 71)
    maxc = cfg.cap // cfg.steps
    nx, leaf, tin, tout = O.traverse(tree, o, d, maxc, mode=1)
    t, _, _ = O.samples(o, d, nx, tin, tout, maxc, cfg.steps, cfg.cap, mode=1, jitter=99)
    p = np.arange(len(o))[::-1]
    tr, _, _ = O.samples(o[p], d[p], nx[p], tin[p], tout[p], maxc, cfg.steps, cfg.cap, mode=1, jitter=99)
    np.testing.assert_array_equal(tr, t[p])
    # different seeds move the samples
    t2, _, _ = O.samples(o, d, nx, tin, tout, maxc, cfg.steps, cfg.cap, mode=1, jitter=100)
    gen = np.arange(cfg.cap)[None, :] < (nx * cfg.steps)[:, None]
    assert np.mean(t2[gen] != t[gen]) > 0.99
    assert O.jitter_fraction(99, o[3], d[3], 0, cfg.steps, 0) == pytest.approx(
        float((t[3, 0] - tin[3, 0]) / ((tout[3, 0] - tin[3, 0]) / cfg.steps)), abs=2e-5)


# ----------------------------------------------------------------------------------
# empty-space skipping over the guidance grid (Sec. 4.1: the density grid marks empty regions)
# ----------------------------------------------------------------------------------

def _brute_skip(tree, grid, thr, o, d, maxc, steps, jitter):
    """Kept crossings by brute force: the full crossing list (FP64), then, in order,
    those with a sample (placed as the crossing's index among the kept ones) in a cell
    of density > thr; the cell of p is floor((p + 1) G / 2) clamped, over [-1, 1]^3."""
    G = grid.shape[0]
    nx, leaf, tin, tout = O.traverse(tree, o, d, 256, mode=0)
    out = []
    for r in range(len(o)):
        kept = []
        for i in range(nx[r]):
            if len(kept) == maxc:
                break
            k = len(kept)
            dl = (tout[r, i] - tin[r, i]) / steps
            occ = False
            for j in range(steps):
                u = O.jitter_fraction(jitter, o[r], d[r], k, steps, j)
                t = tin[r, i] + (j + u) * dl
                p = o[r].astype(np.float64) + t * d[r].astype(np.float64)
                c = np.clip(np.floor((p + 1.0) * (G / 2)), 0, G - 1).astype(int)
                occ = occ or grid[c[2], c[1], c[0]] > thr
            if occ:
                kept.append(leaf[r, i])
        out.append(kept)
    return out


@pytest.mark.parametrize("jitter", [0, 21])
def test_skipping_keeps_exactly_the_occupied_crossings(jitter, mass_scene):
    grid, tree = mass_scene
    thr = float(np.quantile(grid, 0.6))          # about 60 % of the cells empty
    o, d = _camera_rays(150, 83)
    maxc, steps = 12, 8
    nx, leaf, tin, tout = O.traverse(tree, o, d, maxc, mode=0, skip=(grid, thr, steps, jitter))
    want = _brute_skip(tree, grid, thr, o, d, maxc, steps, jitter)
    full, *_ = O.traverse(tree, o, d, maxc, mode=0)
    assert sum(len(w) for w in want) < full.sum()   # the threshold does skip crossings
    for r in range(len(o)):
        assert list(leaf[r, :nx[r]]) == want[r]


def test_skipping_below_every_density_is_the_plain_render(c1_scene):
    cfg, grid, tree = c1_scene
    P = S.xavier_weights(0, S.leaf_mean_density(grid, tree.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    o, d = _camera_rays(200, 89)
    for mode in (0, 1):
        a = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=mode)
        b = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=mode,
                     skip=(grid, -1.0))
        for key in ("rgb", "depth", "opacity", "n_gen"):
            np.testing.assert_array_equal(a[key], b[key])


def test_skipping_above_every_density_leaves_the_background(c1_scene):
    cfg, grid, tree = c1_scene
    P = S.xavier_weights(0, S.leaf_mean_density(grid, tree.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    o, d = _camera_rays(50, 97)
    bg = (0.25, 0.5, 0.75)
    res = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, bg=bg, mode=0,
                   skip=(grid, float(grid.max()) + 1.0))
    assert np.all(res["n_gen"] == 0)
    np.testing.assert_array_equal(res["rgb"], np.tile(bg, (len(o), 1)))
    np.testing.assert_array_equal(res["opacity"], 0.0)


# ----------------------------------------------------------------------------------
# grouping (Sec. 3.5)
# ----------------------------------------------------------------------------------

def test_group_is_a_stable_counting_sort():
    rng = np.random.default_rng(7)
    n, maxc, L, steps = 500, 6, 13, 8
    nx = rng.integers(0, maxc + 1, n).astype(np.int32)
    leaf = np.full((n, maxc), -1, np.int32)
    for r in range(n):
        leaf[r, :nx[r]] = rng.integers(0, L, nx[r])
    counts, offsets, order = O.group(nx, leaf, maxc, steps, L)
    valid = np.concatenate([r * maxc + np.arange(nx[r]) for r in range(n)])
    flat = leaf.reshape(-1)
    np.testing.assert_array_equal(counts, np.bincount(flat[valid], minlength=L) * steps)
    np.testing.assert_array_equal(offsets, np.concatenate([[0], np.cumsum(counts)]))
    np.testing.assert_array_equal(np.sort(order), valid)                  # a permutation
    for l in range(L):
        seg = order[offsets[l] // steps: offsets[l + 1] // steps]
        assert np.all(flat[seg] == l) and np.all(np.diff(seg) > 0)        # grouped, stable


# ----------------------------------------------------------------------------------
# encoding and MLP
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [0, 1])
def test_encoding_exact_values_at_dyadic_points(mode):
    L = 10
    e = O.encode([0.0, 0.5, -0.25], L, mode)
    assert e.shape == (63,)
    np.testing.assert_array_equal(e[:3], [0.0, 0.5, -0.25])
    h = math.sqrt(0.5)
    for k in range(L):
        s, c = e[3 + 6 * k: 6 + 6 * k], e[6 + 6 * k: 9 + 6 * k]
        exp_s = [0.0, 1.0 if k == 0 else 0.0, [-h, -1.0, 0.0][k] if k < 3 else 0.0]
        exp_c = [1.0, [0.0, -1.0][k] if k < 2 else 1.0, [h, 0.0, -1.0][k] if k < 3 else 1.0]
        np.testing.assert_allclose(s, exp_s, atol=1e-7 if mode else 1e-15)
        np.testing.assert_allclose(c, exp_c, atol=1e-7 if mode else 1e-15)


def test_encoding_double_angle_chain():
    rng = np.random.default_rng(3)
    for p in rng.uniform(-1, 1, (50, 3)):
        e = O.encode(p, 10, 0)
        s = e[3:].reshape(10, 2, 3)[:, 0]
        c = e[3:].reshape(10, 2, 3)[:, 1]
        np.testing.assert_allclose(s * s + c * c, 1.0, atol=1e-14)
        np.testing.assert_allclose(s[1:], 2 * s[:-1] * c[:-1], atol=1e-12)
        np.testing.assert_allclose(c[1:], c[:-1] ** 2 - s[:-1] ** 2, atol=1e-12)
        np.testing.assert_allclose(s[0], np.sin(np.pi * p), atol=1e-14)
        # FP32 mode at the same float point: within one rounding of the float64 values
        pf = p.astype(np.float32).astype(np.float64)
        np.testing.assert_allclose(O.encode(pf, 10, 1), O.encode(pf, 10, 0), rtol=0, atol=6e-8)


def _numpy_mlp(P, width, hidden, feats):
    k0 = feats.shape[1]
    ofs, h = 0, feats
    kin = k0
    for _ in range(hidden):
        W = P[ofs: ofs + width * kin].astype(np.float64).reshape(width, kin); ofs += width * kin
        b = P[ofs: ofs + width].astype(np.float64); ofs += width
        h = np.maximum(h @ W.T + b, 0.0)
        kin = width
    W = P[ofs: ofs + 4 * width].astype(np.float64).reshape(4, width); ofs += 4 * width
    b = P[ofs: ofs + 4].astype(np.float64)
    return h @ W.T + b


def test_mlp_matches_library_matmul_chain():
    width, hidden, lx, ld = 64, 4, 10, 4
    rng = np.random.default_rng(9)
    P = S.xavier_weights(1, np.array([3.0]), width, hidden, lx, ld)
    P = P + rng.normal(0, 0.05, P.shape).astype(np.float32)    # nonzero biases too
    x = rng.uniform(-1, 1, (64, 3)); d = rng.normal(size=(64, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    out, raw = O.mlp_eval(P, width, hidden, lx, ld, x, d, mode=0)
    feats = np.stack([np.concatenate([O.encode(a, lx), O.encode(b, ld)]) for a, b in zip(x, d)])
    z = _numpy_mlp(P, width, hidden, feats)
    np.testing.assert_allclose(raw, z, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out[:, 0], np.logaddexp(0.0, z[:, 0]), rtol=1e-12)
    np.testing.assert_allclose(out[:, 1:], 1 / (1 + np.exp(-z[:, 1:])), rtol=1e-12)
    out32, raw32 = O.mlp_eval(P, width, hidden, lx, ld, x, d, mode=1)
    np.testing.assert_allclose(out32, out, atol=2e-4)


def test_mlp_input_absmax_matches_matmul_chain():
    """Per-layer input ranges (the E4M3 static scales' calibration) against the same
    numpy float64 chain: layer 0 is the encoding, layer l the ReLU output of l - 1."""
    width, hidden, lx, ld = 64, 4, 10, 4
    rng = np.random.default_rng(11)
    P = S.xavier_weights(2, np.array([3.0]), width, hidden, lx, ld)
    P = P + rng.normal(0, 0.05, P.shape).astype(np.float32)
    x = rng.uniform(-1, 1, (48, 3)); d = rng.normal(size=(48, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = O.mlp_input_absmax(P, width, hidden, lx, ld, x, d)
    feats = np.stack([np.concatenate([O.encode(a, lx), O.encode(b, ld)]) for a, b in zip(x, d)])
    k0 = feats.shape[1]
    want, h, ofs, kin = [], feats, 0, k0
    for _ in range(hidden):
        want.append(np.abs(h).max())
        W = P[ofs: ofs + width * kin].astype(np.float64).reshape(width, kin); ofs += width * kin
        b = P[ofs: ofs + width].astype(np.float64); ofs += width
        h = np.maximum(h @ W.T + b, 0.0)
        kin = width
    np.testing.assert_allclose(got, want, rtol=1e-12)
    assert 0.999 <= got[0] <= max(1.0, np.abs(x).max(), np.abs(d).max())   # sin/cos of many octaves near 1


def test_mlp_one_hot_routing_closed_form():
    """W0 routes input feature f to hidden unit 0, identities pass it on, the head
    copies it: a transposed operand or a wrong offset breaks the equalities."""
    width, hidden, lx, ld = 32, 3, 10, 4
    k0 = S.mlp_input_width(lx, ld)
    per = S.params_per_leaf(width, hidden, lx, ld)
    P = np.zeros(per, np.float32)
    f = 37
    P[0 * k0 + f] = 1.0                                   # W0[0, f]
    ofs = width * k0 + width
    for _ in range(hidden - 1):
        P[ofs: ofs + width * width] = np.eye(width, dtype=np.float32).ravel(); ofs += width * width + width
    P[ofs + 0 * width + 0] = 1.0                          # Wo[0, 0]
    P[ofs + 2 * width + 0] = -2.0                         # Wo[2, 0]
    P[ofs + 4 * width + 0: ofs + 4 * width + 4] = [0.25, 0.5, -1.0, 0.0]
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (40, 3)); d = rng.normal(size=(40, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    out, raw = O.mlp_eval(P, width, hidden, lx, ld, x, d)
    g = np.array([O.encode(a, lx)[f] for a in x])
    r = np.maximum(g, 0.0)
    np.testing.assert_allclose(raw[:, 0], r + 0.25, atol=1e-15)
    np.testing.assert_allclose(raw[:, 1], 0.5, atol=1e-15)
    np.testing.assert_allclose(raw[:, 2], -2 * r - 1.0, atol=1e-15)
    np.testing.assert_allclose(out[:, 3], 0.5, atol=1e-15)


# ----------------------------------------------------------------------------------
# compositing (Sec. 3.1 quadrature)
# ----------------------------------------------------------------------------------

def _constant_params(n_leaves, width, hidden, lx, ld, sigma, rgb):
    per = S.params_per_leaf(width, hidden, lx, ld)
    P = np.zeros((n_leaves, per), np.float32)
    P[:, -4] = sigma if sigma > 30 else math.log(math.expm1(sigma))   # softplus^-1
    P[:, -3:] = [math.log(c / (1 - c)) for c in rgb]
    return P.reshape(-1)


@pytest.mark.parametrize("jitter", [0, 4242])
def test_constant_density_closed_form(jitter, c1_scene):
    """T = exp(-sigma L) for a constant density, with samples at midpoints or jittered
    inside their strata (the strata widths, hence the quadrature, are the same)."""
    cfg, _, tree = c1_scene
    sigma, rgb = 0.8, (0.2, 0.5, 0.7)
    P = _constant_params(tree.n_leaves, cfg.width, cfg.hidden, cfg.lx, cfg.ld, sigma, rgb)
    s_eff = float(np.logaddexp(0.0, np.float32(math.log(math.expm1(sigma)))))
    c_eff = [1 / (1 + math.exp(-float(np.float32(math.log(c / (1 - c)))))) for c in rgb]
    s3 = math.sqrt(3.0)
    o = np.array([[-3, 0.1, 0.2], [0.3, -3, -0.4], [-3, -3, -3], [-3, 5, 0]], np.float32)
    d = np.array([[1, 0, 0], [0, 1, 0], [1 / s3, 1 / s3, 1 / s3], [1, 0, 0]], np.float32)
    L = np.array([2.0, 2.0, 2 * s3, 0.0])
    bg = (0.1, 0.0, 0.3)
    res = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, 512, t_term=0.0,
                   bg=bg, mode=0, jitter=jitter)
    Tf = np.exp(-s_eff * L)
    np.testing.assert_allclose(res["opacity"], 1 - Tf, atol=2e-7)
    for c in range(3):
        np.testing.assert_allclose(res["rgb"][:, c], c_eff[c] * (1 - Tf) + bg[c] * Tf, atol=2e-7)
    assert res["depth"][3] == 0 and res["n_gen"][3] == 0


def test_depth_small_density_limit_is_midpoint_integral(c1_scene):
    """For sigma -> 0, depth / sigma -> sum_i delta_i t_i, and the midpoint rule is exact
    for the linear integrand: integral of t over the hit = (t1^2 - t0^2) / 2."""
    cfg, _, tree = c1_scene
    sigma = 1e-6
    P = _constant_params(tree.n_leaves, cfg.width, cfg.hidden, cfg.lx, cfg.ld, sigma, (0.5, 0.5, 0.5))
    s_eff = float(np.logaddexp(0.0, np.float32(math.log(math.expm1(sigma)))))
    o = np.array([[-3, 0.1, 0.2], [0.3, -3, -0.4], [0.1, 0.2, 4.0]], np.float32)
    d = np.array([[1, 0, 0], [0, 1, 0], [0, 0, -1]], np.float32)
    t0 = np.array([2.0, 2.0, 3.0]); t1 = np.array([4.0, 4.0, 5.0])
    res = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, 512, t_term=0.0, mode=0)
    np.testing.assert_allclose(res["depth"] / s_eff, (t1 ** 2 - t0 ** 2) / 2, rtol=1e-5)


def test_weights_and_residual_transmittance_sum_to_one(c1_scene):
    cfg, grid, tree = c1_scene
    rho = S.leaf_mean_density(grid, tree.leaf_cells())
    P = S.xavier_weights(0, rho, cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    o, d = S.view_rays(cfg, 0, 0, 24, 24)
    for mode, tol in ((0, 1e-12), (1, 2e-6)):
        res = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap,
                       mode=mode, full=True)
        np.testing.assert_allclose(res["slot_w"].sum(1) + res["t_final"], 1.0, atol=tol)
        np.testing.assert_allclose(res["opacity"], 1 - res["t_final"], atol=tol)


def test_early_termination_stops_after_opaque_sample(c1_scene):
    cfg, _, tree = c1_scene
    P = _constant_params(tree.n_leaves, cfg.width, cfg.hidden, cfg.lx, cfg.ld, 1e4, (0.5, 0.5, 0.5))
    o = np.array([[-3, 0.1, 0.2]], np.float32); d = np.array([[1, 0, 0]], np.float32)
    for mode in (0, 1):
        res = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=mode)
        assert res["n_eval"][0] == 1 and res["n_gen"][0] > 8
        assert res["opacity"][0] == pytest.approx(1.0, abs=1e-6)


def test_fp32_mode_render_close_to_fp64(c1_scene):
    cfg, grid, tree = c1_scene
    rho = S.leaf_mean_density(grid, tree.leaf_cells())
    P = S.xavier_weights(0, rho, cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    o, d = S.view_rays(cfg, 0, 0, 32, 32)
    a = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=4)
    b = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1, threads=4)
    ok = np.minimum(a["ert_margin"], b["ert_margin"]) > 1e-3
    assert np.max(np.abs(a["rgb"] - b["rgb"])[ok]) < 1e-4
    assert np.all(a["n_gen"] == b["n_gen"]) or np.mean(a["n_gen"] == b["n_gen"]) > 0.99


def test_binary16_rounding_hand_ties_and_library_conversion():
    """binary16 keeps 11 significant bits, ties to even, subnormal spacing 2^-24:
    1 + 2^-11 lies halfway between 1 and 1 + 2^-10 and goes to 1, 1 + 3 2^-11 goes to
    1 + 2^-9, 2^-25 (half the smallest subnormal) goes to 0 and 3 2^-25 to 2^-23.
    Random values agree with numpy's float16 conversion (a library routine)."""
    cases = [(1 + 2 ** -11, 1.0), (1 + 3 * 2 ** -11, 1 + 2 ** -9), (2.0 ** -25, 0.0), (3 * 2.0 ** -25, 2.0 ** -23),
             (65504.0, 65504.0), (-(1 + 2 ** -11), -1.0), (0.1, float(np.float16(0.1)))]
    got = O.f16_round(np.array([c[0] for c in cases]))
    np.testing.assert_array_equal(got, [c[1] for c in cases])
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, 50000) * 10.0 ** rng.uniform(-9, 4.8, 50000)
    np.testing.assert_array_equal(O.f16_round(x), x.astype(np.float16).astype(np.float64))


def test_half_precision_sample_store_costs_little_on_its_own(c1_scene):
    """The tensor-core paths store each sample's (sigma, r, g, b) as four binary16
    values between the network and the compositing.  The FP64 oracle with only that
    rounding (slot_fp16) against the plain FP64 oracle isolates its effect: on the c1
    view it is far below the BF16 path's total error against FP64 (about 75 dB on c1,
    79.6 dB on c2), i.e. a few per cent of its squared error."""
    cfg, grid, tree = c1_scene
    rho = S.leaf_mean_density(grid, tree.leaf_cells())
    P = S.xavier_weights(0, rho, cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    o, d = S.view_rays(cfg, 0, 0)
    a = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=4)
    b = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=4,
                 slot_fp16=True)
    mse = float(np.mean((a["rgb"] - b["rgb"]) ** 2))
    psnr = 10 * np.log10(1.0 / mse)
    err = np.abs(a["rgb"] - b["rgb"]).max()
    print(f"binary16 sample store alone, c1 view: PSNR {psnr:.2f} dB, max abs rgb {err:.2e}")
    assert psnr >= 88.0 and err <= 5e-4
    assert 0 < mse
