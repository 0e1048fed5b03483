"""Pins of the oracle's adaptive hierarchical sampling (Sec. 3.5, Algorithm 1's HCheck;
Fig. 1 (c); the ablation table's "w/o hierarchical sampling" row).

Reading: an inner node is descended only while its extent along its split axis
exceeds lod x the ray's entry distance into it; otherwise its own network takes the
whole crossing.  Networks: leaves 0 .. L-1 by leaf id, then the inner nodes in
preorder.  Pins: a hand-built two-level tree whose crossings are worked out by hand;
HCheck always true reproduces the leaf-only traversal and render bit for bit; the
stack traversal equals the set definition (brute force over every node and its
ancestors); the crossings still tile the root interval, every sample lies in its
node's box, coarsening never adds crossings, and the constant-density closed form
holds at any lod.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2310_01881_gb300 import scenes as S


def _two_level_tree():
    """Root [-1,1]^3 split at x = 0: left leaf A (leaf 0); right node [0,1] x [-1,1] x
    [-1,1] split at y = 0 into leaves B (y < 0, leaf 1) and C (y > 0, leaf 2).
    Networks: leaves 0, 1, 2; inner nodes in preorder: root 3, right node 4."""
    box = np.array([[-1, -1, -1, 1, 1, 1], [-1, -1, -1, 0, 1, 1], [0, -1, -1, 1, 1, 1],
                    [0, -1, -1, 1, 0, 1], [0, 0, -1, 1, 1, 1]], np.float32)
    info = np.array([[0, 1, 2, -1, 1, 0], [-1, -1, -1, 0, 2, 1], [1, 3, 4, -1, 3, 1],
                     [-1, -1, -1, 1, 6, 2], [-1, -1, -1, 2, 7, 2]], np.int32)
    split = np.array([0, 0, 0, 0, 0], np.float32)
    return O.make_tree(box, info, split)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("method", [0, 1])
def test_two_level_tree_by_hand(mode, method):
    """Ray from (-3, 0.5, 0.5) along +x: it enters the root at t = 2 (root extent 2 along
    x), the right node at t = 3 (extent 2 along y) and leaves at t = 4.
      lod 0.5: 2 > 1 and 2 > 1.5, both descend: leaf A [2, 3], leaf C [3, 4];
      lod 0.8: 2 > 1.6 descends, 2 > 2.4 does not: leaf A [2, 3], right node [3, 4];
      lod 1.5: 2 > 3 does not: the root alone [2, 4]."""
    tree = _two_level_tree()
    o = np.array([[-3, 0.5, 0.5]], np.float32)
    d = np.array([[1, 0, 0]], np.float32)
    want = {0.5: [(0, 2, 3), (2, 3, 4)], 0.8: [(0, 2, 3), (4, 3, 4)], 1.5: [(3, 2, 4)]}
    for lod, xs in want.items():
        nx, net, tin, tout = O.traverse(tree, o, d, 8, mode=mode, method=method, lod=lod)
        assert nx[0] == len(xs), lod
        for k, (n, a, b) in enumerate(xs):
            assert (net[0, k], tin[0, k], tout[0, k]) == (n, a, b), (lod, k)
    # lod = 0: the three leaves' rule (descend everywhere)
    nx, net, _, _ = O.traverse(tree, o, d, 8, mode=mode, method=method, lod=0.0)
    assert list(net[0, :nx[0]]) == [0, 2]


@pytest.fixture(scope="module")
def scenes():
    out = []
    for name in ("c1", "c2"):
        cfg = S.CONFIGS[name]
        G = cfg.G if name == "c1" else 64
        grid = S.density_grid(S.scene_for(cfg.scene, 0), G)
        tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
        o, d = S.view_rays(cfg, 0, 0, 40, 40)
        out.append((cfg, grid, tree, o, d))
    return out


def test_network_order_is_leaves_then_inner_preorder(scenes):
    for cfg, grid, tree, o, d in scenes:
        nodes = tree.network_nodes()
        L = tree.n_leaves
        assert len(nodes) == tree.n_nodes == 2 * L - 1
        np.testing.assert_array_equal(tree.info[nodes[:L], 3], np.arange(L))
        assert (tree.info[nodes[L:], 0] >= 0).all() and (np.diff(nodes[L:]) > 0).all()


@pytest.mark.parametrize("mode", [0, 1])
def test_hcheck_always_true_is_the_leaf_only_traversal(scenes, mode):
    """lod = 0, and a lod so small that every node descends, give exactly the
    leaf-only crossings."""
    for cfg, grid, tree, o, d in scenes:
        maxc = cfg.cap // cfg.steps
        ref = O.traverse(tree, o, d, maxc, mode=mode)
        for lod in (0.0, 1e-12):
            got = O.traverse(tree, o, d, maxc, mode=mode, lod=lod)
            for a, b in zip(ref, got):
                np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("mode", [0, 1])
def test_stack_traversal_equals_the_set_definition(scenes, mode):
    """Brute force: every node with a positive crossing whose ancestors all have
    positive crossings and descend, and which is a leaf or does not descend, sorted
    by entry -- equal to the stack traversal, bit for bit, at several lods."""
    for cfg, grid, tree, o, d in scenes:
        maxc = 255
        for lod in (0.002, 0.01, 0.05, 0.3, 3.0):
            a = O.traverse(tree, o, d, maxc, mode=mode, method=0, lod=lod)
            b = O.traverse(tree, o, d, maxc, mode=mode, method=1, lod=lod)
            for x, y in zip(a, b):
                np.testing.assert_array_equal(x, y)


def test_crossings_tile_the_root_interval_and_samples_lie_in_their_nodes(scenes):
    """At any lod the emitted nodes partition the ray's path through the root: the
    crossings are contiguous and cover the root interval, and every sample lies in the
    box of its crossing's node (FP64)."""
    for cfg, grid, tree, o, d in scenes:
        maxc = 255
        t0, t1, hit = O.root_interval(tree, o, d)
        nodes = tree.network_nodes()
        for lod in (0.01, 0.05, 0.3):
            nx, net, tin, tout = O.traverse(tree, o, d, maxc, mode=0, lod=lod)
            for r in np.nonzero(hit)[0][::7]:
                k = nx[r]
                assert k >= 1
                assert tin[r, 0] == pytest.approx(t0[r], abs=1e-12)
                assert tout[r, k - 1] == pytest.approx(t1[r], abs=1e-12)
                np.testing.assert_allclose(tout[r, :k - 1], tin[r, 1:k], atol=1e-12)
            t, dl, x = O.samples(o, d, nx, tin, tout, maxc, cfg.steps, maxc * cfg.steps, mode=0)
            for r in np.nonzero(hit)[0][::11]:
                for k in range(nx[r]):
                    bx = tree.box[nodes[net[r, k]]].astype(np.float64)
                    p = x[r, k * cfg.steps:(k + 1) * cfg.steps]
                    assert (p >= bx[:3] - 1e-12).all() and (p <= bx[3:] + 1e-12).all()


def test_coarsening_never_adds_crossings(scenes):
    for cfg, grid, tree, o, d in scenes:
        prev = None
        for lod in (0.0, 0.005, 0.02, 0.08, 0.3, 1.0, 10.0):
            nx = O.traverse(tree, o, d, 255, mode=1, lod=lod)[0]
            if prev is not None:
                assert (nx <= prev).all()
            prev = nx
        assert nx.max() <= 1                  # large enough lod: the root alone


def _constant_params(n_nets, width, hidden, lx, ld, sigma, rgb):
    per = S.params_per_leaf(width, hidden, lx, ld)
    P = np.zeros((n_nets, per), np.float32)
    P[:, -4] = math.log(math.expm1(sigma))   # softplus^-1
    P[:, -3:] = [math.log(c / (1 - c)) for c in rgb]
    return P.reshape(-1)


@pytest.mark.parametrize("lod", [0.0, 0.03, 0.3, 5.0])
def test_constant_density_closed_form_at_any_lod(scenes, lod):
    """Every network (leaves and inner nodes) of constant density sigma and colour c:
    whichever nodes HCheck selects, T = exp(-sigma L), opacity = 1 - T and
    rgb = c (1 - T) + bg T, with L the hit length."""
    cfg, grid, tree, _, _ = scenes[0]
    sigma, rgb = 0.8, (0.2, 0.5, 0.7)
    P = _constant_params(tree.n_nodes, cfg.width, cfg.hidden, cfg.lx, cfg.ld, sigma, rgb)
    s_eff = float(np.logaddexp(0.0, np.float32(math.log(math.expm1(sigma)))))
    c_eff = [1 / (1 + math.exp(-float(np.float32(math.log(c / (1 - c)))))) for c in rgb]
    s3 = math.sqrt(3.0)
    o = np.array([[-3, 0.1, 0.2], [0.3, -3, -0.4], [-3, -3, -3], [-3, 5, 0]], np.float32)
    d = np.array([[1, 0, 0], [0, 1, 0], [1 / s3, 1 / s3, 1 / s3], [1, 0, 0]], np.float32)
    L = np.array([2.0, 2.0, 2 * s3, 0.0])
    bg = (0.1, 0.0, 0.3)
    res = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, 512, t_term=0.0, bg=bg,
                   mode=0, lod=lod)
    Tf = np.exp(-s_eff * L)
    np.testing.assert_allclose(res["opacity"], 1 - Tf, atol=2e-7)
    for c in range(3):
        np.testing.assert_allclose(res["rgb"][:, c], c_eff[c] * (1 - Tf) + bg[c] * Tf, atol=2e-7)


@pytest.mark.parametrize("mode", [0, 1])
def test_render_with_hcheck_always_true_is_the_leaf_only_render(scenes, mode):
    """Per-node networks whose first L are the leaf networks: lod = 0 renders exactly
    the leaf-only image (the inner networks are never evaluated)."""
    cfg, grid, tree, o, d = scenes[0]
    P_leaf = S.xavier_weights(0, S.leaf_mean_density(grid, tree.leaf_cells()), cfg.width, cfg.hidden, cfg.lx,
                              cfg.ld)
    P_net = S.xavier_weights(0, S.leaf_mean_density(grid, tree.network_cells()), cfg.width, cfg.hidden, cfg.lx,
                             cfg.ld)
    per = S.params_per_leaf(cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    np.testing.assert_array_equal(P_net[:tree.n_leaves * per], P_leaf)
    a = O.render(tree, P_leaf, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=mode)
    b = O.render(tree, P_net, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=mode, lod=0.0)
    for k in ("rgb", "depth", "opacity", "n_gen"):
        np.testing.assert_array_equal(a[k], b[k])
    c = O.render(tree, P_net, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=mode, lod=0.3)
    assert c["n_gen"].sum() < a["n_gen"].sum()
