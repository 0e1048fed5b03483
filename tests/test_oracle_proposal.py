"""Pins of the proposal-sampler oracle (a learned sampler; not in the paper).

Gradient: central finite differences of the loss.  Cross-entropy: the closed form
at q = p.  Adam: the first step from zero moments moves every parameter by lr
against the sign of its gradient.  Bin selection: hand-worked cases.  Masked
sampling: an all-bins mask reproduces the plain render, kept crossings are exactly
those that overlap a kept bin, and the binned weights plus the residual
transmittance sum to one.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2310_01881_gb300 import scenes as S


def _rays(n, seed):
    rng = np.random.default_rng(seed)
    u = rng.normal(size=(n, 3)); u /= np.linalg.norm(u, axis=1, keepdims=True)
    o = 3.0 * u
    d = rng.uniform(-0.7, 0.7, (n, 3)) - o; d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, O.PROP_NPARAM)


@pytest.fixture(scope="module")
def c1():
    cfg = S.CONFIGS["c1"]
    grid = S.density_grid(S.scene_for("c1", 0), cfg.G)
    tree = O.build_tree(grid, cfg.max_depth)
    P = S.xavier_weights(0, S.leaf_mean_density(grid, tree.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    return cfg, tree, P


def test_gradient_matches_central_differences():
    o, d = _rays(6, 1)
    t0 = np.random.default_rng(2).uniform(1.5, 2.5, 6)
    tg = np.random.default_rng(3).dirichlet(np.ones(65) * 0.3, 6)
    P = _params(4)
    loss, g = O.prop_loss_grad(P, o, d, t0, tg)
    idx = np.random.default_rng(5).choice(O.PROP_NPARAM, 120, replace=False)
    bad = 0
    for i in idx:
        h = 1e-6 * max(1.0, abs(P[i]))
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        fd = (O.prop_loss_grad(Pp, o, d, t0, tg)[0] - O.prop_loss_grad(Pm, o, d, t0, tg)[0]) / (2 * h)
        if abs(fd - g[i]) > 1e-6 + 1e-5 * abs(g[i]):
            bad += 1
    assert bad <= 2  # a ReLU kink inside +-h is possible but rare
    assert loss > 0


def test_cross_entropy_closed_form_at_matching_prediction():
    """W3 = 0 and b3 = log p make the prediction q = p: loss = H(p), zero bias gradient."""
    p = np.random.default_rng(7).dirichlet(np.ones(65), 1)[0]
    P = _params(8)
    P[-65 - 65 * 32:-65] = 0.0
    P[-65:] = np.log(p)
    o, d = _rays(3, 9)
    t0 = np.full(3, 2.0)
    loss, g = O.prop_loss_grad(P, o, d, t0, np.tile(p, (3, 1)))
    assert loss == pytest.approx(-np.sum(p * np.log(p)), rel=1e-12)
    np.testing.assert_allclose(g[-65:], 0.0, atol=1e-15)
    q = O.prop_predict(P, o, d, t0)
    np.testing.assert_allclose(q, np.tile(p, (3, 1)), rtol=1e-12)


def test_adam_first_step_moves_by_lr_against_gradient_sign():
    P = _params(10)
    P0 = P.copy()
    g = np.random.default_rng(11).normal(size=P.size)
    m = np.zeros_like(P); v = np.zeros_like(P)
    O.prop_adam(P, g, m, v, 1, lr=1e-3)
    np.testing.assert_allclose(P - P0, -1e-3 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_bin_selection_hand_cases():
    q = np.zeros((4, 65))
    # ray 0: bins 3 (0.6) and 10 (0.395) reach 0.995 >= 0.99
    q[0, 3] = 0.6; q[0, 10] = 0.395; q[0, 64] = 0.005
    # ray 1: background 0.9 and bin 5 0.095 -> 0.995 (background counts toward coverage)
    q[1, 64] = 0.9; q[1, 5] = 0.095; q[1, 6] = 0.005
    # ray 2: flat over 64 bins: more than 16 depth bins needed -> fallback
    q[2, :64] = 1.0 / 64
    # ray 3: tie between bins 1 and 2 (0.5 each): lower index first, both needed
    q[3, 1] = 0.5; q[3, 2] = 0.5
    mask, fb = O.prop_select(q, 0.99, 16)
    assert mask[0] == (1 << 3) | (1 << 10) and fb[0] == 0
    assert mask[1] == (1 << 5) and fb[1] == 0
    assert fb[2] == 1 and mask[2] == np.uint64(2 ** 64 - 1)
    assert mask[3] == (1 << 1) | (1 << 2) and fb[3] == 0
    m2, f2 = O.prop_select(q[2:3], 0.99, 64)
    assert f2[0] == 0 and bin(int(m2[0])).count("1") == 64
    # the same decisions with the running sum in binary32: the margins are wide
    ms, fs = O.prop_select(q, 0.99, 16, single=True)
    assert (ms == mask).all() and (fs == fb).all()


def test_bin_selection_binary32_sum_absorbs_small_masses():
    """In binary32 an increment below half an ulp of the running sum is lost: after
    bin 0 (0.5), masses of 2^-26 leave the sum at 0.5, so a coverage of 0.5 + 2^-24
    is never reached and the ray runs past max_bins; in binary64 four of them reach it."""
    q = np.zeros((1, 65))
    q[0, 0] = 0.5
    q[0, 1:9] = 2.0 ** -26
    cov = 0.5 + 2.0 ** -24
    m64, f64 = O.prop_select(q, cov, 16)
    assert f64[0] == 0 and m64[0] == 0b11111
    m32, f32 = O.prop_select(q, cov, 16, single=True)
    assert f32[0] == 1 and m32[0] == np.uint64(2 ** 64 - 1)
    m32, f32 = O.prop_select(q, cov, 64, single=True)
    assert f32[0] == 0 and m32[0] == np.uint64(2 ** 64 - 1)   # every depth bin, zeros included


@pytest.mark.parametrize("mode", [0, 1])
def test_all_bins_mask_is_the_plain_render(c1, mode):
    cfg, tree, P = c1
    o, d = S.view_rays(cfg, 0, 0, 20, 20)
    plain = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=mode)
    ones = np.full(len(o), 2 ** 64 - 1, np.uint64)
    masked = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=mode,
                      mask=ones, fallback=np.zeros(len(o), np.int32))
    for k in ("rgb", "depth", "opacity", "n_gen"):
        np.testing.assert_array_equal(masked[k], plain[k])


def test_masked_sampling_keeps_exactly_the_overlapping_crossings(c1):
    cfg, tree, P = c1
    o, d = S.view_rays(cfg, 0, 0, 16, 16)
    t0, t1, hit = O.root_interval(tree, o, d, mode=0)
    rng = np.random.default_rng(12)
    mask = np.zeros(len(o), np.uint64)
    for r in range(len(o)):
        for k in rng.choice(64, 5, replace=False):
            mask[r] |= np.uint64(1 << int(k))
    res = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, 512, t_term=0.0, mode=0,
                   mask=mask, fallback=np.zeros(len(o), np.int32))
    nx, leaf, tin, tout = O.traverse(tree, o, d, 64, mode=0)
    for r in np.nonzero(hit)[0]:
        w = (t1[r] - t0[r]) / 64.0
        bins = [j for j in range(64) if (int(mask[r]) >> j) & 1]
        sure = maybe = 0
        for k in range(nx[r]):
            a, b = tin[r, k], tout[r, k]
            ov = max(min(b, t0[r] + (j + 1) * w) - max(a, t0[r] + j * w) for j in bins)
            sure += ov > 1e-9      # overlaps a kept bin by a positive length
            maybe += ov > -1e-9    # or touches one within rounding of the bin edges
        assert sure * cfg.steps <= res["n_gen"][r] <= maybe * cfg.steps


def test_binned_weights_sum_to_one(c1):
    cfg, tree, P = c1
    o, d = S.view_rays(cfg, 0, 0, 24, 24)
    for mode, tol in ((0, 1e-12), (1, 2e-6)):
        res = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=mode,
                       bins=True)
        np.testing.assert_allclose(res["bins"].sum(1), 1.0, atol=tol)
        np.testing.assert_allclose(res["bins"][:, 64], 1 - res["opacity"], atol=tol)


def test_proposal_forward_matches_library_matmul_chain():
    """The proposal network's forward pass is gamma_10(o + t0 d) ++ gamma_4(d) (the
    encoding is pinned on its own), then W1, ReLU, W2, ReLU, W3 and a softmax, with
    the weights stored row-major as [output][input] and the biases after each matrix.
    A numpy float64 chain of matmuls and a library softmax gives the same q; a
    transposed operand, a dropped bias or a swapped feature block would not."""
    from scipy.special import softmax
    rng = np.random.default_rng(17)
    P = S.proposal_init(3) * 2.0
    P[2880:2912] = rng.normal(size=32) * 0.3      # b1
    P[3936:3968] = rng.normal(size=32) * 0.3      # b2
    P[6048:6113] = rng.normal(size=65) * 0.3      # b3
    n = 40
    o = (rng.normal(size=(n, 3)) * 2.0).astype(np.float32)
    d = rng.normal(size=(n, 3)); d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    t0 = rng.uniform(0.0, 3.0, size=n)
    e = o + t0.astype(np.float32)[:, None] * d          # the sample point in FP32, as the rays are given
    feat = np.stack([np.concatenate([O.encode(e[r], 10), O.encode(d[r], 4)]) for r in range(n)])
    W1 = P[:2880].reshape(32, 90); b1 = P[2880:2912]
    W2 = P[2912:3936].reshape(32, 32); b2 = P[3936:3968]
    W3 = P[3968:6048].reshape(65, 32); b3 = P[6048:6113]
    h1 = np.maximum(feat @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    q_ref = softmax(h2 @ W3.T + b3, axis=1)
    q = O.prop_predict(P.astype(np.float64), o, d, t0)
    np.testing.assert_allclose(q, q_ref, rtol=1e-10, atol=1e-14)


def test_target_bins_on_hand_worked_edges():
    """The training targets put a sample at t into bin floor((t - t0) / w), w = (t1 -
    t0) / 64, clamped to [0, 63].  Hand-worked rays whose bin edges are exact: a sample
    on edge k is in bin k, one just below it in bin k - 1, one just above in bin k;
    t1 itself is in bin 63.  A width of (t1 - t0) / 63, an off-by-one or rounding
    instead of flooring fails one of these."""
    # FP64: [0, 64] (w = 1) and [2, 3] (w = 1/64)
    for t0, t1, w in ((0.0, 64.0, 1.0), (2.0, 3.0, 1.0 / 64.0)):
        k = np.arange(64)
        on = t0 + k * w
        below = np.nextafter(on[1:], -np.inf)
        above = np.nextafter(on, np.inf)
        three_q = on + 0.75 * w
        t = np.concatenate([on, below, above, three_q, [t1, t1 + 1.0, t0 - 1.0]])
        want = np.concatenate([k, k[1:] - 1, k, k, [63, 63, 0]])
        got = O.bin_indices(np.full(len(t), t0), np.full(len(t), t1), t, mode=0)
        np.testing.assert_array_equal(got, want)
    # FP32: [1, 5] (w = 4 * 2^-6 = 1/16 exactly); edges and their float neighbours
    t0, t1 = 1.0, 5.0
    k = np.arange(64)
    on = (np.float32(t0) + k.astype(np.float32) * np.float32(0.0625)).astype(np.float32)
    below = np.nextafter(on[1:], np.float32(-np.inf), dtype=np.float32)
    above = np.nextafter(on, np.float32(np.inf), dtype=np.float32)
    t = np.concatenate([on, below, above]).astype(np.float64)
    want = np.concatenate([k, k[1:] - 1, k])
    got = O.bin_indices(np.full(len(t), t0), np.full(len(t), t1), t, mode=1)
    np.testing.assert_array_equal(got, want)


def test_target_bins_against_brute_force_edge_count():
    """Brute force: the bin of t is the number of interior edges t0 + k w (k = 1..63)
    at or below t.  Random rays and samples (away from the edges by more than the
    rounding of the mode), both modes."""
    rng = np.random.default_rng(23)
    n = 20000
    t0 = rng.uniform(0.0, 3.0, n)
    t1 = t0 + rng.uniform(0.05, 4.0, n)
    t = t0 + rng.uniform(0.0, 1.0, n) * (t1 - t0)
    for mode in (0, 1):
        if mode == 1:
            t0m, t1m, tm = (a.astype(np.float32).astype(np.float64) for a in (t0, t1, t))
        else:
            t0m, t1m, tm = t0, t1, t
        w = (t1m - t0m) / 64.0
        edges = t0m[:, None] + np.arange(1, 64)[None, :] * w[:, None]
        ref = (tm[:, None] >= edges).sum(1)
        gap = np.abs(tm[:, None] - edges).min(1)
        far = gap > (1e-12 if mode == 0 else 1e-5) * np.maximum(1.0, np.abs(tm))
        assert far.mean() > 0.99
        got = O.bin_indices(t0m, t1m, tm, mode=mode)
        np.testing.assert_array_equal(got[far], ref[far])


def test_bf16_rounding_hand_ties_and_library_conversion():
    """bfloat16 keeps 8 significant bits, ties to even: 1 + 2^-8 lies halfway between
    1 and 1 + 2^-7 and goes to 1; 1 + 3 2^-8 goes to 1 + 2^-6; 255.5 (nine bits) goes
    to 256; just above a tie rounds up.  Random float32 values agree with torch's
    bfloat16 conversion (a library routine)."""
    cases = [(1 + 2 ** -8, 1.0), (1 + 3 * 2 ** -8, 1 + 2 ** -6), (-(1 + 2 ** -8), -1.0), (255.5, 256.0),
             (1 + 2 ** -8 + 2 ** -20, 1 + 2 ** -7), (0.0, 0.0), (3.0, 3.0), (2 ** -100, 2 ** -100)]
    for x, want in cases:
        assert O.bf16_round(x) == want, x
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = (rng.uniform(-1, 1, 4000) * 10.0 ** rng.uniform(-4, 4, 4000)).astype(np.float32)
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.bf16_round(float(v)) for v in x])
    np.testing.assert_array_equal(got, lib)


def test_bf16_proposal_forward_matches_library_chain_on_rounded_operands():
    """prop_predict(bf16=True) is the numpy float64 chain of the proposal network with
    every operand (features, weights, biases, hidden activations) rounded to bfloat16
    by torch; the FP64 prediction differs from it by about the bfloat16 rounding."""
    torch = pytest.importorskip("torch")
    from scipy.special import softmax

    def bf(a):
        return torch.from_numpy(np.asarray(a, np.float64)).to(torch.float32).to(torch.bfloat16).to(
            torch.float64).numpy()

    rng = np.random.default_rng(29)
    P = S.proposal_init(4) * 2.0
    P[2880:2912] = rng.normal(size=32) * 0.3
    P[3936:3968] = rng.normal(size=32) * 0.3
    P[6048:6113] = rng.normal(size=65) * 0.3
    n = 40
    o = (rng.normal(size=(n, 3)) * 2.0).astype(np.float32)
    d = rng.normal(size=(n, 3)); d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    t0 = rng.uniform(0.0, 3.0, size=n)
    e = o + t0.astype(np.float32)[:, None] * d
    feat = np.stack([np.concatenate([O.encode(e[r], 10), O.encode(d[r], 4)]) for r in range(n)])
    W1 = P[:2880].reshape(32, 90); b1 = P[2880:2912]
    W2 = P[2912:3936].reshape(32, 32); b2 = P[3936:3968]
    W3 = P[3968:6048].reshape(65, 32); b3 = P[6048:6113]
    h1 = np.maximum(bf(feat) @ bf(W1).T + bf(b1), 0.0)
    h2 = np.maximum(bf(h1) @ bf(W2).T + bf(b2), 0.0)
    q_ref = softmax(bf(h2) @ bf(W3).T + bf(b3), axis=1)
    q = O.prop_predict(P.astype(np.float64), o, d, t0, bf16=True)
    np.testing.assert_allclose(q, q_ref, rtol=1e-9, atol=1e-14)
    q64 = O.prop_predict(P.astype(np.float64), o, d, t0)
    rel = np.abs(np.log(q / q64))
    assert 1e-5 < rel.max() < 0.2
