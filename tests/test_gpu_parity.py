"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bit-exact: tree, per-ray crossings (leaf ids, entries, exits), per-leaf counts and
offsets, and the grouped crossing sets.  Floating point (FP32 path): pixels within
1e-5 max abs of the FP32-mode oracle, which follows the same sample positions; the
only difference left is the order of the network's sums and of the transmittance
products.  Rays whose transmittance passes within 0.1% of the termination threshold
may legitimately stop one sample apart (both results are correct roundings), and
are held to 2e-4 instead (one sample's weight is at most t_term = 1e-4).
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_01881_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from pixtol import ERT_TOL, PIX_TOL, check_pixels  # noqa: F401


@pytest.fixture(scope="module")
def R():
    from paper_2310_01881_gb300 import amnerf, build
    build.build()
    r = amnerf.Renderer(0)
    yield r
    r.close()


def _setup(R, cfg, seed=0, G=None, prec="fp32", scale=1.0):
    grid = S.density_grid(S.scene_for(cfg.scene, seed), G or cfg.G) * np.float32(scale)
    nl = R.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    assert nl == tree.n_leaves
    # each side derives its weights from its own tree (the trees are compared bit for bit)
    P_gpu = S.xavier_weights(seed, S.leaf_mean_density(grid, R.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    P_or = S.xavier_weights(seed, S.leaf_mean_density(grid, tree.leaf_cells()), cfg.width, cfg.hidden, cfg.lx,
                            cfg.ld)
    R.load_mlps(P_gpu, cfg.width, cfg.hidden, cfg.lx, cfg.ld, prec)
    return grid, tree, P_or


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _compare_tree(R, tree):
    nodes = R.tree()
    assert len(nodes) == tree.n_nodes
    for i, n in enumerate(nodes):
        np.testing.assert_array_equal(np.array(list(n.lo) + list(n.hi), np.float32), tree.box[i])
        np.testing.assert_array_equal(np.array(list(n.cell_lo) + list(n.cell_hi)), tree.cells[i])
        assert [n.axis, n.left, n.right, n.leaf_id, n.code, n.depth] == list(tree.info[i])
        assert n.mass == tree.mass[i]
        if n.axis >= 0:
            assert n.split == tree.split[i]


def _adversarial_rays():
    s3 = 1 / np.sqrt(3.0)
    o = [(-3, 0.1, 0.2), (0.3, -3, -0.4), (-3, -3, -3), (-3, 5, 0), (0, 0, 0), (0.2, -0.3, 0.1),
         (-3, 1, 1), (-3, 0, 0), (0, -3, 0), (0, 0, -3), (-1, -1, -1), (1.5, 0.25, -0.125)]
    d = [(1, 0, 0), (0, 1, 0), (s3, s3, s3), (1, 0, 0), (0, 0, 1), (-s3, s3, -s3),
         (1, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (s3, s3, s3), (-1, 0, 0)]
    return np.array(o, np.float32), np.array(d, np.float32)


def _rays(cfg, seed, views=1, w=None, h=None):
    os_, ds_ = [], []
    for v in range(views):
        o, d = S.view_rays(cfg, seed, v, w, h)
        os_.append(o); ds_.append(d)
    return np.concatenate(os_), np.concatenate(ds_)


def _check_crossings(dbg, tree, o, d, maxc, steps):
    nx, leaf, tin, tout = O.traverse(tree, o, d, maxc, mode=1)
    np.testing.assert_array_equal(dbg["n_x"].astype(np.int64), nx)
    valid = np.arange(maxc)[None, :] < nx[:, None]
    np.testing.assert_array_equal(dbg["leaf"][valid], leaf[valid])
    np.testing.assert_array_equal(dbg["t_in"][valid], tin[valid].astype(np.float32))
    np.testing.assert_array_equal(dbg["t_out"][valid], tout[valid].astype(np.float32))
    counts, offsets, order = O.group(nx, leaf, maxc, steps, tree.n_leaves)
    np.testing.assert_array_equal(dbg["counts"] * steps, counts)
    np.testing.assert_array_equal(dbg["offsets"] * steps, offsets)
    tot = int(nx.sum())
    got = dbg["order"][:tot]
    for l in range(tree.n_leaves):
        a, b = offsets[l] // steps, offsets[l + 1] // steps
        np.testing.assert_array_equal(np.sort(got[a:b]), np.sort(order[a:b]))


def _check_pixels(rgb, depth, opac, ref, tol=PIX_TOL, label="FP32 pixels"):
    return check_pixels(((rgb, ref["rgb"]), (depth, ref["depth"]), (opac, ref["opacity"])), ref["ert_margin"], label,
                        tol)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_c1_tree_traversal_grouping_bit_exact(R, seed):
    cfg = S.CONFIGS["c1"]
    _, tree, _ = _setup(R, cfg, seed)
    _compare_tree(R, tree)
    o, d = _rays(cfg, seed)
    ao, ad = _adversarial_rays()
    o = np.concatenate([o, ao]); d = np.concatenate([d, ad])
    *_, dbg, st = R.render_debug(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)
    _check_crossings(dbg, tree, o, d, cfg.cap // cfg.steps, cfg.steps)
    assert st["samples_generated"] == int(dbg["n_x"].astype(np.int64).sum()) * cfg.steps


@pytest.mark.parametrize("seed", [0, 3])
def test_c1_fp32_pixels_match_fp32_oracle(R, seed):
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, seed)
    o, d = _rays(cfg, seed)
    rgb, depth, opac, dbg, st = R.render_debug(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1, threads=8,
                   full=True)
    _check_pixels(rgb, depth, opac, ref)
    # per-sample network outputs at every generated slot
    gen = np.arange(cfg.cap)[None, :] < ref["n_gen"][:, None]
    so = dbg["slot_out"][gen].astype(np.float64)
    ro = ref["slot_out"][gen]
    assert np.max(np.abs(so[:, 1:] - ro[:, 1:])) <= 2e-6
    assert np.max(np.abs(so[:, 0] - ro[:, 0]) / np.maximum(1.0, ro[:, 0])) <= 2e-6
    assert st["samples_composited"] == int(ref["n_eval"].sum()) or \
        abs(st["samples_composited"] - int(ref["n_eval"].sum())) <= int((ref["ert_margin"] < 1e-3).sum())


def test_c1_fp32_pixels_on_an_opaque_scene(R):
    """Every density x1000: most rays terminate inside their first crossings, so the
    early ray termination of the compositing is exercised; pixels within 1e-5 of the
    FP32-mode oracle, rays near the threshold reported (and held to 2e-4)."""
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, 0, scale=1000.0)
    o, d = _rays(cfg, 0, views=2)
    rgb, depth, opac, dbg, st = R.render_debug(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1, threads=8)
    assert (ref["n_eval"] < ref["n_gen"]).mean() > 0.3          # termination happens on most hit rays
    _check_pixels(rgb, depth, opac, ref, label="FP32 pixels, opaque scene (density x1000)")


def test_c1_fp32_close_to_fp64_definition(R):
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, 0)
    o, d = _rays(cfg, 0)
    rgb, depth, opac = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)]
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8)
    mse = np.mean((rgb - ref["rgb"]) ** 2)
    assert 10 * np.log10(1.0 / max(mse, 1e-30)) > 80.0


@pytest.mark.parametrize("steps,cap", [(1, 24), (2, 32), (4, 16), (8, 8), (16, 64), (32, 96), (8, 2040)])
def test_sampling_rates_and_caps(R, steps, cap):
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, 1)
    o, d = _rays(cfg, 1, 1, 24, 24)
    rgb, depth, opac, dbg, _ = R.render_debug(_dev(o), _dev(d), steps=steps, cap=cap)
    _check_crossings(dbg, tree, o, d, cap // steps, steps)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, steps, cap, mode=1, threads=8)
    _check_pixels(rgb, depth, opac, ref)


def test_single_leaf_tree_and_inside_origins(R):
    cfg = S.CONFIGS["c1"]
    grid = S.density_grid(S.scene_for("c1", 2), 16)
    assert R.build_tree(grid, 0) == 1
    tree = O.build_tree(grid, 0)
    P = S.xavier_weights(5, np.array([3.0]), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, "fp32")
    rng = np.random.default_rng(4)
    o = rng.uniform(-0.9, 0.9, (300, 3)).astype(np.float32)
    d = rng.normal(size=(300, 3)); d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    rgb, depth, opac, dbg, _ = R.render_debug(_dev(o), _dev(d), steps=8, cap=64)
    _check_crossings(dbg, tree, o, d, 8, 8)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, 8, 64, bg=(0.2, 0.4, 0.6), mode=1)
    rgb2, depth2, opac2 = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), steps=8, cap=64, bg=(0.2, 0.4, 0.6))]
    _check_pixels(rgb2, depth2, opac2, ref)


def test_empty_batch_and_all_miss(R):
    cfg = S.CONFIGS["c1"]
    _setup(R, cfg, 0)
    e = torch.zeros((0, 3), device="cuda")
    rgb, depth, opac, st = R.render(e, e, stats=True)
    assert rgb.shape == (0, 3) and st["samples_generated"] == 0
    o = np.tile(np.array([[-3, 5, 0]], np.float32), (1000, 1))
    d = np.tile(np.array([[1, 0, 0]], np.float32), (1000, 1))
    rgb, depth, opac, st = R.render(_dev(o), _dev(d), bg=(0.25, 0.5, 0.75), stats=True)
    assert st["samples_generated"] == 0
    np.testing.assert_array_equal(rgb.cpu().numpy(), np.tile([[0.25, 0.5, 0.75]], (1000, 1)).astype(np.float32))
    assert float(depth.abs().max()) == 0.0 and float(opac.abs().max()) == 0.0


def test_c2_scale_tree_and_sampled_pixels(R):
    """Paper-scale workload (800x800 x 8 views, <=256 leaves, 4x64 MLP, cap 192) in the
    launch configuration of the benchmark; a seeded sample of rays is checked against
    the FP32-mode oracle, and properties are checked on all rays."""
    cfg = S.CONFIGS["c2"]
    _, tree, P = _setup(R, cfg, 0)
    _compare_tree(R, tree)
    o, d = _rays(cfg, 0, cfg.views)
    do, dd = _dev(o), _dev(d)
    rgb, depth, opac, st = R.render(do, dd, steps=cfg.steps, cap=cfg.cap, stats=True)
    rgb, depth, opac = rgb.cpu().numpy(), depth.cpu().numpy(), opac.cpu().numpy()
    assert np.all(np.isfinite(rgb)) and np.all((opac >= 0) & (opac <= 1 + 1e-6))
    assert np.all(rgb >= -1e-6) and np.all(rgb <= 1 + 1e-6)
    idx = S.ray_subset(len(o), 2048, 1)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o[idx], d[idx], cfg.steps, cfg.cap, mode=1,
                   threads=16)
    _check_pixels(rgb[idx], depth[idx], opac[idx], ref)
    nx, *_ = O.traverse(tree, o[idx], d[idx], cfg.cap // cfg.steps, mode=1)
    assert st["samples_generated"] >= int(nx.sum()) * cfg.steps


# ---- stratified jitter of the sample positions (Sec. 3.5: random placement within an interval) ----

@pytest.mark.parametrize("seed", [0, 3])
def test_c1_fp32_jittered_pixels_match_fp32_oracle(R, seed):
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, seed)
    o, d = _rays(cfg, seed)
    jit = 1000 + seed
    rgb, depth, opac, dbg, st = R.render_debug(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap, jitter=jit)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1, threads=8,
                   full=True, jitter=jit)
    _check_pixels(rgb, depth, opac, ref)
    gen = np.arange(cfg.cap)[None, :] < ref["n_gen"][:, None]
    so = dbg["slot_out"][gen].astype(np.float64)
    ro = ref["slot_out"][gen]
    assert np.max(np.abs(so[:, 1:] - ro[:, 1:])) <= 2e-6
    assert np.max(np.abs(so[:, 0] - ro[:, 0]) / np.maximum(1.0, ro[:, 0])) <= 2e-6
    # the jitter moved the samples: the midpoint render differs
    mid = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1, threads=8,
                   full=True)
    assert np.mean(np.abs(mid["slot_out"][gen][:, 0] - ro[:, 0]) > 1e-6) > 0.5


def test_c1_bf16_jittered_against_fp64_oracle(R):
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, 1, prec="bf16")
    o, d = _rays(cfg, 1)
    rgb = R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap, jitter=77)[0].cpu().numpy()
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8,
                   jitter=77)
    assert _psnr(rgb, ref["rgb"]) >= 45.0


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_jitter_is_keyed_by_the_ray_not_its_batch_position(R, prec):
    cfg = S.CONFIGS["c1"]
    _setup(R, cfg, 2, prec=prec)
    o, d = _rays(cfg, 2)
    p = np.random.default_rng(5).permutation(len(o))
    a = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap, jitter=31)]
    b = [t.cpu().numpy() for t in R.render(_dev(o[p]), _dev(d[p]), steps=cfg.steps, cap=cfg.cap, jitter=31)]
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x[p], y)


# ---- empty-space skipping over the guidance grid (Sec. 4.1: the density grid marks empty regions) ----

@pytest.mark.parametrize("seed,jitter", [(0, 0), (3, 0), (1, 9)])
def test_c1_skipping_crossings_bit_exact_and_fp32_pixels(R, seed, jitter):
    cfg = S.CONFIGS["c1"]
    grid, tree, P = _setup(R, cfg, seed)
    thr = float(np.quantile(grid, 0.7))
    o, d = _rays(cfg, seed)
    ao, ad = _adversarial_rays()
    o = np.concatenate([o, ao]); d = np.concatenate([d, ad])
    maxc = cfg.cap // cfg.steps
    rgb, depth, opac, dbg, st = R.render_debug(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap, jitter=jitter,
                                               skip_empty=thr)
    nx, leaf, tin, tout = O.traverse(tree, o, d, maxc, mode=1, skip=(grid, thr, cfg.steps, jitter))
    np.testing.assert_array_equal(dbg["n_x"].astype(np.int64), nx)
    valid = np.arange(maxc)[None, :] < nx[:, None]
    np.testing.assert_array_equal(dbg["leaf"][valid], leaf[valid])
    np.testing.assert_array_equal(dbg["t_in"][valid], tin[valid].astype(np.float32))
    np.testing.assert_array_equal(dbg["t_out"][valid], tout[valid].astype(np.float32))
    full, *_ = O.traverse(tree, o, d, maxc, mode=1)
    assert nx.sum() < full.sum()                   # crossings were skipped
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1, threads=8,
                   jitter=jitter, skip=(grid, thr))
    _check_pixels(rgb, depth, opac, ref)
    assert st["samples_generated"] == int(ref["n_gen"].sum())


def test_c2_skipping_bf16_sampled_psnr(R):
    cfg = S.CONFIGS["c2"]
    grid, tree, P = _setup(R, cfg, 0, prec="bf16")
    thr = 0.01
    o, d = _rays(cfg, 0, 1, 400, 400)
    rgb, _, _, st = R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap, stats=True, skip_empty=thr)
    plain = R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap, stats=True)[3]
    assert st["samples_generated"] < plain["samples_generated"]
    idx = S.ray_subset(len(o), 2048, 3)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o[idx], d[idx], cfg.steps, cfg.cap, mode=0,
                   threads=16, skip=(grid, thr))
    assert _psnr(rgb.cpu().numpy()[idx], ref["rgb"]) >= 45.0


def test_skipping_with_proposal_masks_matches_oracle(R):
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c1"]
    grid, tree, P = _setup(R, cfg, 0)
    amnerf.amnerf_proposal_set(R.ctx, S.proposal_init(11) * 3.0)
    thr = float(np.quantile(grid, 0.6))
    o, d = S.view_rays(cfg, 0, 4)
    rgb, depth, opac, dbg, st = R.render_debug(_dev(o), _dev(d), cfg.steps, cfg.cap, proposal=True, coverage=0.7,
                                               max_bins=64, skip_empty=thr)
    mask, fb = dbg["prop_mask"], dbg["prop_fallback"].astype(np.int32)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1,
                   mask=mask, fallback=fb, skip=(grid, thr))
    np.testing.assert_array_equal(dbg["n_x"].astype(np.int64) * cfg.steps, ref["n_gen"])
    check_pixels(((rgb, ref["rgb"]),), ref["ert_margin"], "skipping with proposal masks")


@pytest.mark.parametrize("prec,jitter,scale", [("fp32", 0, 1000.0), ("bf16", 5, 1000.0), ("fp32", 3, 1.0),
                                               ("bf16", 0, 30.0)])
def test_waves_bit_identical_to_one_pass(R, prec, jitter, scale):
    """Early ray termination in waves changes which samples are evaluated, not the
    pixels: every wave size gives the one-pass render bit for bit, with the same
    composited samples and fewer or equally many evaluated."""
    cfg = S.CONFIGS["c1"]
    _setup(R, cfg, 0, prec=prec, scale=scale)
    o, d = _rays(cfg, 0, views=2)
    do, dd = _dev(o), _dev(d)
    *ref, st0 = R.render(do, dd, cfg.steps, cfg.cap, jitter=jitter, stats=True)
    ref = [t.cpu().numpy() for t in ref]
    assert st0["samples_evaluated"] == st0["samples_generated"]
    for W in (1, 2, 3, 8):
        *out, st = R.render(do, dd, cfg.steps, cfg.cap, jitter=jitter, stats=True, ert_wave=W)
        for a, b in zip(ref, out):
            np.testing.assert_array_equal(a, b.cpu().numpy())
        assert st["samples_composited"] == st0["samples_composited"]
        assert st["crossings"] == st0["crossings"] and st["samples_generated"] == st0["samples_generated"]
        assert st["samples_composited"] <= st["samples_evaluated"] <= st["samples_generated"]


def test_waves_evaluate_only_up_to_the_terminating_wave(R):
    """On the x1000 density scene most rays end inside their first crossings.  With
    waves of W crossings a ray is evaluated through the wave in which T drops below
    t_term: min(n_x, W ceil(composited / (8 W))) crossings, or all n_x when it never
    terminates.  The total matches that count from the FP32-mode oracle's composited
    samples (rays within 1e-3 of the termination threshold may differ by their
    crossings), and it is well below the samples generated."""
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, 0, scale=1000.0)
    o, d = _rays(cfg, 0)
    do, dd = _dev(o), _dev(d)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1, threads=8)
    comp, gen = ref["n_eval"].astype(np.int64), ref["n_gen"].astype(np.int64)
    nx = gen // cfg.steps
    amb = ref["ert_margin"] < 1e-3
    for W in (1, 2):
        per = W * cfg.steps
        waves_run = np.where(comp < gen, (comp + per - 1) // per, -1)
        xc = np.where(comp < gen, np.minimum(nx, waves_run * W), nx)
        *_, st = R.render(do, dd, cfg.steps, cfg.cap, stats=True, ert_wave=W)
        expect = int(xc.sum()) * cfg.steps
        assert abs(st["samples_evaluated"] - expect) <= int(nx[amb].sum()) * cfg.steps
        assert st["samples_evaluated"] < (0.9 if W == 1 else 1.0) * st["samples_generated"]


def test_waves_with_proposal_masks_and_skipping(R):
    """Waves run on whatever crossings the traversal kept (proposal masks, empty-space
    skipping): the pixels are those of the one-pass render with the same options."""
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c1"]
    _setup(R, cfg, 0, prec="bf16", scale=100.0)
    amnerf.amnerf_proposal_set(R.ctx, S.proposal_init(11) * 3.0)
    o, d = _rays(cfg, 0)
    do, dd = _dev(o), _dev(d)
    for kw in (dict(proposal=True, coverage=0.9, max_bins=64), dict(skip_empty=0.01),
               dict(proposal=True, coverage=0.99, max_bins=16, skip_empty=0.01, jitter=9)):
        ref = [t.cpu().numpy() for t in R.render(do, dd, cfg.steps, cfg.cap, **kw)]
        out = [t.cpu().numpy() for t in R.render(do, dd, cfg.steps, cfg.cap, ert_wave=1, **kw)]
        for a, b in zip(ref, out):
            np.testing.assert_array_equal(a, b)


def test_wave_parameters_are_checked(R):
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c1"]
    _setup(R, cfg, 0)
    o = _dev(np.zeros((4, 3)))
    for steps, cap, W in ((8, 64, 256), (8, 64, -1), (4, 64, 1)):
        with pytest.raises(amnerf.AmnerfError) as ei:
            R.render(o, o, steps, cap, ert_wave=W)
        assert ei.value.status == amnerf.E_INVAL


def test_host_buffer_entry_point_matches_device(R):
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c1"]
    _setup(R, cfg, 0)
    o, d = _rays(cfg, 0)
    rgb, depth, opac = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)]
    h = [np.zeros((len(o), 3), np.float32), np.zeros(len(o), np.float32), np.zeros(len(o), np.float32)]
    amnerf.amnerf_render_host(R.ctx, o, d, *h, steps=cfg.steps, cap=cfg.cap)
    np.testing.assert_array_equal(h[0], rgb)
    np.testing.assert_array_equal(h[1], depth)
    np.testing.assert_array_equal(h[2], opac)


def test_host_buffer_entry_point_in_chunks_matches_device(R):
    """2.1 M rays: the host path renders in chunks with overlapped copies."""
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c1"]
    _setup(R, cfg, 0, prec="bf16")
    o, d = S.view_rays(cfg, 0, 0, 1448, 1448)
    rgb, depth, opac = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)]
    h = [torch.empty((len(o), 3)).pin_memory().numpy(), torch.empty(len(o)).pin_memory().numpy(),
         torch.empty(len(o)).pin_memory().numpy()]
    amnerf.amnerf_render_host(R.ctx, o, d, *h, steps=cfg.steps, cap=cfg.cap)
    np.testing.assert_array_equal(h[0], rgb)
    np.testing.assert_array_equal(h[1], depth)
    np.testing.assert_array_equal(h[2], opac)


def test_invalid_arguments_are_rejected(R):
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c1"]
    ctx = amnerf.amnerf_create(0, None)
    try:
        o = _dev(np.zeros((4, 3)))
        out = (torch.empty((4, 3), device="cuda"), torch.empty(4, device="cuda"), torch.empty(4, device="cuda"))
        with pytest.raises(amnerf.AmnerfError) as ei:
            amnerf.amnerf_render(ctx, o, o, *out)
        assert ei.value.status == amnerf.E_NOTREE
        grid = S.density_grid(S.scene_for("c1", 0), 16)
        with pytest.raises(amnerf.AmnerfError) as ei:
            amnerf.amnerf_build_tree(ctx, grid, 13)
        assert ei.value.status == amnerf.E_INVAL
        bad = grid.copy(); bad[0, 0, 0] = -1
        with pytest.raises(amnerf.AmnerfError):
            amnerf.amnerf_build_tree(ctx, bad, 3)
        nl = amnerf.amnerf_build_tree(ctx, grid, 3)
        with pytest.raises(amnerf.AmnerfError) as ei:
            amnerf.amnerf_render(ctx, o, o, *out)
        assert ei.value.status == amnerf.E_NOMLP
        P = S.xavier_weights(0, np.ones(nl), 32, 2, 10, 4)
        with pytest.raises(amnerf.AmnerfError):
            amnerf.amnerf_load_mlps(ctx, P, nl + 1, 32, 2, 10, 4)
        with pytest.raises(amnerf.AmnerfError):
            amnerf.amnerf_load_mlps(ctx, P, nl, 48, 2, 10, 4)
        amnerf.amnerf_load_mlps(ctx, P, nl, 32, 2, 10, 4)
        for kw in ({"steps": 3}, {"steps": 8, "cap": 4}, {"steps": 1, "cap": 300}, {"t_term": -1.0}):
            with pytest.raises(amnerf.AmnerfError) as ei:
                amnerf.amnerf_render(ctx, o, o, *out, **kw)
            assert ei.value.status == amnerf.E_INVAL
        amnerf.amnerf_render(ctx, o, _dev(np.tile([[1, 0, 0]], (4, 1))), *out)
        amnerf.amnerf_sync(ctx)
    finally:
        amnerf.amnerf_destroy(ctx)


# ----------------------------------------------------------------------------------
# BF16 tcgen05 path: every result states max abs and PSNR against the FP64 oracle.
# BF16 keeps 8 significant bits (relative rounding 2^-9 per operand); with FP32
# accumulation over at most 96 terms the pre-activation error stays near 1e-2 of
# its scale, which moves sigmoid colours by < 5e-3 and PSNR stays far above 45 dB.
# ----------------------------------------------------------------------------------

def _psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - b) ** 2))
    return 10 * np.log10(1.0 / max(mse, 1e-30))


@pytest.mark.parametrize("seed", [0, 2])
def test_c1_bf16_against_fp64_oracle(R, seed):
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, seed, prec="bf16")
    o, d = _rays(cfg, seed)
    rgb, depth, opac, dbg, st = R.render_debug(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)
    _check_crossings(dbg, tree, o, d, cfg.cap // cfg.steps, cfg.steps)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8,
                   full=True)
    psnr = _psnr(rgb, ref["rgb"])
    err = np.abs(rgb - ref["rgb"]).max()
    print(f"bf16 c1 seed {seed}: PSNR {psnr:.2f} dB, max abs rgb {err:.3e}")
    assert psnr >= 45.0
    assert err <= 3e-2
    assert np.abs(opac - ref["opacity"]).max() <= 3e-2
    gen = np.arange(cfg.cap)[None, :] < ref["n_gen"][:, None]
    so = dbg["slot_out"][gen].astype(np.float64)
    ro = ref["slot_out"][gen]
    assert np.max(np.abs(so[:, 1:] - ro[:, 1:])) <= 2e-2
    assert np.max(np.abs(so[:, 0] - ro[:, 0]) / np.maximum(1.0, ro[:, 0])) <= 5e-2


@pytest.mark.parametrize("width,hidden", [(64, 1), (64, 3), (32, 5)])
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8", "fp8s"])
def test_network_shapes_outside_the_specialised_ones(R, width, hidden, prec):
    """The network kernels are specialised for the 4 x 64 and 2 x 32 shapes; every other
    shape runs the generic instantiation (hidden count read at run time).  c1 scene
    and view with these shapes, against the FP64 oracle: the FP32 path to 1e-5 of the
    FP32-mode oracle, the others by PSNR."""
    import dataclasses
    cfg = dataclasses.replace(S.CONFIGS["c1"], width=width, hidden=hidden)
    grid, tree, P = _setup(R, cfg, 1, prec="fp32" if prec == "fp8s" else prec)
    o, d = _rays(cfg, 1)
    if prec == "fp8s":
        oc, dc = S.view_rays(cfg, 1, 7, 64, 64)
        amax = R.calibrate_fp8(_dev(oc), _dev(dc), cfg.hidden, steps=cfg.steps, cap=cfg.cap)
        R.load_mlps(_gpu_weights(R, cfg, grid, 1), cfg.width, cfg.hidden, cfg.lx, cfg.ld, act_max=amax)
    rgb, depth, opac = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)]
    assert np.all(np.isfinite(rgb))
    if prec == "fp32":
        ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1, threads=8)
        _check_pixels(rgb, depth, opac, ref)
        return
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8)
    psnr = _psnr(rgb, ref["rgb"])
    print(f"{prec} {hidden} x {width}: PSNR {psnr:.2f} dB")
    assert psnr >= (45.0 if prec == "bf16" else 30.0)


def test_c2_bf16_sampled_psnr(R):
    cfg = S.CONFIGS["c2"]
    _, tree, P = _setup(R, cfg, 0, prec="bf16")
    o, d = _rays(cfg, 0, cfg.views)
    rgb, depth, opac = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)]
    assert np.all(np.isfinite(rgb))
    idx = S.ray_subset(len(o), 4096, 2)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o[idx], d[idx], cfg.steps, cfg.cap, mode=0,
                   threads=16)
    psnr = _psnr(rgb[idx], ref["rgb"])
    print(f"bf16 c2: PSNR {psnr:.2f} dB, max abs {np.abs(rgb[idx] - ref['rgb']).max():.3e}")
    assert psnr >= 45.0


def test_c4_full_size_grouped_launch_sampled(R):
    """The batching workload at its full size, in the benchmark's launch: 4096 leaves,
    16 views of 1920x1080 (33.2 M rays, about 2.5 G samples) in one persistent
    grouped BF16 launch.  Tree bit-exact; a seeded subset of rays: crossing counts equal
    to the FP32-mode oracle's and pixels >= 45 dB against the FP64 oracle."""
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c4"]
    _, tree, P = _setup(R, cfg, 0, prec="bf16")
    _compare_tree(R, tree)
    o, d = _rays(cfg, 0, cfg.views)
    assert len(o) == 16 * 1920 * 1080
    do, dd = _dev(o), _dev(d)
    rgb, depth, opac, st = R.render(do, dd, steps=cfg.steps, cap=cfg.cap, stats=True)
    rgb = rgb.cpu().numpy()
    assert np.all(np.isfinite(rgb))
    idx = S.ray_subset(len(o), 4096, 5)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o[idx], d[idx], cfg.steps, cfg.cap, mode=0,
                   threads=16)
    psnr = _psnr(rgb[idx], ref["rgb"])
    print(f"bf16 c4 full size: {st['samples_generated'] / 1e9:.2f} G samples, PSNR {psnr:.2f} dB on 4096 rays")
    assert st["samples_generated"] > 2e9
    assert psnr >= 45.0
    # the sampled rays' crossing counts, through the FP32-mode oracle (bit-exact traversal)
    nx, _, _, _ = O.traverse(tree, o[idx], d[idx], cfg.cap // cfg.steps, mode=1)
    sub = R.render_debug(_dev(o[idx]), _dev(d[idx]), steps=cfg.steps, cap=cfg.cap)[3]
    np.testing.assert_array_equal(sub["n_x"].astype(np.int64), nx)
    del do, dd
    torch.cuda.empty_cache()


@pytest.mark.parametrize("steps,cap", [(1, 24), (4, 16), (16, 64), (32, 96)])
def test_bf16_sampling_rates(R, steps, cap):
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, 1, prec="bf16")
    o, d = _rays(cfg, 1, 1, 24, 24)
    rgb, depth, opac, dbg, _ = R.render_debug(_dev(o), _dev(d), steps=steps, cap=cap)
    _check_crossings(dbg, tree, o, d, cap // steps, steps)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, steps, cap, mode=0)
    assert _psnr(rgb, ref["rgb"]) >= 45.0


# ----------------------------------------------------------------------------------
# FP8 E4M3 tcgen05 path (per-output-channel weight scales, per-row activation
# scales, FP32 accumulation).  E4M3 keeps 4 significant bits (relative rounding
# 2^-4 per operand), so the bar is a stated error, not BF16's: PSNR >= 30 dB and
# colour error below 0.1 on these scenes; the numbers are printed.
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 2])
def test_c1_fp8_against_fp64_oracle(R, seed):
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, seed, prec="fp8")
    o, d = _rays(cfg, seed)
    rgb, depth, opac, dbg, st = R.render_debug(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)
    _check_crossings(dbg, tree, o, d, cfg.cap // cfg.steps, cfg.steps)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8)
    psnr = _psnr(rgb, ref["rgb"])
    err = np.abs(rgb - ref["rgb"]).max()
    print(f"fp8 c1 seed {seed}: PSNR {psnr:.2f} dB, max abs rgb {err:.3e}")
    assert np.all(np.isfinite(rgb))
    assert psnr >= 30.0
    assert err <= 0.1


def test_c2_fp8_sampled_psnr(R):
    cfg = S.CONFIGS["c2"]
    _, tree, P = _setup(R, cfg, 0, prec="fp8")
    o, d = _rays(cfg, 0, cfg.views)
    rgb = R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)[0].cpu().numpy()
    idx = S.ray_subset(len(o), 4096, 2)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o[idx], d[idx], cfg.steps, cfg.cap, mode=0,
                   threads=16)
    psnr = _psnr(rgb[idx], ref["rgb"])
    print(f"fp8 c2: PSNR {psnr:.2f} dB, max abs {np.abs(rgb[idx] - ref['rgb']).max():.3e}")
    assert np.all(np.isfinite(rgb)) and psnr >= 30.0


# ----------------------------------------------------------------------------------
# E4M3 with static per-leaf, per-layer activation scales: the calibration (FP32
# networks on the GPU) against the oracle's input ranges over the same samples, then
# the network with those scales against the FP64 oracle, calibrated on another view.
# ----------------------------------------------------------------------------------

def _gpu_weights(R, cfg, grid, seed):
    return S.xavier_weights(seed, S.leaf_mean_density(grid, R.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)


def test_fp8_calibration_matches_oracle_input_ranges(R):
    cfg = S.CONFIGS["c1"]
    _, tree, P = _setup(R, cfg, 0, prec="fp32")
    o, d = _rays(cfg, 0)
    got = R.calibrate_fp8(_dev(o), _dev(d), cfg.hidden, steps=cfg.steps, cap=cfg.cap)
    maxc = cfg.cap // cfg.steps
    nx, leaf, tin, tout = O.traverse(tree, o, d, maxc, mode=1)
    _, _, x = O.samples(o, d, nx, tin, tout, maxc, cfg.steps, cfg.cap, mode=1)
    Pl = np.asarray(P).reshape(tree.n_leaves, -1)
    want = np.zeros((tree.n_leaves, cfg.hidden))
    valid = np.arange(maxc)[None, :] < nx[:, None]
    for lf in range(tree.n_leaves):
        rr, kk = np.nonzero(valid & (leaf == lf))
        if len(rr) == 0:
            continue
        slots = (kk[:, None] * cfg.steps + np.arange(cfg.steps)[None, :]).ravel()
        rows = np.repeat(rr, cfg.steps)
        want[lf] = O.mlp_input_absmax(Pl[lf], cfg.width, cfg.hidden, cfg.lx, cfg.ld, x[rows, slots], d[rows])
    assert (want > 0).any()
    np.testing.assert_allclose(got, want, rtol=2e-5, atol=1e-6)


@pytest.mark.parametrize("seed", [0, 2])
def test_c1_fp8_static_scales_against_fp64_oracle(R, seed):
    cfg = S.CONFIGS["c1"]
    grid, tree, P = _setup(R, cfg, seed, prec="fp32")
    oc, dc = S.view_rays(cfg, seed, 7, 64, 64)  # calibration view, not the test view
    amax = R.calibrate_fp8(_dev(oc), _dev(dc), cfg.hidden, steps=cfg.steps, cap=cfg.cap)
    R.load_mlps(_gpu_weights(R, cfg, grid, seed), cfg.width, cfg.hidden, cfg.lx, cfg.ld, act_max=amax)
    o, d = _rays(cfg, seed)
    rgb, depth, opac = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)]
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8)
    psnr = _psnr(rgb, ref["rgb"])
    err = np.abs(rgb - ref["rgb"]).max()
    print(f"fp8 static c1 seed {seed}: PSNR {psnr:.2f} dB, max abs rgb {err:.3e}")
    assert np.all(np.isfinite(rgb))
    assert psnr >= 30.0
    assert err <= 0.1


def test_c2_fp8_static_scales_sampled_psnr(R):
    cfg = S.CONFIGS["c2"]
    grid, tree, P = _setup(R, cfg, 0, prec="fp32")
    oc, dc = S.view_rays(cfg, 0, 100, 400, 400)  # calibration view outside the 8 test views
    amax = R.calibrate_fp8(_dev(oc), _dev(dc), cfg.hidden, steps=cfg.steps, cap=cfg.cap)
    R.load_mlps(_gpu_weights(R, cfg, grid, 0), cfg.width, cfg.hidden, cfg.lx, cfg.ld, act_max=amax)
    o, d = _rays(cfg, 0, cfg.views)
    rgb = R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)[0].cpu().numpy()
    idx = S.ray_subset(len(o), 4096, 2)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o[idx], d[idx], cfg.steps, cfg.cap, mode=0,
                   threads=16)
    psnr = _psnr(rgb[idx], ref["rgb"])
    print(f"fp8 static c2: PSNR {psnr:.2f} dB, max abs {np.abs(rgb[idx] - ref['rgb']).max():.3e}")
    assert np.all(np.isfinite(rgb)) and psnr >= 30.0


def test_fp8_static_weight_scales_are_per_output_channel(R):
    """The rows of the last hidden layer of every leaf scaled by factors from 10^-3 to
    10^3, and the head's columns by the inverse factors: the same network function
    (ReLU is positively homogeneous).  With per-output-channel weight scales the scaled
    rows quantise to the same E4M3 values and the scale moves into the epilogue's FMA,
    so the render is as close to the FP64 oracle as the unscaled one's.  One weight
    scale per layer would flush the rows scaled by 10^-3 (10^-6 of the layer's largest
    weight) to zero."""
    cfg = S.CONFIGS["c1"]
    grid, tree, P = _setup(R, cfg, 0, prec="fp32")
    W = _gpu_weights(R, cfg, grid, 0).reshape(R.n_leaves, -1).copy()
    k0, w, h = S.mlp_input_width(cfg.lx, cfg.ld), cfg.width, cfg.hidden
    last = w * k0 + w + (h - 2) * (w * w + w)          # start of the last hidden layer
    head = last + w * w + w
    f = 10.0 ** np.random.default_rng(9).uniform(-3, 3, w)
    Ws = W.copy()
    Ws[:, last:last + w * w] = (W[:, last:last + w * w].reshape(-1, w, w) * f[None, :, None]).reshape(len(W), -1)
    Ws[:, last + w * w:head] = W[:, last + w * w:head] * f[None, :]
    Ws[:, head:head + 4 * w] = (W[:, head:head + 4 * w].reshape(-1, 4, w) / f[None, None, :]).reshape(len(W), -1)
    oc, dc = S.view_rays(cfg, 0, 7, 64, 64)
    o, d = _rays(cfg, 0)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8)
    out = {}
    for name, Wx in (("plain", W), ("scaled", Ws)):
        Wx = Wx.astype(np.float32).reshape(-1)
        R.load_mlps(Wx, cfg.width, cfg.hidden, cfg.lx, cfg.ld, "fp32")
        amax = R.calibrate_fp8(_dev(oc), _dev(dc), cfg.hidden, steps=cfg.steps, cap=cfg.cap)
        R.load_mlps(Wx, cfg.width, cfg.hidden, cfg.lx, cfg.ld, act_max=amax)
        out[name] = R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)[0].cpu().numpy()
    p_plain, p_scaled = _psnr(out["plain"], ref["rgb"]), _psnr(out["scaled"], ref["rgb"])
    p_pair = _psnr(out["scaled"], out["plain"])
    print(f"fp8 static, rows x 10^-3..10^3: PSNR vs FP64 {p_scaled:.2f} dB (unscaled {p_plain:.2f}); "
          f"scaled vs unscaled render {p_pair:.2f} dB")
    assert p_scaled >= 30.0 and p_scaled >= p_plain - 1.0
    assert p_pair >= p_plain + 6.0


def test_fp8_static_entry_points_reject_bad_use(R):
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c1"]
    grid, _, _ = _setup(R, cfg, 0, prec="bf16")
    o, d = _rays(cfg, 0, 1, 8, 8)
    with pytest.raises(amnerf.AmnerfError) as e:        # calibration needs the FP32 networks
        R.calibrate_fp8(_dev(o), _dev(d), cfg.hidden, steps=cfg.steps, cap=cfg.cap)
    assert e.value.status == amnerf.E_INVAL
    W = _gpu_weights(R, cfg, grid, 0)
    bad = np.full((R.n_leaves, cfg.hidden), np.nan, np.float32)
    with pytest.raises(amnerf.AmnerfError) as e:
        R.load_mlps(W, cfg.width, cfg.hidden, cfg.lx, cfg.ld, act_max=bad)
    assert e.value.status == amnerf.E_INVAL


# ----------------------------------------------------------------------------------
# Launch configurations, CUDA-graph capture and 64-bit sample slots.  A sample's
# network output does not depend on which worker computes it, so every schedule
# must give bit-identical pixels.
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp32"])
def test_every_schedule_gives_identical_pixels(R, prec):
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c2"]
    _setup(R, cfg, 0, prec=prec)
    o, d = _rays(cfg, 0, 1, 256, 256)
    do, dd = _dev(o), _dev(d)
    amnerf.amnerf_set_tuning(R.ctx, 0, amnerf.SCHED_CONTIGUOUS, 1)
    ref = [t.cpu().numpy() for t in R.render(do, dd, cfg.steps, cfg.cap)]
    _, _, max_groups, _ = amnerf.amnerf_get_tuning(R.ctx)
    groups = range(1, max_groups + 1) if prec != "fp32" else [0]
    splits = (1, 2) if prec == "bf16" else (1,)
    for ws in splits:     # hidden-width tiling: one or two threads per sample row
        for g in groups:
            for sched in (amnerf.SCHED_CONTIGUOUS, amnerf.SCHED_INTERLEAVED, amnerf.SCHED_DYNAMIC,
                          amnerf.SCHED_PER_LEAF):
                amnerf.amnerf_set_tuning(R.ctx, g, sched, ws)
                got = [t.cpu().numpy() for t in R.render(do, dd, cfg.steps, cfg.cap)]
                for a, b in zip(got, ref):
                    np.testing.assert_array_equal(a, b, err_msg=f"groups {g} schedule {sched} width split {ws}")
    amnerf.amnerf_set_tuning(R.ctx, 0, amnerf.SCHED_CONTIGUOUS)


def test_autotune_picks_a_valid_configuration(R):
    from paper_2310_01881_gb300 import amnerf
    cfg = S.CONFIGS["c2"]
    _setup(R, cfg, 0, prec="bf16")
    o, d = _rays(cfg, 0, 1, 400, 400)
    do, dd = _dev(o), _dev(d)
    ref = [t.cpu().numpy() for t in R.render(do, dd, cfg.steps, cfg.cap)]
    out = (torch.empty((len(o), 3), device="cuda"), torch.empty(len(o), device="cuda"), torch.empty(len(o), device="cuda"))
    g, sched, ws, ms = amnerf.amnerf_autotune(R.ctx, do, dd, *out, steps=cfg.steps, cap=cfg.cap, reps=2)
    g2, s2, max_groups, ws2 = amnerf.amnerf_get_tuning(R.ctx)
    assert 1 <= g <= max_groups and sched in (0, 1, 2) and ws in (1, 2) and ms > 0
    assert (g2, s2, ws2) == (g, sched, ws)
    got = [t.cpu().numpy() for t in R.render(do, dd, cfg.steps, cfg.cap)]
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    amnerf.amnerf_set_tuning(R.ctx, 0, amnerf.SCHED_CONTIGUOUS)


def test_cuda_graph_capture_and_replay(R):
    cfg = S.CONFIGS["c2"]
    _setup(R, cfg, 0, prec="bf16")
    o1, d1 = _rays(cfg, 0, 1, 320, 320)
    o2, d2 = _rays(cfg, 1, 1, 320, 320)
    do, dd = _dev(o1), _dev(d1)
    g, out = R.capture(do, dd, cfg.steps, cfg.cap)
    for o, d in ((o2, d2), (o1, d1)):
        do.copy_(_dev(o)); dd.copy_(_dev(d))
        g.replay()
        torch.cuda.synchronize()
        got = [t.cpu().numpy() for t in out]
        ref = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), cfg.steps, cfg.cap)]
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)
    R.sync()


def test_sample_slots_beyond_32_bits(R):
    """25.6 M rays x cap 192 = 4.9 G sample slots: the last copies of a repeated ray
    set must render exactly like the first copies."""
    cfg = S.CONFIGS["c2"]
    _, tree, P = _setup(R, cfg, 0, prec="bf16")
    o, d = _rays(cfg, 0, cfg.views)
    reps = 5
    assert len(o) * reps * cfg.cap > 2 ** 32
    do = _dev(o).repeat(reps, 1)
    dd = _dev(d).repeat(reps, 1)
    rgb, depth, opac = R.render(do, dd, cfg.steps, cfg.cap)
    torch.cuda.synchronize()
    n = len(o)
    first = rgb[:n].cpu().numpy()
    last = rgb[(reps - 1) * n:].cpu().numpy()
    np.testing.assert_array_equal(first, last)
    np.testing.assert_array_equal(opac[:n].cpu().numpy(), opac[(reps - 1) * n:].cpu().numpy())
    idx = S.ray_subset(n, 512, 3)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o[idx], d[idx], cfg.steps, cfg.cap, mode=0,
                   threads=16)
    assert _psnr(last[idx], ref["rgb"]) >= 45.0
    del do, dd, rgb, depth, opac
    torch.cuda.empty_cache()


def test_bounded_device_wait_reports_timeout_and_context_survives(R):
    """Failure detection without a fault: a device wait that nothing completes gives up
    after its cycle limit, the call reports E_TIMEOUT, and the next render works."""
    from paper_2310_01881_gb300 import amnerf
    st = amnerf.amnerf_selftest_wait(R.ctx, 20_000_000)   # ~10 ms at 2 GHz
    assert st == amnerf.E_TIMEOUT
    amnerf.amnerf_sync(R.ctx)                              # status word was cleared
    cfg = S.CONFIGS["c1"]
    _setup(R, cfg, 0, prec="bf16")
    o, d = _rays(cfg, 0, 1, 16, 16)
    rgb = R.render(_dev(o), _dev(d), cfg.steps, cfg.cap)[0]
    torch.cuda.synchronize()
    assert torch.isfinite(rgb).all()
