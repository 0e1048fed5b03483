"""Networks with a nonzero bias in every layer.  The seeded weights elsewhere have
zero hidden biases (only the density head's is not), so these tests are the ones
that reach each precision's bias path: the FP32 path's bias adds, BF16's layer-0 bias
input (a weight column against a constant-1 feature) and later layers' bias MMAs,
the two-threads-per-row kernel's bias stores, E4M3's epilogue bias (per-row scales)
and its BF16 bias MMA in accumulator units (static scales).  Against the oracle of
Sec. 3.1's network on the same tree and samples."""
import numpy as np
import pytest

import oracle as O
from paper_2310_01881_gb300 import scenes as S
from pixtol import check_pixels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2310_01881_gb300 import amnerf, build
    build.build()
    r = amnerf.Renderer(0)
    yield r
    r.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _psnr(a, b):
    return 10 * np.log10(1.0 / max(float(np.mean((np.asarray(a, np.float64) - b) ** 2)), 1e-30))


@pytest.fixture(scope="module")
def scene():
    cfg = S.CONFIGS["c1"]
    grid = S.density_grid(S.scene_for(cfg.scene, 3), cfg.G)
    tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    P0 = S.xavier_weights(3, S.leaf_mean_density(grid, tree.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    P = S.with_biases(P0, 3, cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    o, d = S.view_rays(cfg, 3, 0)
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8)
    ref0 = O.render(tree, P0, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8)
    return cfg, grid, tree, P, o, d, ref, ref0


def _load(R, scene, prec):
    cfg, grid, tree, P, o, d, _, _ = scene
    assert R.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac) == tree.n_leaves
    if prec == "fp8s":
        R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, "fp32")
        oc, dc = S.view_rays(cfg, 3, 7, 64, 64)   # calibration view, not the test view
        amax = R.calibrate_fp8(_dev(oc), _dev(dc), cfg.hidden, steps=cfg.steps, cap=cfg.cap)
        R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, act_max=amax)
    else:
        R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, prec)


def test_the_biases_change_the_image(scene):
    """The oracle's images with and without the drawn biases differ by far more than
    any tolerance below, so a bias path that dropped them would fail."""
    *_, ref, ref0 = scene
    assert _psnr(ref["rgb"], ref0["rgb"]) < 30.0


def test_fp32_pixels_with_biases(R, scene):
    cfg, grid, tree, P, o, d, _, _ = scene
    _load(R, scene, "fp32")
    rgb, depth, opac = [t.cpu().numpy() for t in R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)]
    ref = O.render(tree, P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=1, threads=8)
    check_pixels(((rgb, ref["rgb"]), (depth, ref["depth"]), (opac, ref["opacity"])), ref["ert_margin"],
                 "FP32 pixels, nonzero biases")


@pytest.mark.parametrize("prec,width_split,floor", [("bf16", 1, 45.0), ("bf16", 2, 45.0), ("fp8", 1, 30.0),
                                                     ("fp8s", 1, 30.0)])
def test_tensor_core_paths_with_biases(R, scene, prec, width_split, floor):
    from paper_2310_01881_gb300 import amnerf
    cfg, grid, tree, P, o, d, ref, ref0 = scene
    _load(R, scene, prec)
    amnerf.amnerf_set_tuning(R.ctx, 0, amnerf.SCHED_CONTIGUOUS, width_split)
    try:
        rgb = R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)[0].cpu().numpy()
    finally:
        amnerf.amnerf_set_tuning(R.ctx, 0, amnerf.SCHED_CONTIGUOUS)
    psnr = _psnr(rgb, ref["rgb"])
    print(f"{prec} (width split {width_split}) with biases: PSNR {psnr:.2f} dB against the FP64 oracle, "
          f"{_psnr(rgb, ref0['rgb']):.2f} dB against the bias-free image")
    assert np.all(np.isfinite(rgb))
    assert psnr >= floor
    assert psnr > _psnr(rgb, ref0["rgb"]) + 10.0


@pytest.mark.parametrize("width,hidden", [(64, 1), (64, 3), (32, 5), (64, 4)])
@pytest.mark.parametrize("prec", ["bf16", "fp8s"])
def test_bias_paths_across_network_shapes(R, width, hidden, prec):
    """The bias operands are per hidden layer (block bb, chunk l - 1 for BF16, l for
    E4M3 static): shapes outside the specialised ones run the generic instantiation,
    one hidden layer has no BF16 bias MMA at all.  Each against the FP64 oracle."""
    import dataclasses
    cfg = dataclasses.replace(S.CONFIGS["c1"], width=width, hidden=hidden)
    grid = S.density_grid(S.scene_for(cfg.scene, 4), cfg.G)
    tree = O.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    assert R.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac) == tree.n_leaves
    P0 = S.xavier_weights(4, S.leaf_mean_density(grid, tree.leaf_cells()), width, hidden, cfg.lx, cfg.ld)
    P = S.with_biases(P0, 4, width, hidden, cfg.lx, cfg.ld)
    if prec == "fp8s":
        R.load_mlps(P, width, hidden, cfg.lx, cfg.ld, "fp32")
        oc, dc = S.view_rays(cfg, 4, 7, 64, 64)
        amax = R.calibrate_fp8(_dev(oc), _dev(dc), hidden, steps=cfg.steps, cap=cfg.cap)
        R.load_mlps(P, width, hidden, cfg.lx, cfg.ld, act_max=amax)
    else:
        R.load_mlps(P, width, hidden, cfg.lx, cfg.ld, prec)
    o, d = S.view_rays(cfg, 4, 0)
    rgb = R.render(_dev(o), _dev(d), steps=cfg.steps, cap=cfg.cap)[0].cpu().numpy()
    ref = O.render(tree, P, width, hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8)
    ref0 = O.render(tree, P0, width, hidden, cfg.lx, cfg.ld, o, d, cfg.steps, cfg.cap, mode=0, threads=8)
    psnr = _psnr(rgb, ref["rgb"])
    print(f"{prec} {hidden} x {width} with biases: PSNR {psnr:.2f} dB (bias-free image {_psnr(ref['rgb'], ref0['rgb']):.2f} dB away)")
    assert np.all(np.isfinite(rgb))
    assert psnr >= (45.0 if prec == "bf16" else 30.0)
    assert psnr > _psnr(rgb, ref0["rgb"]) + 10.0
