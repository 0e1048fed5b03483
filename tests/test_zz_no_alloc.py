"""The allocation-free grouping entry point, checked against the render's own grouping.

amnerf_group_by_leaf_static serves callers that may not allocate device memory when
they call (fixed-budget frame loops, render threads where cudaMalloc/cudaFree are
banned because they can synchronise the device).  Its scratch is a static device
array, so this test runs it twice in a row on the crossings of a render and compares
its counts, offsets and per-leaf crossing sets with what amnerf_render_debug reports
(exact: they are integers).  Kept in its own file, collected last.
"""
import numpy as np
import pytest

from paper_2310_01881_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_grouping_matches_render_grouping_twice():
    from paper_2310_01881_gb300 import amnerf, build
    build.build()
    cfg = S.CONFIGS["c1"]
    R = amnerf.Renderer(0)
    try:
        grid = S.density_grid(S.scene_for("c1", 0), cfg.G)
        nl = R.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
        P = S.xavier_weights(0, S.leaf_mean_density(grid, R.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
        R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, "fp32")
        maxc = cfg.cap // cfg.steps
        for seed in (0, 1):
            o, d = S.view_rays(cfg, 0, seed)
            _, _, _, dbg, _ = R.render_debug(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                                             steps=cfg.steps, cap=cfg.cap)
            n = len(o)
            n_x = torch.from_numpy(dbg["n_x"]).cuda()
            leaf = torch.from_numpy(dbg["leaf"].astype(np.uint16).view(np.int16).reshape(-1).copy()).cuda()
            counts = torch.full((nl,), 7, dtype=torch.int32, device="cuda")      # stale contents on purpose
            offsets = torch.zeros(nl + 1, dtype=torch.int32, device="cuda")
            order = torch.zeros(n * maxc, dtype=torch.int32, device="cuda")
            amnerf.amnerf_group_by_leaf_static(n_x, leaf, n, maxc, nl, counts, offsets, order,
                                               torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            c = counts.cpu().numpy().view(np.uint32).astype(np.int64)
            off = offsets.cpu().numpy().view(np.uint32).astype(np.int64)
            got = order.cpu().numpy().view(np.uint32).astype(np.int64)
            np.testing.assert_array_equal(c, dbg["counts"])
            np.testing.assert_array_equal(off, dbg["offsets"])
            for l in range(nl):
                a, b = off[l], off[l + 1]
                np.testing.assert_array_equal(np.sort(got[a:b]), np.sort(dbg["order"][a:b]))
                assert np.all(dbg["leaf"].reshape(-1)[got[a:b]] == l)
        with pytest.raises(amnerf.AmnerfError) as ei:
            amnerf.amnerf_group_by_leaf_static(n_x, leaf, n, maxc, 4097, counts, offsets, order)
        assert ei.value.status == amnerf.E_INVAL
    finally:
        R.close()


def test_static_grouping_at_its_largest_size_ignores_foreign_leaf_ids_and_takes_empty_batches():
    """The documented limits, against a numpy counting sort (exact integers):
    n_leaves = 4096, the largest the static scratch holds (32 KB of shared memory in the
    scatter, the scan's full width); leaf ids drawn from [0, 4200), so ids >= n_leaves
    must be ignored; random crossing counts; then a batch of zero rays, which leaves
    all-zero counts and offsets (stale contents are overwritten)."""
    from paper_2310_01881_gb300 import amnerf, build
    build.build()
    rng = np.random.default_rng(3)
    n, maxc, nl = 50000, 24, 4096
    n_x = rng.integers(0, maxc + 1, n).astype(np.uint8)
    leaf = rng.integers(0, 4200, (n, maxc)).astype(np.uint16)
    valid = (np.arange(maxc)[None, :] < n_x[:, None]) & (leaf < nl)
    ids = np.nonzero(valid.reshape(-1))[0]
    lf = leaf.reshape(-1)[ids].astype(np.int64)
    want_counts = np.bincount(lf, minlength=nl)
    want_off = np.concatenate([[0], np.cumsum(want_counts)])
    stream = torch.cuda.current_stream().cuda_stream
    counts = torch.full((nl,), 9, dtype=torch.int32, device="cuda")
    offsets = torch.full((nl + 1,), 9, dtype=torch.int32, device="cuda")
    order = torch.zeros(n * maxc, dtype=torch.int32, device="cuda")
    amnerf.amnerf_group_by_leaf_static(torch.from_numpy(n_x).cuda(),
                                       torch.from_numpy(leaf.view(np.int16).reshape(-1).copy()).cuda(), n, maxc, nl,
                                       counts, offsets, order, stream)
    torch.cuda.synchronize()
    c = counts.cpu().numpy().view(np.uint32).astype(np.int64)
    off = offsets.cpu().numpy().view(np.uint32).astype(np.int64)
    got = order.cpu().numpy().view(np.uint32).astype(np.int64)[: want_off[-1]]
    np.testing.assert_array_equal(c, want_counts)
    np.testing.assert_array_equal(off, want_off)
    srt = ids[np.argsort(lf, kind="stable")]
    for a, b in zip(want_off[:-1], want_off[1:]):
        if b > a:
            np.testing.assert_array_equal(np.sort(got[a:b]), srt[a:b])
    # zero rays: only the clear and the scan run
    amnerf.amnerf_group_by_leaf_static(None, None, 0, maxc, nl, counts, offsets, None, stream)
    torch.cuda.synchronize()
    assert (counts.cpu().numpy() == 0).all() and (offsets.cpu().numpy() == 0).all()
