"""Rendering from crossings given by the caller (amnerf_render_crossings): the
grouping, network and compositing steps (Sec. 3.5 Fig. "parallel", Sec. 3.1) driven
with arbitrary per-network counts.  Crossings taken from a render's own traversal
render bit for bit as that render; Zipf-distributed counts over the 4096-leaf tree's
networks give identical pixels with the grouped launch and with one launch per leaf;
out-of-range input is reported by the status word and leaves the context usable."""
import numpy as np
import pytest

import oracle as O
from paper_2310_01881_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2310_01881_gb300 import amnerf, build
    build.build()
    r = amnerf.Renderer(0)
    yield r
    r.close()


def _dev(a, dtype=None):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a if dtype is None else a.astype(dtype)).cuda()


def _setup(R, name, prec):
    cfg = S.CONFIGS[name]
    grid = S.density_grid(S.scene_for(cfg.scene, 0), cfg.G)
    R.build_tree(grid, cfg.max_depth, cfg.leaf_mass_frac)
    P = S.xavier_weights(0, S.leaf_mean_density(grid, R.leaf_cells()), cfg.width, cfg.hidden, cfg.lx, cfg.ld)
    R.load_mlps(P, cfg.width, cfg.hidden, cfg.lx, cfg.ld, prec)
    return cfg, grid


@pytest.mark.parametrize("prec,jitter", [("fp32", 0), ("bf16", 0), ("bf16", 99)])
def test_crossings_of_the_traversal_render_as_the_render(R, prec, jitter):
    from paper_2310_01881_gb300 import amnerf
    cfg, _ = _setup(R, "c2", prec)
    o, d = S.view_rays(cfg, 0, 0, 256, 256)
    do, dd = _dev(o), _dev(d)
    rgb, depth, opac, dbg, st = R.render_debug(do, dd, cfg.steps, cfg.cap, jitter=jitter)
    n = len(o)
    out = (torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"), torch.empty(n, device="cuda"))
    st2 = amnerf.amnerf_render_crossings(R.ctx, do, dd, _dev(dbg["n_x"]),
                                         _dev(dbg["leaf"].astype(np.uint16).view(np.int16).reshape(-1)),
                                         _dev(dbg["t_in"].reshape(-1)), _dev(dbg["t_out"].reshape(-1)), *out,
                                         steps=cfg.steps, cap=cfg.cap, stats=True, jitter=jitter)
    for a, b in zip((rgb, depth, opac), out):
        np.testing.assert_array_equal(a, b.cpu().numpy())
    assert st2["samples_generated"] == st["samples_generated"]


def test_zipf_counts_over_4096_leaves_grouped_equals_per_leaf_launches(R):
    """Counts drawn from Zipf s = 1.1 over the 4096 leaf networks (seeded rank
    permutation): the per-network totals are the drawn ones, and the grouped
    persistent launch gives the same pixels as one launch per leaf."""
    from paper_2310_01881_gb300 import amnerf
    cfg, _ = _setup(R, "c4", "bf16")
    maxc = cfg.cap // cfg.steps
    n = 60000
    n_x, leaf, t_in, t_out = S.zipf_crossings(n, maxc, R.n_leaves, 1.1, 3)
    o, d = S.view_rays(cfg, 0, 0, 300, 200)
    do, dd = _dev(o), _dev(d)
    args = (do, dd, _dev(n_x), _dev(leaf.view(np.int16).reshape(-1)), _dev(t_in.reshape(-1)),
            _dev(t_out.reshape(-1)))
    outs = []
    for sched in (amnerf.SCHED_CONTIGUOUS, amnerf.SCHED_PER_LEAF):
        amnerf.amnerf_set_tuning(R.ctx, 0, sched)
        out = (torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"), torch.empty(n, device="cuda"))
        st = amnerf.amnerf_render_crossings(R.ctx, *args, *out, steps=cfg.steps, cap=cfg.cap, stats=True)
        assert st["crossings"] == n * maxc
        outs.append([t.cpu().numpy() for t in out])
    amnerf.amnerf_set_tuning(R.ctx, 0, amnerf.SCHED_CONTIGUOUS)
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    assert np.isfinite(outs[0][0]).all()
    # the drawn counts are Zipf-distributed (the oracle's counting sort of the lists)
    counts, _, _ = O.group(n_x.astype(np.int32), leaf.astype(np.int32), maxc, cfg.steps, R.n_leaves)
    c = np.sort(counts[counts > 0])[::-1].astype(np.float64)
    slope = np.polyfit(np.log(np.arange(1, len(c) + 1)), np.log(c), 1)[0]
    assert -1.25 < slope < -0.95


def test_out_of_range_crossings_are_reported_and_the_context_survives(R):
    from paper_2310_01881_gb300 import amnerf
    cfg, _ = _setup(R, "c1", "bf16")
    maxc = cfg.cap // cfg.steps
    n = 1000
    n_x, leaf, t_in, t_out = S.zipf_crossings(n, maxc, R.n_leaves, 1.1, 5)
    leaf[17, 3] = R.n_leaves + 5                     # a network that is not loaded
    o, d = S.view_rays(cfg, 0, 0, 50, 20)
    do, dd = _dev(o), _dev(d)
    out = (torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"), torch.empty(n, device="cuda"))
    with pytest.raises(amnerf.AmnerfError) as e:
        amnerf.amnerf_render_crossings(R.ctx, do, dd, _dev(n_x), _dev(leaf.view(np.int16).reshape(-1)),
                                       _dev(t_in.reshape(-1)), _dev(t_out.reshape(-1)), *out, steps=cfg.steps,
                                       cap=cfg.cap, stats=True)
    assert e.value.status == amnerf.E_INVAL
    rgb, _, _ = R.render(do, dd, cfg.steps, cfg.cap)
    R.sync()
    assert np.isfinite(rgb.cpu().numpy()).all()
