"""Thin ctypes binding of libamnerf (include/amnerf.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device buffers
are torch CUDA tensors (PyTorch provides memory and streams); all arithmetic of the
rendering path runs in the library's CUDA kernels.  There is no fallback: when the
library is missing or does not load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libamnerf.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_NOTREE, E_NOMLP, E_TIMEOUT, E_DEVICE, E_UNSUPPORTED = range(9)
FP32, BF16, FP8E4M3 = 0, 1, 2
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp8": FP8E4M3}


class AmnerfError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({_status_name(status)}) {msg}".rstrip())


class amnerf_tree_params(ctypes.Structure):
    _fields_ = [("max_depth", ctypes.c_int), ("leaf_mass_frac", ctypes.c_double)]


class amnerf_node(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("cell_lo", ctypes.c_int32 * 3),
                ("cell_hi", ctypes.c_int32 * 3), ("axis", ctypes.c_int32), ("split", ctypes.c_float),
                ("left", ctypes.c_int32), ("right", ctypes.c_int32), ("leaf_id", ctypes.c_int32),
                ("code", ctypes.c_uint32), ("depth", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mass", ctypes.c_double)]


class amnerf_mlp_desc(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_int), ("ld", ctypes.c_int), ("hidden", ctypes.c_int), ("width", ctypes.c_int),
                ("prec", ctypes.c_int)]


class amnerf_render_params(ctypes.Structure):
    _fields_ = [("steps_per_leaf", ctypes.c_int), ("max_samples", ctypes.c_int), ("t_term", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("use_proposal", ctypes.c_int), ("coverage", ctypes.c_float),
                ("max_bins", ctypes.c_int), ("jitter_seed", ctypes.c_uint64), ("skip_empty", ctypes.c_int),
                ("empty_threshold", ctypes.c_float), ("ert_wave", ctypes.c_int), ("lod", ctypes.c_float)]


PROPOSAL_PARAMS = 6113


SCHED_CONTIGUOUS, SCHED_INTERLEAVED, SCHED_DYNAMIC, SCHED_PER_LEAF = range(4)


class amnerf_tuning(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int), ("schedule", ctypes.c_int), ("width_split", ctypes.c_int)]


class amnerf_stats(ctypes.Structure):
    _fields_ = [("rays", ctypes.c_uint64), ("crossings", ctypes.c_uint64), ("samples_generated", ctypes.c_uint64),
                ("samples_composited", ctypes.c_uint64), ("tiles", ctypes.c_uint64),
                ("fallback_rays", ctypes.c_uint64), ("ms", ctypes.c_float * 4), ("proposal_ms", ctypes.c_float),
                ("samples_evaluated", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {"rays": self.rays, "crossings": self.crossings, "samples_generated": self.samples_generated,
                "samples_composited": self.samples_composited, "tiles": self.tiles,
                "fallback_rays": self.fallback_rays, "ms": list(self.ms), "proposal_ms": self.proposal_ms,
                "samples_evaluated": self.samples_evaluated}


class amnerf_debug(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("n_x", "leaf", "t_in", "t_out", "counts", "offsets", "order",
                                               "slot_out", "prop_mask", "prop_fallback", "prop_q")]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libamnerf (build it first with paper_2310_01881_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libamnerf is not built ({p} missing); run paper_2310_01881_gb300.build.build()")
    lib = ctypes.CDLL(p)
    V, I, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    S = ctypes.c_int
    sig = {
        "amnerf_create": ([ctypes.POINTER(V), I, V], S),
        "amnerf_set_stream": ([V, V], S),
        "amnerf_build_tree": ([V, V, I, V, ctypes.POINTER(amnerf_tree_params), ctypes.POINTER(I)], S),
        "amnerf_get_tree": ([V, V, I, ctypes.POINTER(I)], S),
        "amnerf_load_mlps": ([V, ctypes.POINTER(amnerf_mlp_desc), I, V], S),
        "amnerf_load_mlps_fp8_static": ([V, ctypes.POINTER(amnerf_mlp_desc), I, V, V], S),
        "amnerf_calibrate_fp8": ([V, V, V, L, ctypes.POINTER(amnerf_render_params), V], S),
        "amnerf_render": ([V, V, V, L, ctypes.POINTER(amnerf_render_params), V, V, V, V], S),
        "amnerf_render_debug": ([V, V, V, L, ctypes.POINTER(amnerf_render_params), V, V, V,
                                 ctypes.POINTER(amnerf_debug), V], S),
        "amnerf_render_host": ([V, V, V, L, ctypes.POINTER(amnerf_render_params), V, V, V, V], S),
        "amnerf_render_crossings": ([V, V, V, L, ctypes.POINTER(amnerf_render_params), V, V, V, V, V, V, V, V], S),
        "amnerf_sync": ([V], S),
        "amnerf_selftest_wait": ([V, ctypes.c_uint64], S),
        "amnerf_group_by_leaf_static": ([V, V, L, I, I, V, V, V, V], S),
        "amnerf_proposal_set": ([V, V, V, V, I], S),
        "amnerf_proposal_get": ([V, V, V, V, ctypes.POINTER(I)], S),
        "amnerf_proposal_targets": ([V, V, V, L, ctypes.POINTER(amnerf_render_params), V, V, V, V, V], S),
        "amnerf_proposal_train": ([V, V, V, V, V, L, I, I, ctypes.c_float, ctypes.c_uint64, V], S),
        "amnerf_proposal_grad": ([V, V, V, V, V, L, V, V], S),
        "amnerf_proposal_predict": ([V, V, V, L, ctypes.c_float, I, V, V, V], S),
        "amnerf_set_timing": ([V, I], S),
        "amnerf_set_tuning": ([V, ctypes.POINTER(amnerf_tuning)], S),
        "amnerf_get_tuning": ([V, ctypes.POINTER(amnerf_tuning), ctypes.POINTER(I)], S),
        "amnerf_autotune": ([V, V, V, L, ctypes.POINTER(amnerf_render_params), V, V, V, I,
                             ctypes.POINTER(amnerf_tuning), ctypes.POINTER(ctypes.c_float)], S),
        "amnerf_status_string": ([S], ctypes.c_char_p),
        "amnerf_last_error": ([V], ctypes.c_char_p),
        "amnerf_destroy": ([V], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _status_name(s: int) -> str:
    try:
        return load().amnerf_status_string(s).decode()
    except Exception:  # pragma: no cover - only used in messages
        return "?"


def _check(ctx, status: int, where: str):
    if status != OK:
        msg = load().amnerf_last_error(ctx).decode() if ctx else ""
        raise AmnerfError(status, where, msg)


def _ptr(t) -> int | None:
    """Device pointer of a contiguous CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _hptr(a: np.ndarray) -> int:
    return a.ctypes.data


# --------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# --------------------------------------------------------------------------------------

def amnerf_create(device: int = 0, stream: int | None = None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = load().amnerf_create(ctypes.byref(ctx), device, stream)
    _check(None, st, "amnerf_create")
    return ctx


def amnerf_destroy(ctx) -> None:
    load().amnerf_destroy(ctx)


def amnerf_set_stream(ctx, stream: int | None) -> None:
    _check(ctx, load().amnerf_set_stream(ctx, stream), "amnerf_set_stream")


def amnerf_set_timing(ctx, enable: bool) -> None:
    _check(ctx, load().amnerf_set_timing(ctx, int(enable)), "amnerf_set_timing")


def amnerf_build_tree(ctx, grid: np.ndarray, max_depth: int, leaf_mass_frac: float = 0.0,
                      bbox=(-1.0, -1.0, -1.0, 1.0, 1.0, 1.0)) -> int:
    g = np.ascontiguousarray(grid, dtype=np.float32)
    if g.ndim != 3 or not (g.shape[0] == g.shape[1] == g.shape[2]):
        raise ValueError("grid must be (G, G, G)")
    bb = np.ascontiguousarray(bbox, dtype=np.float64)
    tp = amnerf_tree_params(max_depth, leaf_mass_frac)
    nl = ctypes.c_int()
    st = load().amnerf_build_tree(ctx, _hptr(g), g.shape[0], _hptr(bb), ctypes.byref(tp), ctypes.byref(nl))
    _check(ctx, st, "amnerf_build_tree")
    return nl.value


def amnerf_get_tree(ctx) -> list:
    n = ctypes.c_int()
    load().amnerf_get_tree(ctx, None, 0, ctypes.byref(n))
    arr = (amnerf_node * max(n.value, 1))()
    _check(ctx, load().amnerf_get_tree(ctx, arr, n.value, ctypes.byref(n)), "amnerf_get_tree")
    return list(arr[: n.value])


def amnerf_load_mlps(ctx, weights: np.ndarray, n_leaves: int, width: int, hidden: int, lx: int, ld: int,
                     prec: int = FP32) -> None:
    w = np.ascontiguousarray(weights, dtype=np.float32)
    desc = amnerf_mlp_desc(lx, ld, hidden, width, prec)
    _check(ctx, load().amnerf_load_mlps(ctx, ctypes.byref(desc), n_leaves, _hptr(w)), "amnerf_load_mlps")


def amnerf_load_mlps_fp8_static(ctx, weights: np.ndarray, n_leaves: int, width: int, hidden: int, lx: int, ld: int,
                                act_max: np.ndarray) -> None:
    w = np.ascontiguousarray(weights, dtype=np.float32)
    a = np.ascontiguousarray(act_max, dtype=np.float32)
    if a.size != n_leaves * hidden:
        raise ValueError("act_max must hold n_leaves x hidden values")
    desc = amnerf_mlp_desc(lx, ld, hidden, width, FP8E4M3)
    _check(ctx, load().amnerf_load_mlps_fp8_static(ctx, ctypes.byref(desc), n_leaves, _hptr(w), _hptr(a)),
           "amnerf_load_mlps_fp8_static")


def amnerf_calibrate_fp8(ctx, o, d, n_leaves: int, hidden: int, steps: int = 8, cap: int = 64,
                         t_term: float = 1e-4, bg=(0.0, 0.0, 0.0), lod: float = 0.0) -> np.ndarray:
    """Largest |input| of every hidden layer per network over the samples of these rays
    (FP32 networks must be loaded); returns float32 [n_networks, hidden]."""
    out = np.zeros((n_leaves, hidden), dtype=np.float32)
    p = _params(steps, cap, t_term, bg, lod=lod)
    _check(ctx, load().amnerf_calibrate_fp8(ctx, _ptr(o), _ptr(d), o.shape[0], ctypes.byref(p), _hptr(out)),
           "amnerf_calibrate_fp8")
    return out


def _params(steps: int, cap: int, t_term: float, bg, proposal: bool = False, coverage: float = 0.99,
            max_bins: int = 16, jitter: int = 0, skip_empty=None, ert_wave: int = 0,
            lod: float = 0.0) -> amnerf_render_params:
    """jitter: 0 = samples at stratum midpoints, else the seed of the stratified jitter.
    skip_empty: None, or the density threshold of empty-space skipping.
    ert_wave: 0 = one pass, else crossings per wave of early ray termination.
    lod: 0 = leaves only, else the adaptive hierarchical sampling threshold."""
    return amnerf_render_params(steps, cap, t_term, (ctypes.c_float * 3)(*bg), int(proposal), coverage, max_bins,
                                int(jitter) & ((1 << 64) - 1), int(skip_empty is not None),
                                float(skip_empty) if skip_empty is not None else 0.0, int(ert_wave), float(lod))


def amnerf_render(ctx, o, d, rgb, depth, opacity, steps: int = 8, cap: int = 64, t_term: float = 1e-4,
                  bg=(0.0, 0.0, 0.0), stats: bool = False, proposal: bool = False, coverage: float = 0.99,
                  max_bins: int = 16, jitter: int = 0, skip_empty=None, ert_wave: int = 0, lod: float = 0.0):
    """Enqueue a render of CUDA tensors o, d (n, 3) into rgb (n, 3), depth, opacity (n,)."""
    p = _params(steps, cap, t_term, bg, proposal, coverage, max_bins, jitter, skip_empty, ert_wave, lod)
    sp = amnerf_stats() if stats else None
    st = load().amnerf_render(ctx, _ptr(o), _ptr(d), o.shape[0], ctypes.byref(p), _ptr(rgb), _ptr(depth),
                              _ptr(opacity), ctypes.byref(sp) if sp is not None else None)
    _check(ctx, st, "amnerf_render")
    return sp.as_dict() if sp is not None else None


def amnerf_render_debug(ctx, o, d, rgb, depth, opacity, dbg: dict, steps: int = 8, cap: int = 64,
                        t_term: float = 1e-4, bg=(0.0, 0.0, 0.0), stats: bool = True, proposal: bool = False,
                        coverage: float = 0.99, max_bins: int = 16, jitter: int = 0, skip_empty=None,
                        ert_wave: int = 0, lod: float = 0.0):
    p = _params(steps, cap, t_term, bg, proposal, coverage, max_bins, jitter, skip_empty, ert_wave, lod)
    db = amnerf_debug(*[_ptr(dbg.get(k)) for k, _ in amnerf_debug._fields_])
    sp = amnerf_stats() if stats else None
    st = load().amnerf_render_debug(ctx, _ptr(o), _ptr(d), o.shape[0], ctypes.byref(p), _ptr(rgb), _ptr(depth),
                                    _ptr(opacity), ctypes.byref(db), ctypes.byref(sp) if sp is not None else None)
    _check(ctx, st, "amnerf_render_debug")
    return sp.as_dict() if sp is not None else None


def amnerf_render_crossings(ctx, o, d, n_x, leaf, t_in, t_out, rgb, depth, opacity, steps: int = 8,
                            cap: int = 64, t_term: float = 1e-4, bg=(0.0, 0.0, 0.0), stats: bool = False,
                            jitter: int = 0, ert_wave: int = 0):
    """Render from crossings given as CUDA tensors (n_x uint8 [n]; leaf int16 and t_in,
    t_out float32 [n * maxc], maxc = cap // steps)."""
    p = _params(steps, cap, t_term, bg, jitter=jitter, ert_wave=ert_wave)
    sp = amnerf_stats() if stats else None
    st = load().amnerf_render_crossings(ctx, _ptr(o), _ptr(d), o.shape[0], ctypes.byref(p), _ptr(n_x), _ptr(leaf),
                                        _ptr(t_in), _ptr(t_out), _ptr(rgb), _ptr(depth), _ptr(opacity),
                                        ctypes.byref(sp) if sp is not None else None)
    _check(ctx, st, "amnerf_render_crossings")
    return sp.as_dict() if sp is not None else None


def amnerf_render_host(ctx, o: np.ndarray, d: np.ndarray, rgb: np.ndarray, depth: np.ndarray,
                       opacity: np.ndarray, steps: int = 8, cap: int = 64, t_term: float = 1e-4,
                       bg=(0.0, 0.0, 0.0), stats: bool = False, jitter: int = 0, skip_empty=None,
                       ert_wave: int = 0, lod: float = 0.0):
    """Render from HOST arrays (page-locked buffers make the copies asynchronous)."""
    for a in (o, d, rgb, depth, opacity):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise ValueError("host buffers must be contiguous float32")
    p = _params(steps, cap, t_term, bg, jitter=jitter, skip_empty=skip_empty, ert_wave=ert_wave, lod=lod)
    sp = amnerf_stats() if stats else None
    st = load().amnerf_render_host(ctx, _hptr(o), _hptr(d), o.shape[0], ctypes.byref(p), _hptr(rgb),
                                   _hptr(depth), _hptr(opacity), ctypes.byref(sp) if sp is not None else None)
    _check(ctx, st, "amnerf_render_host")
    return sp.as_dict() if sp is not None else None


def amnerf_group_by_leaf_static(n_x, leaf, n_rays: int, maxc: int, n_leaves: int, counts, offsets, order,
                                stream: int | None = None) -> None:
    """Grouping without any allocation (scratch in a static device array); CUDA tensors."""
    st = load().amnerf_group_by_leaf_static(_ptr(n_x), _ptr(leaf), n_rays, maxc, n_leaves, _ptr(counts),
                                            _ptr(offsets), _ptr(order), stream)
    _check(None, st, "amnerf_group_by_leaf_static")


def amnerf_set_tuning(ctx, groups: int = 0, schedule: int = SCHED_CONTIGUOUS, width_split: int = 0) -> None:
    t = amnerf_tuning(groups, schedule, width_split)
    _check(ctx, load().amnerf_set_tuning(ctx, ctypes.byref(t)), "amnerf_set_tuning")


def amnerf_get_tuning(ctx) -> tuple[int, int, int, int]:
    """(groups, schedule, largest group count the loaded network shape allows, width_split)."""
    t = amnerf_tuning()
    mg = ctypes.c_int()
    _check(ctx, load().amnerf_get_tuning(ctx, ctypes.byref(t), ctypes.byref(mg)), "amnerf_get_tuning")
    return t.groups, t.schedule, mg.value, t.width_split


def amnerf_autotune(ctx, o, d, rgb, depth, opacity, steps: int = 8, cap: int = 64, t_term: float = 1e-4,
                    bg=(0.0, 0.0, 0.0), reps: int = 3, lod: float = 0.0) -> tuple[int, int, int, float]:
    """Time every launch configuration on this batch; returns (groups, schedule,
    width_split, ms) of the fastest, which the context keeps."""
    p = _params(steps, cap, t_term, bg, lod=lod)
    best = amnerf_tuning()
    ms = ctypes.c_float()
    st = load().amnerf_autotune(ctx, _ptr(o), _ptr(d), o.shape[0], ctypes.byref(p), _ptr(rgb), _ptr(depth),
                                _ptr(opacity), reps, ctypes.byref(best), ctypes.byref(ms))
    _check(ctx, st, "amnerf_autotune")
    return best.groups, best.schedule, best.width_split, ms.value


def amnerf_proposal_set(ctx, params: np.ndarray, adam_m=None, adam_v=None, step: int = 0) -> None:
    P = np.ascontiguousarray(params, np.float32)
    assert P.size == PROPOSAL_PARAMS
    m = None if adam_m is None else np.ascontiguousarray(adam_m, np.float32)
    v = None if adam_v is None else np.ascontiguousarray(adam_v, np.float32)
    st = load().amnerf_proposal_set(ctx, _hptr(P), _hptr(m) if m is not None else None,
                                    _hptr(v) if v is not None else None, step)
    _check(ctx, st, "amnerf_proposal_set")


def amnerf_proposal_get(ctx):
    """(params, adam_m, adam_v, step) as float32 numpy arrays."""
    P = np.zeros(PROPOSAL_PARAMS, np.float32); m = np.zeros_like(P); v = np.zeros_like(P)
    step = ctypes.c_int()
    _check(ctx, load().amnerf_proposal_get(ctx, _hptr(P), _hptr(m), _hptr(v), ctypes.byref(step)),
           "amnerf_proposal_get")
    return P, m, v, step.value


def amnerf_proposal_targets(ctx, o, d, rgb, depth, opacity, targets, root, steps: int = 8, cap: int = 64,
                            t_term: float = 1e-4, bg=(0.0, 0.0, 0.0)) -> None:
    p = _params(steps, cap, t_term, bg)
    st = load().amnerf_proposal_targets(ctx, _ptr(o), _ptr(d), o.shape[0], ctypes.byref(p), _ptr(rgb), _ptr(depth),
                                        _ptr(opacity), _ptr(targets), _ptr(root))
    _check(ctx, st, "amnerf_proposal_targets")


def amnerf_proposal_train(ctx, o, d, root, targets, steps: int, batch: int, lr: float = 1e-3,
                          seed: int = 1) -> np.ndarray:
    losses = np.zeros(max(steps, 1), np.float32)
    st = load().amnerf_proposal_train(ctx, _ptr(o), _ptr(d), _ptr(root), _ptr(targets), o.shape[0], steps, batch,
                                      lr, seed, _hptr(losses))
    _check(ctx, st, "amnerf_proposal_train")
    return losses[:steps]


def amnerf_proposal_grad(ctx, o, d, root, targets):
    g = np.zeros(PROPOSAL_PARAMS, np.float32)
    loss = np.zeros(1, np.float32)
    st = load().amnerf_proposal_grad(ctx, _ptr(o), _ptr(d), _ptr(root), _ptr(targets), o.shape[0], _hptr(g),
                                     _hptr(loss))
    _check(ctx, st, "amnerf_proposal_grad")
    return float(loss[0]), g


def amnerf_proposal_predict(ctx, o, d, probs, mask, fallback, coverage: float = 0.99, max_bins: int = 16) -> None:
    st = load().amnerf_proposal_predict(ctx, _ptr(o), _ptr(d), o.shape[0], coverage, max_bins, _ptr(probs),
                                        _ptr(mask), _ptr(fallback))
    _check(ctx, st, "amnerf_proposal_predict")


def amnerf_selftest_wait(ctx, cycles: int) -> int:
    """Run the bounded-wait self-test; returns the status code (E_TIMEOUT expected)."""
    return load().amnerf_selftest_wait(ctx, cycles)


def amnerf_sync(ctx) -> None:
    _check(ctx, load().amnerf_sync(ctx), "amnerf_sync")


# --------------------------------------------------------------------------------------
# convenience wrapper
# --------------------------------------------------------------------------------------

@dataclass
class Renderer:
    """Owns one context; all methods call the entry points above."""

    device: int = 0

    def __post_init__(self):
        import torch
        self._torch = torch
        torch.cuda.set_device(self.device)
        self.ctx = amnerf_create(self.device, torch.cuda.current_stream(self.device).cuda_stream)
        self.n_leaves = 0
        self.n_nets = 0

    def close(self):
        if getattr(self, "ctx", None) is not None:
            amnerf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def build_tree(self, grid, max_depth, leaf_mass_frac=0.0, bbox=(-1.0, -1.0, -1.0, 1.0, 1.0, 1.0)) -> int:
        self.n_leaves = amnerf_build_tree(self.ctx, grid, max_depth, leaf_mass_frac, bbox)
        return self.n_leaves

    def tree(self) -> list:
        return amnerf_get_tree(self.ctx)

    def leaf_cells(self) -> np.ndarray:
        nodes = [n for n in self.tree() if n.axis < 0]
        nodes.sort(key=lambda n: n.leaf_id)
        return np.array([list(n.cell_lo) + list(n.cell_hi) for n in nodes], dtype=np.int64)

    def network_cells(self) -> np.ndarray:
        """Cell ranges of every node in network order: the leaves by leaf id, then the
        inner nodes in preorder (one network per node, adaptive hierarchical sampling)."""
        tree = self.tree()
        leaves = sorted((n for n in tree if n.axis < 0), key=lambda n: n.leaf_id)
        inner = [n for n in tree if n.axis >= 0]
        return np.array([list(n.cell_lo) + list(n.cell_hi) for n in leaves + inner], dtype=np.int64)

    def load_mlps(self, weights, width, hidden, lx, ld, prec="fp32", act_max=None) -> None:
        """prec: "fp32", "bf16", "fp8" (per-row activation scales) or, with act_max
        (see calibrate_fp8), E4M3 with static per-leaf, per-layer activation scales.
        One network per leaf, or per node when the weights hold that many."""
        per = (3 + 6 * lx + 3 + 6 * ld) * width + width + (hidden - 1) * (width * width + width) + 4 * width + 4
        self.n_nets = int(np.asarray(weights).size // per)
        if act_max is not None:
            amnerf_load_mlps_fp8_static(self.ctx, weights, self.n_nets, width, hidden, lx, ld, act_max)
        else:
            amnerf_load_mlps(self.ctx, weights, self.n_nets, width, hidden, lx, ld, PRECISIONS.get(prec, prec))

    def calibrate_fp8(self, o, d, hidden, steps=8, cap=64, t_term=1e-4, lod=0.0):
        torch = self._torch
        amnerf_set_stream(self.ctx, torch.cuda.current_stream(o.device).cuda_stream)
        return amnerf_calibrate_fp8(self.ctx, o, d, self.n_nets, hidden, steps=steps, cap=cap, t_term=t_term,
                                    lod=lod)

    def render(self, o, d, steps=8, cap=64, t_term=1e-4, bg=(0.0, 0.0, 0.0), stats=False, out=None,
               proposal=False, coverage=0.99, max_bins=16, jitter=0, skip_empty=None, ert_wave=0, lod=0.0):
        torch = self._torch
        n = o.shape[0]
        if out is None:
            out = (torch.empty((n, 3), device=o.device, dtype=torch.float32),
                   torch.empty((n,), device=o.device, dtype=torch.float32),
                   torch.empty((n,), device=o.device, dtype=torch.float32))
        amnerf_set_stream(self.ctx, torch.cuda.current_stream(o.device).cuda_stream)
        s = amnerf_render(self.ctx, o, d, *out, steps=steps, cap=cap, t_term=t_term, bg=bg, stats=stats,
                          proposal=proposal, coverage=coverage, max_bins=max_bins, jitter=jitter,
                          skip_empty=skip_empty, ert_wave=ert_wave, lod=lod)
        return (*out, s) if stats else out

    def render_debug(self, o, d, steps=8, cap=64, t_term=1e-4, bg=(0.0, 0.0, 0.0), proposal=False, coverage=0.99,
                     max_bins=16, jitter=0, skip_empty=None, ert_wave=0, lod=0.0):
        torch = self._torch
        n = o.shape[0]
        maxc = cap // steps
        dev = o.device
        dbg = {
            "n_x": torch.zeros(n, dtype=torch.uint8, device=dev),
            "leaf": torch.zeros(n * maxc, dtype=torch.int16, device=dev),
            "t_in": torch.zeros(n * maxc, dtype=torch.float32, device=dev),
            "t_out": torch.zeros(n * maxc, dtype=torch.float32, device=dev),
            "counts": torch.zeros(max(self.n_nets, 1), dtype=torch.int32, device=dev),
            "offsets": torch.zeros(self.n_nets + 1, dtype=torch.int32, device=dev),
            "order": torch.zeros(max(n * maxc, 1), dtype=torch.int32, device=dev),
            "slot_out": torch.zeros(max(n * cap * 4, 1), dtype=torch.float32, device=dev),
        }
        if proposal:
            dbg["prop_mask"] = torch.zeros(max(n, 1), dtype=torch.int64, device=dev)
            dbg["prop_fallback"] = torch.zeros(max(n, 1), dtype=torch.uint8, device=dev)
            dbg["prop_q"] = torch.full((max(n, 1) * 65,), float("nan"), dtype=torch.float32, device=dev)
        rgb = torch.empty((n, 3), device=dev, dtype=torch.float32)
        depth = torch.empty((n,), device=dev, dtype=torch.float32)
        opac = torch.empty((n,), device=dev, dtype=torch.float32)
        amnerf_set_stream(self.ctx, torch.cuda.current_stream(dev).cuda_stream)
        s = amnerf_render_debug(self.ctx, o, d, rgb, depth, opac, dbg, steps=steps, cap=cap, t_term=t_term, bg=bg,
                                proposal=proposal, coverage=coverage, max_bins=max_bins, jitter=jitter,
                                skip_empty=skip_empty, ert_wave=ert_wave, lod=lod)
        host = {k: v.cpu().numpy() for k, v in dbg.items()}
        host["leaf"] = host["leaf"].view(np.uint16).astype(np.int64).reshape(n, maxc)
        host["t_in"] = host["t_in"].reshape(n, maxc)
        host["t_out"] = host["t_out"].reshape(n, maxc)
        host["order"] = host["order"].view(np.uint32).astype(np.int64)
        host["counts"] = host["counts"].view(np.uint32).astype(np.int64)[: self.n_nets]
        host["offsets"] = host["offsets"].view(np.uint32).astype(np.int64)
        host["slot_out"] = host["slot_out"][: n * cap * 4].reshape(n, cap, 4)
        if proposal:
            host["prop_mask"] = host["prop_mask"][:n].view(np.uint64)
            host["prop_fallback"] = host["prop_fallback"][:n]
            host["prop_q"] = host["prop_q"][: n * 65].reshape(n, 65)
        return rgb.cpu().numpy(), depth.cpu().numpy(), opac.cpu().numpy(), host, s

    def sync(self):
        amnerf_sync(self.ctx)

    def capture(self, o, d, steps=8, cap=64, t_term=1e-4, bg=(0.0, 0.0, 0.0)):
        """Capture one render of (o, d) in a CUDA graph; returns (graph, (rgb, depth, opacity)).
        Replaying the graph re-renders whatever o and d hold.  Renders once first so
        that the library's scratch is allocated outside the capture."""
        torch = self._torch
        out = self.render(o, d, steps, cap, t_term, bg)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(o.device)
        side.wait_stream(torch.cuda.current_stream(o.device))
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
                amnerf_set_stream(self.ctx, side.cuda_stream)
                amnerf_render(self.ctx, o, d, *out, steps=steps, cap=cap, t_term=t_term, bg=bg)
        torch.cuda.current_stream(o.device).wait_stream(side)
        amnerf_set_stream(self.ctx, torch.cuda.current_stream(o.device).cuda_stream)
        return g, out
