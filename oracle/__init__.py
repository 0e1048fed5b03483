"""CPU oracle of the Adaptive Multi-NeRF rendering hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline leg
of the benchmark are the only users.  The product path (the CUDA library and its
Python binding) never imports this package, and this package never imports the
product.  The arithmetic lives in ``amnerf_oracle.c`` (plain C, FP64 definition
plus an FP32 mode in the GPU's operation order); ``build()`` compiles it with gcc.

Parity status per function (what pins it is in tests/test_oracle_pins.py):
  build_tree  pinned: tiling invariants, brute-force median over k, hand-derived
              G=4 fixture, leaf rule.
  traverse    pinned: point-in-box brute force along the ray, sorted-all-leaves form,
              contiguity, union = root interval.
  samples     pinned: every sample inside its leaf box; sum of deltas = hit length.
  group       pinned: permutation, histogram, exclusive scan, stable order.
  encode      pinned: exact values at dyadic points, double-angle identities.
  mlp_eval    pinned: numpy float64 matmul chain; zero-weight closed form.
  render      pinned: constant-density closed form, sum(w) + T = 1, midpoint-rule
              depth limit, early termination.
Proposal sampler (pins in tests/test_oracle_proposal.py):
  prop_predict    pinned: numpy float64 matmul chain with a library softmax.
  prop_loss_grad  pinned: central finite differences; entropy closed form at q = p.
  prop_adam       pinned: first step from zero moments moves by lr against sign(g).
  prop_select     pinned: hand-worked cases (ties, background, fallback); binary32
                  mode: absorption of masses below half an ulp of the sum.
  prop_predict(bf16=True)  pinned: bf16_round against hand-worked ties and a library
                  bfloat16 conversion; the same numpy chain on rounded operands.
  bin_indices     pinned: hand-worked rays with samples on, just below and just above
                  the bin edges (both modes); brute-force edge counting in numpy.
  masked render   pinned: all-bins mask = plain render; kept crossings by brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amnerf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

F32 = np.float32
F64 = np.float64
I32 = np.int32
I64 = np.int64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            V, I, L, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            _lib.or_build_tree.argtypes = [V, I, V, I, D, I, V, V, V, V, V, V]
            _lib.or_traverse.argtypes = [V, V, V, I, V, V, L, I, I, I, V, V, V, V, D]
            U = ctypes.c_uint64
            _lib.or_samples.argtypes = [V, V, L, V, V, V, I, I, I, I, U, V, V, V]
            _lib.or_group.argtypes = [V, V, L, I, I, I, V, V, V]
            _lib.or_splitmix64_mix.argtypes = [U]
            _lib.or_splitmix64_mix.restype = U
            _lib.or_jitter_fraction.argtypes = [U, V, V, I, I, I]
            _lib.or_jitter_fraction.restype = ctypes.c_float
            _lib.or_encode.argtypes = [V, I, I, V]
            _lib.or_encode.restype = None
            _lib.or_mlp_eval.argtypes = [V, I, I, I, I, V, V, L, I, V, V]
            _lib.or_mlp_input_absmax.argtypes = [V, I, I, I, I, V, V, L, V]
            _lib.or_render.argtypes = [V, V, V, I, V, I, I, I, I, V, V, L, I, I, D, V, I, U, V, I, V, D, I,
                                       V, V, V, V, V, V, V, V, V, V, V, V, I, D]
            _lib.or_f16_round_n.argtypes = [V, L, V]
            _lib.or_traverse_skip.argtypes = [V, V, V, I, V, V, L, I, I, I, I, U, V, I, V, D, V, V, V, V, D]
            _lib.or_prop_predict.argtypes = [V, V, V, V, L, V, I]
            _lib.or_bin_indices.argtypes = [I, V, V, V, L, V]
            _lib.or_bf16_round.argtypes = [D]
            _lib.or_bf16_round.restype = D
            _lib.or_bf16_round_n.argtypes = [V, L, V]
            _lib.or_prop_loss_grad.argtypes = [V, V, V, V, V, L, V, V]
            _lib.or_prop_adam.argtypes = [V, V, V, V, I, I, D, D, D, D]
            _lib.or_prop_select.argtypes = [V, L, D, I, V, V, I]
    return _lib


class Tree:
    """Flat preorder node arrays (see amnerf_oracle.c for the field meaning)."""

    def __init__(self, box, cells, info, split, mass, n_leaves):
        self.box, self.cells, self.info, self.split, self.mass = box, cells, info, split, mass
        self.n_leaves = int(n_leaves)

    @property
    def n_nodes(self) -> int:
        return len(self.split)

    def leaves(self) -> np.ndarray:
        """Node indices of the leaves, ordered by leaf id."""
        idx = np.nonzero(self.info[:, 0] < 0)[0]
        return idx[np.argsort(self.info[idx, 3])]

    def leaf_cells(self) -> np.ndarray:
        return self.cells[self.leaves()]

    def network_nodes(self) -> np.ndarray:
        """Node indices in network order: the leaves by leaf id, then the inner nodes
        in preorder (the networks of adaptive hierarchical sampling)."""
        inner = np.nonzero(self.info[:, 0] >= 0)[0]
        return np.concatenate([self.leaves(), inner])

    def network_cells(self) -> np.ndarray:
        return self.cells[self.network_nodes()]


def build_tree(grid: np.ndarray, max_depth: int, leaf_frac: float = 0.0,
               bbox=(-1.0, -1.0, -1.0, 1.0, 1.0, 1.0)) -> Tree:
    grid = np.ascontiguousarray(grid, dtype=F32)
    G = grid.shape[0]
    cap = 2 ** (max_depth + 1) + 1
    box = np.zeros((cap, 6), F32); cells = np.zeros((cap, 6), I32); info = np.zeros((cap, 6), I32)
    split = np.zeros(cap, F32); mass = np.zeros(cap, F64); nl = np.zeros(1, I32)
    bb = np.asarray(bbox, dtype=F64)
    n = lib().or_build_tree(_p(grid), G, _p(bb), max_depth, float(leaf_frac), cap,
                            _p(box), _p(cells), _p(info), _p(split), _p(mass), _p(nl))
    if n <= 0:
        raise RuntimeError("oracle tree build failed")
    return Tree(box[:n].copy(), cells[:n].copy(), info[:n].copy(), split[:n].copy(), mass[:n].copy(), nl[0])


def make_tree(box, info, split) -> Tree:
    """Tree from hand-written arrays (used by pin tests)."""
    box = np.ascontiguousarray(box, F32); info = np.ascontiguousarray(info, I32)
    split = np.ascontiguousarray(split, F32)
    n = len(split)
    return Tree(box, np.zeros((n, 6), I32), info, split, np.zeros(n, F64), int((info[:, 0] < 0).sum()))


BBOX = (-1.0, -1.0, -1.0, 1.0, 1.0, 1.0)


def traverse(tree: Tree, o, d, maxc: int, mode: int = 0, method: int = 0, skip=None, lod: float = 0.0):
    """Per ray: crossing count, network ids, entries, exits (ray-major, stride maxc).
    skip = (grid, threshold, steps, jitter): empty-space skipping -- a crossing is kept
    only when one of its samples (placed as its index among the kept crossings) lies
    in a grid cell of density > threshold.
    lod > 0: adaptive hierarchical sampling -- an inner node is descended only while
    its extent along its split axis exceeds lod x the ray's entry distance into it,
    else it is one crossing with its own network (ids: leaves 0..L-1 by leaf id, then
    inner nodes in preorder, L + rank; see Tree.network_nodes)."""
    o = np.ascontiguousarray(o, F32); d = np.ascontiguousarray(d, F32)
    n = len(o)
    nx = np.zeros(n, I32); leaf = np.full((n, maxc), -1, I32)
    tin = np.zeros((n, maxc), F64); tout = np.zeros((n, maxc), F64)
    if skip is not None:
        grid, thr, steps, jitter = skip
        grid = np.ascontiguousarray(grid, F32)
        bb = np.asarray(BBOX, F64)
        rc = lib().or_traverse_skip(_p(tree.box), _p(tree.info), _p(tree.split), tree.n_nodes, _p(o), _p(d), n,
                                    maxc, mode, method, steps, int(jitter), _p(grid), grid.shape[0], _p(bb),
                                    float(thr), _p(nx), _p(leaf), _p(tin), _p(tout), float(lod))
        if rc != 0:
            raise RuntimeError("oracle traversal failed")
        return nx, leaf, tin, tout
    rc = lib().or_traverse(_p(tree.box), _p(tree.info), _p(tree.split), tree.n_nodes, _p(o), _p(d), n,
                           maxc, mode, method, _p(nx), _p(leaf), _p(tin), _p(tout), float(lod))
    if rc != 0:
        raise RuntimeError("oracle traversal failed")
    return nx, leaf, tin, tout


def samples(o, d, nx, tin, tout, maxc: int, steps: int, cap: int, mode: int = 0, jitter: int = 0):
    """Slot arrays t, delta (n, cap) and x (n, cap, 3); unused slots are zero.
    jitter: 0 = stratum midpoints, else the seed of the stratified jitter."""
    o = np.ascontiguousarray(o, F32); d = np.ascontiguousarray(d, F32)
    n = len(o)
    t = np.zeros((n, cap), F64); dl = np.zeros((n, cap), F64); x = np.zeros((n, cap, 3), F64)
    lib().or_samples(_p(o), _p(d), n, _p(np.ascontiguousarray(nx, I32)), _p(np.ascontiguousarray(tin, F64)),
                     _p(np.ascontiguousarray(tout, F64)), maxc, steps, cap, mode, int(jitter), _p(t), _p(dl), _p(x))
    return t, dl, x


def splitmix64_mix(z: int) -> int:
    """The splitmix64 finaliser of the stratified-jitter generator."""
    return int(lib().or_splitmix64_mix(z & ((1 << 64) - 1)))


def jitter_fraction(seed: int, o, d, k: int, steps: int, j: int) -> float:
    """Fraction u of its stratum at which sample j of crossing k of ray (o, d) sits."""
    o = np.ascontiguousarray(o, F32); d = np.ascontiguousarray(d, F32)
    return float(lib().or_jitter_fraction(seed, _p(o), _p(d), k, steps, j))


def group(nx, leaf, maxc: int, steps: int, n_leaves: int):
    nx = np.ascontiguousarray(nx, I32); leaf = np.ascontiguousarray(leaf, I32)
    n = len(nx)
    counts = np.zeros(n_leaves, I64); offsets = np.zeros(n_leaves + 1, I64)
    order = np.zeros(int(nx.sum()), I64)
    rc = lib().or_group(_p(nx), _p(leaf), n, maxc, steps, n_leaves, _p(counts), _p(offsets), _p(order))
    if rc != 0:
        raise RuntimeError("oracle grouping failed")
    return counts, offsets, order


def encode(p, L: int, mode: int = 0) -> np.ndarray:
    p = np.ascontiguousarray(p, F64).reshape(3)
    out = np.zeros(3 + 6 * L, F64)
    lib().or_encode(_p(p), L, mode, _p(out))
    return out


def mlp_eval(params_leaf, width: int, hidden: int, lx: int, ld: int, x, d, mode: int = 0):
    P = np.ascontiguousarray(params_leaf, F32)
    x = np.ascontiguousarray(x, F64).reshape(-1, 3); d = np.ascontiguousarray(d, F64).reshape(-1, 3)
    n = len(x)
    out = np.zeros((n, 4), F64); raw = np.zeros((n, 4), F64)
    rc = lib().or_mlp_eval(_p(P), width, hidden, lx, ld, _p(x), _p(d), n, mode, _p(out), _p(raw))
    if rc != 0:
        raise RuntimeError("oracle mlp failed")
    return out, raw


def mlp_input_absmax(params_leaf, width: int, hidden: int, lx: int, ld: int, x, d) -> np.ndarray:
    """Largest |input| of every hidden layer (layer 0: the encoding) over the samples
    x, d of one leaf's network, in FP64."""
    P = np.ascontiguousarray(params_leaf, F32)
    x = np.ascontiguousarray(x, F64).reshape(-1, 3); d = np.ascontiguousarray(d, F64).reshape(-1, 3)
    out = np.zeros(hidden, F64)
    if lib().or_mlp_input_absmax(_p(P), width, hidden, lx, ld, _p(x), _p(d), len(x), _p(out)) != 0:
        raise RuntimeError("oracle mlp failed")
    return out


def render(tree: Tree, params, width: int, hidden: int, lx: int, ld: int, o, d, steps: int, cap: int,
           t_term: float = 1e-4, bg=(0.0, 0.0, 0.0), mode: int = 0, threads: int = 1, full: bool = False,
           mask=None, fallback=None, bins: bool = False, jitter: int = 0, skip=None, slot_fp16: bool = False,
           lod: float = 0.0):
    """Full render of every ray; returns a dict of float64 / int32 arrays.
    slot_fp16 (FP64 mode): each sample's sigma and rgb rounded to binary16 (sigma
    limited to 65504) before compositing, to measure a half-precision store alone.
    lod > 0: adaptive hierarchical sampling (see traverse); params then hold one network
    per node in network order (Tree.network_nodes).
    jitter: 0 = samples at stratum midpoints, else the seed of the stratified jitter.
    skip = (grid, threshold): empty-space skipping over the guidance grid (see traverse).
    mask/fallback (proposal sampler): per-ray kept-bin masks and fallback flags;
    bins: also return the compositing weight per depth bin (n, 65)."""
    params = np.ascontiguousarray(params, F32)
    o = np.ascontiguousarray(o, F32); d = np.ascontiguousarray(d, F32)
    n = len(o)
    res = {
        "rgb": np.zeros((n, 3), F64), "depth": np.zeros(n, F64), "opacity": np.zeros(n, F64),
        "n_gen": np.zeros(n, I32), "n_eval": np.zeros(n, I32), "ert_margin": np.zeros(n, F64),
        "t_final": np.zeros(n, F64),
    }
    so = sw = None
    if full:
        so = np.zeros((n, cap, 4), F64); sw = np.zeros((n, cap), F64)
        res["slot_out"] = so; res["slot_w"] = sw
    mk = fb = None
    if mask is not None:
        mk = np.ascontiguousarray(mask, np.uint64)
        fb = np.ascontiguousarray(fallback, I32)
    if bins:
        res["bins"] = np.zeros((n, 65), F64)
    bgv = np.asarray(bg, F64)
    og, oG, othr = None, 0, 0.0
    if skip is not None:
        og = np.ascontiguousarray(skip[0], F32); oG = og.shape[0]; othr = float(skip[1])
    bb = np.asarray(BBOX, F64)
    rc = lib().or_render(_p(tree.box), _p(tree.info), _p(tree.split), tree.n_nodes, _p(params), width, hidden,
                         lx, ld, _p(o), _p(d), n, steps, cap, float(t_term), _p(bgv), mode, int(jitter),
                         _p(og) if og is not None else None, oG, _p(bb), othr, threads,
                         _p(res["rgb"]), _p(res["depth"]), _p(res["opacity"]), _p(res["n_gen"]),
                         _p(res["n_eval"]), _p(res["ert_margin"]),
                         _p(so) if so is not None else None, _p(sw) if sw is not None else None,
                         _p(res["t_final"]), _p(mk) if mk is not None else None, _p(fb) if fb is not None else None,
                         _p(res["bins"]) if bins else None, int(slot_fp16), float(lod))
    if rc != 0:
        raise RuntimeError("oracle render failed")
    return res


def f16_round(x) -> np.ndarray:
    """x rounded to the nearest IEEE binary16 value (ties to even), as float64."""
    a = np.ascontiguousarray(x, F64)
    out = np.empty_like(a)
    lib().or_f16_round_n(_p(a), a.size, _p(out))
    return out


# ---------------------------------------------------------------------------------
# proposal sampler (not in the paper)
# ---------------------------------------------------------------------------------

PROP_NPARAM = 32 * 90 + 32 + 32 * 32 + 32 + 65 * 32 + 65


def root_interval(tree: Tree, o, d, mode: int = 0):
    """(t0, t1, hit) of every ray against the root box (node 0)."""
    box = tree.box[0:1]
    info = np.array([[-1, -1, -1, 0, 1, 0]], I32)
    split = np.zeros(1, F32)
    nx, leaf, tin, tout = traverse(make_tree(box, info, split), o, d, 1, mode=mode)
    return tin[:, 0], tout[:, 0], nx > 0


def prop_predict(P, o, d, t0, bf16: bool = False):
    """Softmax outputs (n, 65).  bf16=True rounds every operand of the three affine
    maps (inputs, weights, biases, hidden activations) to bfloat16 and accumulates
    in double: the operand rounding of a BF16 tensor-core evaluation."""
    P = np.ascontiguousarray(P, F64); o = np.ascontiguousarray(o, F32); d = np.ascontiguousarray(d, F32)
    t0 = np.ascontiguousarray(t0, F64)
    q = np.zeros((len(o), 65), F64)
    lib().or_prop_predict(_p(P), _p(o), _p(d), _p(t0), len(o), _p(q), int(bf16))
    return q


def bf16_round(x):
    """x (a number or an array) rounded to the nearest bfloat16 value (ties to even)."""
    if np.ndim(x) == 0:
        return float(lib().or_bf16_round(float(x)))
    a = np.ascontiguousarray(x, F64)
    out = np.empty_like(a)
    lib().or_bf16_round_n(_p(a), a.size, _p(out))
    return out


def bin_indices(t0, t1, t, mode: int = 0) -> np.ndarray:
    """Depth bin of samples at t on rays with root interval [t0, t1] (the training
    targets' binning): floor((t - t0) / w), w = (t1 - t0) / 64, clamped to [0, 63],
    in the mode's precision."""
    t0 = np.ascontiguousarray(t0, F64); t1 = np.ascontiguousarray(t1, F64); t = np.ascontiguousarray(t, F64)
    out = np.zeros(len(t), I32)
    lib().or_bin_indices(int(mode), _p(t0), _p(t1), _p(t), len(t), _p(out))
    return out


def prop_loss_grad(P, o, d, t0, targets):
    P = np.ascontiguousarray(P, F64); o = np.ascontiguousarray(o, F32); d = np.ascontiguousarray(d, F32)
    t0 = np.ascontiguousarray(t0, F64); tg = np.ascontiguousarray(targets, F64)
    loss = np.zeros(1, F64); g = np.zeros(PROP_NPARAM, F64)
    lib().or_prop_loss_grad(_p(P), _p(o), _p(d), _p(t0), _p(tg), len(o), _p(loss), _p(g))
    return float(loss[0]), g


def prop_adam(P, g, m, v, t: int, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """In-place Adam step on float64 arrays P, m, v."""
    for a in (P, m, v):
        assert a.dtype == F64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, F64)
    lib().or_prop_adam(_p(P), _p(g), _p(m), _p(v), len(P), t, lr, b1, b2, eps)


def prop_select(q, coverage: float = 0.99, max_bins: int = 16, single: bool = False):
    """Kept depth bins per ray (mask) and fallback flags.  single=True keeps the
    running sum in binary32 (q is rounded to float32 first), as the GPU kernels do."""
    if single:
        q = np.asarray(q, F32)
    q = np.ascontiguousarray(q, F64)
    mask = np.zeros(len(q), np.uint64); fb = np.zeros(len(q), I32)
    lib().or_prop_select(_p(q), len(q), coverage, max_bins, _p(mask), _p(fb), int(single))
    return mask, fb
