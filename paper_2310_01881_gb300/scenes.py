"""Seeded synthetic inputs for the Adaptive Multi-NeRF rendering hot path.

This module builds the *inputs* of the method and nothing else: guidance density
grids (the stand-in for the uniformly sampled, normalised point cloud of Sec. 3.3),
pinhole camera rays, and Xavier-initialised per-leaf MLP weights.  It holds none of
the method's arithmetic (no subdivision, traversal, sampling, encoding, network
evaluation or compositing), so that both the CPU oracle and the CUDA library can
consume its arrays without sharing any code of the method.

The paper's own scenes (Lego, Material, Ueno, Dragon, House1/2; Sec. 4.1) are
datasets that are not available; the scenes here stand in for their size and
imbalance: sums of Gaussians and thin spherical shells inside [-1, 1]^3.

Grid layout: float32 array of shape (G, G, G) indexed [z, y, x] (x fastest), value at
the cell centre c_i = -1 + (i + 1/2) * 2 / G.
Ray layout: float32 arrays o, d of shape (n, 3), row-major, d of unit length (normalised
in float64, then rounded to float32).
Weight layout (float32, flat): leaf-major; per leaf, for each hidden layer l the matrix
W_l (rows = outputs, row-major) followed by its bias b_l, then the head W_o (4 x width)
and b_o (4).  The input width is (3 + 6 Lx) + (3 + 6 Ld).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Scene", "RenderConfig", "CONFIGS", "scene_for", "density_grid", "camera_rays",
    "view_rays", "params_per_leaf", "mlp_input_width", "leaf_mean_density",
    "xavier_weights", "ray_subset", "proposal_init", "PROPOSAL_PARAMS", "zipf_crossings",
]


@dataclasses.dataclass
class Scene:
    """Analytic density field: Gaussians (centre, 3x3 inverse covariance, peak) and
    shells (centre, radius, width, peak) with a Gaussian radial profile."""

    centres: np.ndarray          # (g, 3)
    inv_cov: np.ndarray          # (g, 3, 3)
    extent: np.ndarray           # (g,) window half-width (6 x largest axis std)
    peak: np.ndarray             # (g,)
    shell_c: np.ndarray          # (s, 3)
    shell_r: np.ndarray          # (s,)
    shell_w: np.ndarray          # (s,)
    shell_peak: np.ndarray       # (s,)


@dataclasses.dataclass(frozen=True)
class RenderConfig:
    """One synthetic workload: scene recipe, grid, tree rule, network shape, image."""

    name: str
    scene: str                   # "c1" | "c2" | "c4"
    G: int                       # guidance grid resolution
    max_depth: int               # tree depth limit
    leaf_mass_frac: float        # leaf if mass <= frac * total (0 = no mass rule)
    width: int                   # hidden width of every leaf MLP
    hidden: int                  # number of hidden ReLU layers
    lx: int                      # xyz encoding frequencies
    ld: int                      # direction encoding frequencies
    px_w: int
    px_h: int
    views: int
    cap: int                     # max samples per ray
    steps: int                   # samples per leaf crossing
    t_term: float                # early-termination transmittance
    fov_deg: float = 40.0
    radius: float = 3.0


CONFIGS = {
    # Plain method, tiny, FP32 (parity size).
    "c1": RenderConfig("c1", "c1", 64, 4, 0.0, 32, 2, 10, 4, 64, 64, 1, 64, 8, 1e-4),
    # Plain method, paper scale: 800x800, 8 views, <=256 leaves, 4x64 MLP, cap 192.
    "c2": RenderConfig("c2", "c2", 128, 8, 1.0 / 256.0, 64, 4, 10, 4, 800, 800, 8, 192, 8, 1e-4),
    # Highly unbalanced scene, <=4096 leaves, 1920x1080 x 16 views.
    "c4": RenderConfig("c4", "c4", 256, 12, 0.0, 64, 4, 10, 4, 1920, 1080, 16, 192, 8, 1e-4),
}


def _quat_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (Shoemake's subgroup algorithm for unit quaternions)."""
    u1, u2, u3 = rng.uniform(0.0, 1.0, 3)
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    x, y = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    z, w = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def scene_for(kind: str, seed: int) -> Scene:
    """Build the seeded density recipe of one workload family.

    c1: 4 isotropic Gaussians, centres U[-0.6,0.6]^3, std U[0.1,0.3], peak 50.
    c2: 8 anisotropic Gaussians (axis stds U[0.05,0.3], uniform random rotation,
        centres U[-0.6,0.6]^3, peak 50) plus a shell of radius 0.7, width 0.02,
        peak 200 centred at the origin.
    c4: 64 isotropic Gaussians (ln std ~ N(ln 0.05, 0.7) clipped to [0.005, 0.5],
        centres U[-0.9,0.9]^3, peak 50) plus 3 shells (centres U[-0.3,0.3]^3, radii
        U[0.2,0.6], width 0.01, peak 200).
    """
    rng = np.random.default_rng([seed, 0x5CE7E])
    cs, ics, ext, pk = [], [], [], []
    sc, sr, sw, sp = [], [], [], []
    if kind == "c1":
        for _ in range(4):
            c = rng.uniform(-0.6, 0.6, 3)
            s = rng.uniform(0.1, 0.3)
            cs.append(c); ics.append(np.eye(3) / (s * s)); ext.append(6 * s); pk.append(50.0)
    elif kind == "c2":
        for _ in range(8):
            c = rng.uniform(-0.6, 0.6, 3)
            s = rng.uniform(0.05, 0.3, 3)
            R = _quat_rotation(rng)
            cs.append(c); ics.append(R @ np.diag(1.0 / (s * s)) @ R.T); ext.append(6 * s.max()); pk.append(50.0)
        sc.append(np.zeros(3)); sr.append(0.7); sw.append(0.02); sp.append(200.0)
    elif kind == "c4":
        for _ in range(64):
            c = rng.uniform(-0.9, 0.9, 3)
            s = float(np.clip(math.exp(rng.normal(math.log(0.05), 0.7)), 0.005, 0.5))
            cs.append(c); ics.append(np.eye(3) / (s * s)); ext.append(6 * s); pk.append(50.0)
        for _ in range(3):
            sc.append(rng.uniform(-0.3, 0.3, 3)); sr.append(rng.uniform(0.2, 0.6)); sw.append(0.01); sp.append(200.0)
    else:
        raise ValueError(f"unknown scene kind {kind!r}")
    f = lambda a, shape: np.asarray(a, dtype=np.float64).reshape(shape)
    return Scene(f(cs, (-1, 3)), f(ics, (-1, 3, 3)), f(ext, (-1,)), f(pk, (-1,)),
                 f(sc, (-1, 3)), f(sr, (-1,)), f(sw, (-1,)), f(sp, (-1,)))


def density_grid(scene: Scene, G: int) -> np.ndarray:
    """Sample the scene density at the G^3 cell centres of [-1,1]^3 (float64 sums,
    float32 result).  Each Gaussian contributes inside the axis-aligned window of
    half-width 6 x its largest std around its centre, each shell inside the window
    of half-width radius + 6 x width (contributions outside are below 1.6e-8 of
    their peak and are left out)."""
    centres = -1.0 + (np.arange(G) + 0.5) * (2.0 / G)
    grid = np.zeros((G, G, G), dtype=np.float64)

    def window(c, half):
        lo = np.searchsorted(centres, c - half, side="left")
        hi = np.searchsorted(centres, c + half, side="right")
        return lo, hi

    for c, ic, e, p in zip(scene.centres, scene.inv_cov, scene.extent, scene.peak):
        lo, hi = window(c, e)
        if np.any(hi <= lo):
            continue
        x = centres[lo[0]:hi[0]] - c[0]
        y = centres[lo[1]:hi[1]] - c[1]
        z = centres[lo[2]:hi[2]] - c[2]
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        q = (ic[0, 0] * X * X + ic[1, 1] * Y * Y + ic[2, 2] * Z * Z
             + 2 * ic[0, 1] * X * Y + 2 * ic[0, 2] * X * Z + 2 * ic[1, 2] * Y * Z)
        grid[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += p * np.exp(-0.5 * q)
    for c, r, w, p in zip(scene.shell_c, scene.shell_r, scene.shell_w, scene.shell_peak):
        lo, hi = window(c, r + 6 * w)
        if np.any(hi <= lo):
            continue
        x = centres[lo[0]:hi[0]] - c[0]
        y = centres[lo[1]:hi[1]] - c[1]
        z = centres[lo[2]:hi[2]] - c[2]
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        rad = np.sqrt(X * X + Y * Y + Z * Z)
        grid[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += p * np.exp(-0.5 * ((rad - r) / w) ** 2)
    return grid.astype(np.float32)


def camera_rays(direction: np.ndarray, px_w: int, px_h: int, fov_deg: float = 40.0,
                radius: float = 3.0) -> tuple[np.ndarray, np.ndarray]:
    """Pinhole camera at radius * direction looking at the origin; up = +z, or +y
    when the view direction is within 0.99 of +-z; vertical field of view fov_deg;
    one ray through each pixel centre, rows top to bottom.  Built in float64,
    rounded to float32 (directions normalised before rounding)."""
    u = np.asarray(direction, dtype=np.float64)
    u = u / np.linalg.norm(u)
    eye = radius * u
    fwd = -u
    up = np.array([0.0, 0.0, 1.0]) if abs(u[2]) <= 0.99 else np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    tup = np.cross(right, fwd)
    th = math.tan(math.radians(fov_deg) / 2.0)
    aspect = px_w / px_h
    ii = (np.arange(px_w) + 0.5) / px_w * 2.0 - 1.0
    jj = 1.0 - (np.arange(px_h) + 0.5) / px_h * 2.0
    J, I = np.meshgrid(jj, ii, indexing="ij")
    d = (fwd[None, None, :] + (I * th * aspect)[..., None] * right[None, None, :]
         + (J * th)[..., None] * tup[None, None, :]).reshape(-1, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(eye, d.shape)
    return np.ascontiguousarray(o, dtype=np.float32), np.ascontiguousarray(d, dtype=np.float32)


def view_rays(cfg: RenderConfig, seed: int, view: int, px_w: int | None = None,
              px_h: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Rays of view `view` of workload `cfg`: camera direction uniform on the sphere
    (normalised standard normal draw from a seeded stream per (seed, view))."""
    rng = np.random.default_rng([seed, 0xCA3E7A, view])
    u = rng.normal(size=3)
    return camera_rays(u, px_w or cfg.px_w, px_h or cfg.px_h, cfg.fov_deg, cfg.radius)


def zipf_crossings(n_rays: int, maxc: int, n_nets: int, s: float, seed: int):
    """Synthetic crossing lists whose per-network counts follow a Zipf law: every ray
    has maxc crossings; each crossing's network is drawn independently with
    probability proportional to rank^-s over ranks 1..n_nets, the ranks mapped to
    network ids by a seeded permutation.  Crossing k of a ray spans
    [2 + 0.03 k, 2.03 + 0.03 k].  Returns n_x uint8 [n], leaf uint16 [n, maxc], t_in,
    t_out float32 [n, maxc] (the layout of the render's crossing list)."""
    rng = np.random.default_rng([seed, 0x21FF])
    p = np.arange(1, n_nets + 1, dtype=np.float64) ** (-float(s))
    p /= p.sum()
    perm = rng.permutation(n_nets)
    ranks = rng.choice(n_nets, size=(n_rays, maxc), p=p)
    leaf = perm[ranks].astype(np.uint16)
    k = np.arange(maxc, dtype=np.float32)
    t_in = np.broadcast_to(np.float32(2.0) + np.float32(0.03) * k, (n_rays, maxc)).astype(np.float32)
    t_out = (t_in + np.float32(0.03)).astype(np.float32)
    return np.full(n_rays, maxc, np.uint8), leaf, t_in, t_out


def ray_subset(n_total: int, k: int, seed: int) -> np.ndarray:
    """A seeded, sorted subset of k distinct ray indices out of n_total."""
    rng = np.random.default_rng([seed, 0x5AB5E7])
    return np.sort(rng.choice(n_total, size=min(k, n_total), replace=False))


def mlp_input_width(lx: int, ld: int) -> int:
    return (3 + 6 * lx) + (3 + 6 * ld)


def params_per_leaf(width: int, hidden: int, lx: int, ld: int) -> int:
    k0 = mlp_input_width(lx, ld)
    return width * k0 + width + (hidden - 1) * (width * width + width) + 4 * width + 4


def leaf_mean_density(grid: np.ndarray, leaf_cells: np.ndarray) -> np.ndarray:
    """Mean guidance density over each leaf's cell range.  leaf_cells is (L, 6) int:
    x0, y0, z0, x1, y1, z1 (half-open)."""
    out = np.empty(len(leaf_cells), dtype=np.float64)
    for i, (x0, y0, z0, x1, y1, z1) in enumerate(np.asarray(leaf_cells)):
        blk = grid[z0:z1, y0:y1, x0:x1]
        out[i] = float(blk.astype(np.float64).mean()) if blk.size else 0.0
    return out


def xavier_weights(seed: int, leaf_density: np.ndarray, width: int, hidden: int,
                   lx: int, ld: int) -> np.ndarray:
    """Xavier-uniform FP32 weights for every leaf MLP.

    W ~ U[-a, a] with a = sqrt(6 / (fan_in + fan_out)); all biases zero except the
    density-head bias b_o[0] = log(max(mean leaf density, 1e-6)).  Draws come from one
    PCG64 stream in leaf, layer, row-major order."""
    rng = np.random.default_rng([seed, 0x3EA7])
    k0 = mlp_input_width(lx, ld)
    shapes = [(width, k0)] + [(width, width)] * (hidden - 1) + [(4, width)]
    per = params_per_leaf(width, hidden, lx, ld)
    out = np.empty((len(leaf_density), per), dtype=np.float32)
    for leaf, rho in enumerate(np.asarray(leaf_density, dtype=np.float64)):
        parts = []
        for li, (fo, fi) in enumerate(shapes):
            a = math.sqrt(6.0 / (fi + fo))
            W = rng.uniform(-a, a, size=(fo, fi))
            b = np.zeros(fo)
            if li == len(shapes) - 1:
                b[0] = math.log(max(rho, 1e-6))
            parts += [W.ravel(), b]
        out[leaf] = np.concatenate(parts).astype(np.float32)
    return out.reshape(-1)


def with_biases(params: np.ndarray, seed: int, width: int, hidden: int, lx: int, ld: int,
                scale: float = 0.5) -> np.ndarray:
    """A copy of per-leaf MLP parameters (the xavier_weights layout) with every bias
    b_l and the head's b_o drawn from U[-scale, scale] (added to the density bias
    b_o[0]), one PCG64 stream in leaf, layer order: networks whose every layer has a
    nonzero bias."""
    rng = np.random.default_rng([seed, 0xB1A5])
    k0 = mlp_input_width(lx, ld)
    per = params_per_leaf(width, hidden, lx, ld)
    out = np.array(params, dtype=np.float32).reshape(-1, per).copy()
    for leaf in range(out.shape[0]):
        off = 0
        for fi, fo in [(k0, width)] + [(width, width)] * (hidden - 1) + [(width, 4)]:
            off += fi * fo
            out[leaf, off:off + fo] += rng.uniform(-scale, scale, size=fo).astype(np.float32)
            off += fo
    return out.reshape(-1)


PROPOSAL_PARAMS = 32 * 90 + 32 + 32 * 32 + 32 + 65 * 32 + 65


def proposal_init(seed: int) -> np.ndarray:
    """Xavier-uniform FP32 parameters of the proposal network (layers 90 -> 32 -> 32 ->
    65; layout W1, b1, W2, b2, W3, b3, rows = outputs), zero biases."""
    rng = np.random.default_rng([seed, 0x960905])
    parts = []
    for fo, fi in ((32, 90), (32, 32), (65, 32)):
        a = math.sqrt(6.0 / (fi + fo))
        parts += [rng.uniform(-a, a, size=(fo, fi)).ravel(), np.zeros(fo)]
    return np.concatenate(parts).astype(np.float32)
