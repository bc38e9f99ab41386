"""Seeded synthetic stereo scenes (inputs only; none of the matching arithmetic).

The paper evaluates on the Middlebury V3 benchmark (Sec. IV), which is not available
here.  These generators produce rectified grayscale pairs of the same shape class:
band-limited random texture, a Voronoi partition into regions that each carry a
constant or slanted-plane disparity, a z-buffered warp into the right view with
occlusions refilled by fresh texture, and additive Gaussian noise.  The left image is
the reference view: a left pixel (y, x) with disparity d appears in the right view at
column x - d.

Every array is produced from ``numpy.random.Generator(PCG64(seed))`` so that the
oracle and the CUDA path are fed identical inputs.  Only numpy is used.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "Scene",
    "SceneSpec",
    "SPECS",
    "make_texture",
    "make_pair",
    "make_batch_specs",
    "make_float_pair",
    "bad_rate",
]


@dataclasses.dataclass(frozen=True)
class SceneSpec:
    """Shape and content of one synthetic pair plus the matching parameters used on it."""

    width: int
    height: int
    regions: int
    max_disp: int          # D: candidate disparities 0..D-1
    levels: int            # K pyramid levels (1 = flat block matching)
    window: int            # odd ZNCC window side w = 2n+1
    radius: int            # refinement radius r
    noise_sigma: float
    slanted: bool          # slanted planes (real-valued) vs integer constants
    gain: float = 1.0      # right image photometric gain ...
    offset: float = 0.0    # ... and offset, applied before noise


# The five workloads: a small integer-shift pair, a half-resolution benchmark-shaped
# pair, the batching mix (sizes drawn by make_batch_specs), the float pair used by the
# differentiable level, and a large full-resolution pair with a photometric change.
SPECS = {
    "small_320x240": SceneSpec(320, 240, 4, 32, 3, 5, 2, 2.0, False),
    "bench_1400x1000": SceneSpec(1400, 1000, 12, 256, 4, 7, 2, 3.0, True),
    "diff_640x480": SceneSpec(640, 480, 12, 64, 1, 7, 0, 0.01, True),
    "large_2880x1984": SceneSpec(2880, 1984, 20, 640, 5, 9, 3, 5.0, True, 1.2, -10.0),
}


@dataclasses.dataclass
class Scene:
    left: np.ndarray       # uint8 (H, W)   (float64 in [0,1] for make_float_pair)
    right: np.ndarray      # same dtype as left
    gt: np.ndarray         # float64 (H, W) true left disparity
    mask: np.ndarray       # bool (H, W)  pixels where gt is meaningful
    spec: SceneSpec
    seed: int
    labels: np.ndarray | None = None   # int32 (H, W) Voronoi region of each left pixel


def _gauss_kernel(sigma: float, radius: int) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    return k / k.sum()


def _blur_axis(img: np.ndarray, k: np.ndarray, axis: int) -> np.ndarray:
    r = (len(k) - 1) // 2
    pad = [(0, 0), (0, 0)]
    pad[axis] = (r, r)
    p = np.pad(img, pad, mode="symmetric")
    out = np.zeros_like(img)
    n = img.shape[axis]
    for i, kv in enumerate(k):
        sl = [slice(None), slice(None)]
        sl[axis] = slice(i, i + n)
        out += kv * p[tuple(sl)]
    return out


def make_texture(rng: np.random.Generator, h: int, w: int, sigma: float = 1.5,
                 radius: int = 6) -> np.ndarray:
    """Band-limited texture in [0, 255] (float64): Gaussian-filtered uniform noise,
    min-max stretched."""
    u = rng.random((h, w))
    k = _gauss_kernel(sigma, radius)
    t = _blur_axis(_blur_axis(u, k, 0), k, 1)
    lo, hi = t.min(), t.max()
    return (t - lo) * (255.0 / max(hi - lo, 1e-12))


def _voronoi(rng: np.random.Generator, h: int, w: int, n: int):
    sy = rng.random(n) * h
    sx = rng.random(n) * w
    yy = np.arange(h, dtype=np.float64)[:, None]
    xx = np.arange(w, dtype=np.float64)[None, :]
    best = np.full((h, w), np.inf)
    lab = np.zeros((h, w), dtype=np.int32)
    for i in range(n):                      # ties keep the lower index
        dist = (yy - sy[i]) ** 2 + (xx - sx[i]) ** 2
        sel = dist < best
        best[sel] = dist[sel]
        lab[sel] = i
    return lab, sy, sx


def _planes(rng: np.random.Generator, n: int, d: int, slanted: bool):
    if slanted:
        c = rng.uniform(0.05 * d, 0.95 * d, n)
        a = rng.uniform(-0.05, 0.05, n)
        b = rng.uniform(-0.05, 0.05, n)
    else:
        c = rng.integers(0, d, n).astype(np.float64)
        a = np.zeros(n)
        b = np.zeros(n)
    return c, a, b


def _warp(left_tex: np.ndarray, lab: np.ndarray, sy, sx, c, a, b, d_max: int):
    """Z-buffered warp of the left view into the right view.

    Returns the right texture (NaN where no left pixel lands), the left disparity map
    (float64, clamped to [0, d_max-1]) and the visibility mask of left pixels."""
    h, w = lab.shape
    yy = np.arange(h, dtype=np.float64)[:, None]
    xr = np.arange(w, dtype=np.float64)[None, :]
    xl_all = np.arange(w, dtype=np.float64)[None, :]
    best_d = np.full((h, w), -np.inf)
    best_x = np.full((h, w), np.nan)
    best_r = np.full((h, w), -1, dtype=np.int32)
    for r in range(len(c)):
        # left x solving x - d_r(x, y) = x_r for the (unclamped) plane of region r
        xl = (xr + c[r] - a[r] * sx[r] + b[r] * (yy - sy[r])) / (1.0 - a[r])
        xl = np.broadcast_to(xl, (h, w))
        dv = xl - xr
        xi = np.rint(xl)
        inside = (xi >= 0) & (xi <= w - 1) & (dv >= 0) & (dv <= d_max - 1)
        xi_c = np.clip(xi, 0, w - 1).astype(np.int64)
        rows = np.broadcast_to(np.arange(h)[:, None], (h, w))
        own = lab[rows, xi_c] == r
        ok = inside & own & (dv > best_d)
        best_d = np.where(ok, dv, best_d)
        best_x = np.where(ok, xl, best_x)
        best_r = np.where(ok, r, best_r)
    # sample the left texture linearly along the row at the winning source column
    right = np.full((h, w), np.nan)
    have = best_r >= 0
    x0 = np.floor(np.where(have, best_x, 0.0)).astype(np.int64)
    fx = np.where(have, best_x, 0.0) - x0
    x0c = np.clip(x0, 0, w - 1)
    x1c = np.clip(x0 + 1, 0, w - 1)
    rows = np.broadcast_to(np.arange(h)[:, None], (h, w))
    samp = (1.0 - fx) * left_tex[rows, x0c] + fx * left_tex[rows, x1c]
    right[have] = samp[have]
    # left disparity map and visibility
    d_left_raw = c[lab] + a[lab] * (xl_all - sx[lab]) + b[lab] * (yy - sy[lab])
    d_left = np.clip(d_left_raw, 0.0, d_max - 1)
    xr_of_left = np.rint(xl_all - d_left_raw)
    in_img = (xr_of_left >= 0) & (xr_of_left <= w - 1) & (d_left_raw >= 0) & (d_left_raw <= d_max - 1)
    xr_c = np.clip(xr_of_left, 0, w - 1).astype(np.int64)
    vis = in_img & (best_r[rows, xr_c] == lab) & (np.abs(best_x[rows, xr_c] - xl_all) <= 1.0)
    return right, d_left, vis


def make_pair(spec: SceneSpec, seed: int) -> Scene:
    """One uint8 stereo pair with ground truth for ``spec`` from ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h, w = spec.height, spec.width
    tex_l = make_texture(rng, h, w)
    tex_fill = make_texture(rng, h, w)
    lab, sy, sx = _voronoi(rng, h, w, spec.regions)
    c, a, b = _planes(rng, spec.regions, spec.max_disp, spec.slanted)
    left_f = np.rint(tex_l)
    right_f, d_left, vis = _warp(left_f, lab, sy, sx, c, a, b, spec.max_disp)
    hole = np.isnan(right_f)
    right_f[hole] = np.rint(tex_fill[hole])
    right_f = spec.gain * right_f + spec.offset
    if spec.noise_sigma > 0:
        right_f = right_f + rng.normal(0.0, spec.noise_sigma, (h, w))
    left = np.clip(left_f, 0, 255).astype(np.uint8)
    right = np.clip(np.rint(right_f), 0, 255).astype(np.uint8)
    n = spec.window // 2
    border = np.zeros((h, w), dtype=bool)
    border[n:h - n, n:w - n] = True
    xx = np.arange(w)[None, :]
    mask = vis & border & (xx - np.rint(d_left) >= 0)
    return Scene(left, right, np.rint(d_left), mask, spec, seed, lab)


def make_float_pair(spec: SceneSpec, seed: int) -> Scene:
    """Float64 pair in [0, 1] (for the differentiable level): the same scene model,
    with the noise sigma applied on the [0, 1] scale and no rounding."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h, w = spec.height, spec.width
    tex_l = make_texture(rng, h, w) / 255.0
    tex_fill = make_texture(rng, h, w) / 255.0
    lab, sy, sx = _voronoi(rng, h, w, spec.regions)
    c, a, b = _planes(rng, spec.regions, spec.max_disp, spec.slanted)
    right, d_left, vis = _warp(tex_l, lab, sy, sx, c, a, b, spec.max_disp)
    hole = np.isnan(right)
    right[hole] = tex_fill[hole]
    if spec.noise_sigma > 0:
        right = right + rng.normal(0.0, spec.noise_sigma, (h, w))
    right = np.clip(right, 0.0, 1.0)
    return Scene(tex_l, right, d_left, vis, spec, seed, lab)


_BATCH_SIZES = [(320, 240), (640, 480), (1280, 720), (1400, 1000), (1920, 1080)]


def make_batch_specs(n_pairs: int, seed: int) -> list[SceneSpec]:
    """Per-pair specs for the mixed-size batch: size drawn uniformly from five
    resolutions; D = W/5 rounded (half up) to a multiple of 16; K the deepest pyramid
    whose coarsest width stays >= 160; window 5 or 7; radius 2; slanted planes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for _ in range(n_pairs):
        w, h = _BATCH_SIZES[int(rng.integers(0, len(_BATCH_SIZES)))]
        d = 16 * int(np.floor(w / 80.0 + 0.5))
        k = 1
        while -(-w // (1 << k)) >= 160:
            k += 1
        win = int(rng.choice([5, 7]))
        specs.append(SceneSpec(w, h, 12, d, k, win, 2, 3.0, True))
    return specs


def bad_rate(d: np.ndarray, gt: np.ndarray, mask: np.ndarray, tau: float = 1.0) -> float:
    """Fraction of masked pixels whose disparity is off by more than ``tau``."""
    m = mask.astype(bool)
    if not m.any():
        return 0.0
    return float(np.mean(np.abs(d.astype(np.float64)[m] - gt[m]) > tau))
