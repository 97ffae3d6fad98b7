"""Seeded synthetic inputs: noisy 1D piecewise-constant signals, noisy polygon images,
block start vectors and mixed-size batches.

This module holds data generation only -- none of the filter's arithmetic. Both the CUDA
path and the CPU oracle receive the arrays it returns, so every random number the method
consumes (noise, the extra start columns of a block) is drawn here and passed in.

Recipes (numpy ``default_rng(seed)``, PCG64):

* ``signal_1d``: ``segments`` constant pieces; the ``segments - 1`` breakpoints are distinct
  sorted integers in [1, n) redrawn until every piece is at least ``min_len`` samples;
  levels U[0, 1]; additive N(0, noise^2).  Section 7 uses piecewise-linear signals with
  0.1*randn noise; ``kind="linear"`` gives that variant (ramps between random levels).
* ``polygon_image``: a linear-gradient background a + b*(u.p)/side (a, b ~ U[0, 1], u a
  random unit vector, p the pixel centre), then ``polygons`` star-shaped polygons painted
  in order (3..8 vertices at sorted random angles, radii U[0.05, 0.3]*side, centre uniform
  in the image, level U[0, 1]), then additive N(0, noise^2).  This stands in for the
  natural test image of Section 7, which is not available.
* ``block_start``: column 0 is the signal itself, columns 1..k-1 are N(0, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def signal_1d(n: int, seed: int, segments: int = 12, noise: float = 0.1,
              min_len: int = 16, kind: str = "constant", dtype=np.float64):
    """Return (clean, noisy) 1D signals of length n."""
    rng = np.random.default_rng(seed)
    segments = max(1, min(segments, n // max(min_len, 1)))
    while True:
        if segments == 1:
            bps = np.array([], dtype=np.int64)
            break
        bps = np.sort(rng.choice(np.arange(1, n), size=segments - 1, replace=False))
        edges = np.concatenate(([0], bps, [n]))
        if np.all(np.diff(edges) >= min_len):
            break
    edges = np.concatenate(([0], bps, [n]))
    levels = rng.uniform(0.0, 1.0, size=segments + 1)
    clean = np.empty(n, dtype=np.float64)
    for s in range(segments):
        a, b = edges[s], edges[s + 1]
        if kind == "constant":
            clean[a:b] = levels[s]
        elif kind == "linear":
            t = np.arange(b - a, dtype=np.float64) / max(b - a, 1)
            clean[a:b] = levels[s] + (levels[s + 1] - levels[s]) * t
        else:
            raise ValueError(f"unknown kind {kind!r}")
    noisy = clean + noise * rng.standard_normal(n)
    return clean.astype(dtype), noisy.astype(dtype)


def _inside_polygon(px, py, vx, vy):
    """Even-odd crossing test of points (px, py) against the closed polygon (vx, vy)."""
    inside = np.zeros(px.shape, dtype=bool)
    m = len(vx)
    for a in range(m):
        b = (a + 1) % m
        x0, y0, x1, y1 = vx[a], vy[a], vx[b], vy[b]
        if y0 == y1:
            continue
        cond = (py >= min(y0, y1)) & (py < max(y0, y1))
        xc = x0 + (py - y0) * (x1 - x0) / (y1 - y0)
        inside ^= cond & (px < xc)
    return inside


def polygon_image(ny: int, nx: int, seed: int, polygons: int = 20, noise: float = 0.05,
                  dtype=np.float32):
    """Return (clean, noisy) images of shape (ny, nx), row-major with x fastest."""
    rng = np.random.default_rng(seed)
    side = float(max(nx, ny))
    a, b = rng.uniform(0.0, 1.0, size=2)
    ang = rng.uniform(0.0, 2.0 * math.pi)
    ux, uy = math.cos(ang), math.sin(ang)
    ys, xs = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    proj = ux * xs + uy * ys
    proj -= proj.min()
    clean = a + b * proj / side
    for _ in range(polygons):
        nv = int(rng.integers(3, 9))
        th = np.sort(rng.uniform(0.0, 2.0 * math.pi, size=nv))
        rad = rng.uniform(0.05, 0.3, size=nv) * side
        cx, cy = rng.uniform(0.0, nx), rng.uniform(0.0, ny)
        level = rng.uniform(0.0, 1.0)
        vx = cx + rad * np.cos(th)
        vy = cy + rad * np.sin(th)
        x0 = max(0, int(math.floor(vx.min())))
        x1 = min(nx, int(math.ceil(vx.max())) + 1)
        y0 = max(0, int(math.floor(vy.min())))
        y1 = min(ny, int(math.ceil(vy.max())) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        sub = _inside_polygon(xs[y0:y1, x0:x1], ys[y0:y1, x0:x1], vx, vy)
        clean[y0:y1, x0:x1][sub] = level
    noisy = clean + noise * rng.standard_normal((ny, nx))
    return clean.astype(dtype), noisy.astype(dtype)


def block_start(x0: np.ndarray, k: int, seed: int, dtype=None):
    """Block start vectors [n][k] (pixel-major): column 0 = x0, the rest N(0, 1)."""
    x0 = np.asarray(x0).reshape(-1)
    dtype = dtype or x0.dtype
    rng = np.random.default_rng(seed + 7919)
    X = np.empty((x0.size, k), dtype=np.float64)
    X[:, 0] = x0
    if k > 1:
        X[:, 1:] = rng.standard_normal((x0.size, k - 1))
    return X.astype(dtype)


# Named workloads: the parameters of the five measured configurations.
@dataclass(frozen=True)
class Workload:
    name: str
    ndim: int
    nx: int
    ny: int
    radius: int
    sigma_s: float
    sigma_r: float
    noise: float
    seed: int
    cg_iters: int
    lobpcg_k: int
    lobpcg_iters: int
    dtype: str
    extra: dict = field(default_factory=dict)


SIGNAL_1D_4096 = Workload("signal1d_n4096_r5_fp64", 1, 4096, 1, 5, 3.0, 0.1, 0.1, 1,
                          20, 4, 10, "f64")
IMAGE_512 = Workload("image512_w7x7_fp32", 2, 512, 512, 3, 2.0, 0.08, 0.05, 2,
                     50, 16, 30, "f32")
IMAGE_2048 = Workload("image2048_w7x7_precision", 2, 2048, 2048, 3, 2.0, 0.08, 0.05, 3,
                      50, 32, 30, "f32")
IMAGE_1024 = Workload("image1024_w7x7_learned", 2, 1024, 1024, 3, 2.0, 0.08, 0.05, 5,
                      50, 16, 30, "f32")


def make_input(w: Workload, ny: int | None = None, nx: int | None = None):
    """(clean, noisy) for a workload; ny/nx override the size (smaller test cases)."""
    nx = nx or w.nx
    ny = ny or w.ny
    if w.ndim == 1:
        return signal_1d(nx, w.seed, noise=w.noise,
                         dtype=np.float64 if w.dtype == "f64" else np.float32)
    return polygon_image(ny, nx, w.seed, noise=w.noise,
                         dtype=np.float64 if w.dtype == "f64" else np.float32)


def batch_sizes(seed: int = 4, images: int = 192, signals: int = 64,
                img_range=(64, 1024), sig_range=(1e3, 1e6)):
    """Shapes of a mixed batch: images with log-uniform sides, signals with log-uniform
    lengths.  Returns a list of (ndim, ny, nx)."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi = math.log(img_range[0]), math.log(img_range[1])
    for _ in range(images):
        h = int(round(math.exp(rng.uniform(lo, hi))))
        w = int(round(math.exp(rng.uniform(lo, hi))))
        out.append((2, h, w))
    lo, hi = math.log(sig_range[0]), math.log(sig_range[1])
    for _ in range(signals):
        out.append((1, 1, int(round(math.exp(rng.uniform(lo, hi))))))
    return out


def psnr(clean: np.ndarray, img: np.ndarray, peak: float = 1.0) -> float:
    """Peak signal-to-noise ratio in dB."""
    mse = float(np.mean((np.asarray(img, np.float64) - np.asarray(clean, np.float64)) ** 2))
    return 10.0 * math.log10(peak * peak / mse)
