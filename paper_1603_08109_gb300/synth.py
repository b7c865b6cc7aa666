"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's experiments use 512x512 8-bit grayscale natural images
(Sec. IV, Fig. 5); those images are not available, so every workload here is
a seeded synthetic stand-in with intensities in [0, 255]:

* ``blocks_image``: piecewise-constant square blocks with levels drawn
  uniformly from [0, 255], plus i.i.d. Gaussian noise, clipped to [0, 255].
* ``gradient_polygons_image``: a smooth bilinear gradient spanning [0, 255],
  overpainted with random sharp-edged polygons of uniform random level, plus
  Gaussian noise, clipped.
* ``batch_specs``: the uneven-size batch (sizes, spatial kind, sigma_s,
  sigma_r per image).

This module holds none of the filter's arithmetic; it only draws numbers.
Every generator uses numpy's PCG64 ``default_rng(seed)`` in float64 and casts
the image to float32 at the end, so the CPU checker and the GPU path receive
the same bytes.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "blocks_image",
    "gradient_polygons_image",
    "batch_specs",
    "random_like",
    "workload_seed",
]


def workload_seed(config_index: int, image_index: int = 0) -> int:
    """Seed convention: config index * 1000 + image index."""
    return int(config_index) * 1000 + int(image_index)


def blocks_image(height: int, width: int, block: int = 16, noise_sigma: float = 20.0,
                 seed: int = 0) -> np.ndarray:
    """Piecewise-constant ``block`` x ``block`` tiles, uniform levels in [0,255],
    plus N(0, noise_sigma^2) noise, clipped to [0, 255]; float32, C order."""
    rng = np.random.default_rng(seed)
    by = -(-height // block)
    bx = -(-width // block)
    levels = rng.uniform(0.0, 255.0, size=(by, bx))
    img = np.repeat(np.repeat(levels, block, axis=0), block, axis=1)[:height, :width]
    img = img + rng.normal(0.0, noise_sigma, size=(height, width))
    return np.ascontiguousarray(np.clip(img, 0.0, 255.0).astype(np.float32))


def _fill_polygon(img: np.ndarray, vx: np.ndarray, vy: np.ndarray, level: float) -> None:
    """Even-odd scanline fill of one polygon (pixel centres at integer coords)."""
    h, w = img.shape
    y0 = max(int(np.floor(vy.min())), 0)
    y1 = min(int(np.ceil(vy.max())), h - 1)
    x0 = max(int(np.floor(vx.min())), 0)
    x1 = min(int(np.ceil(vx.max())), w - 1)
    if y1 < y0 or x1 < x0:
        return
    bw = x1 - x0 + 2
    toggle = np.zeros((y1 - y0 + 1, bw), dtype=np.int32)
    ys = np.arange(y0, y1 + 1, dtype=np.float64)
    nv = len(vx)
    for k in range(nv):
        ax, ay = vx[k], vy[k]
        bx_, by_ = vx[(k + 1) % nv], vy[(k + 1) % nv]
        if ay == by_:
            continue
        lo, hi = (ay, by_) if ay < by_ else (by_, ay)
        sel = (ys >= lo) & (ys < hi)
        if not sel.any():
            continue
        yy = ys[sel]
        xx = ax + (yy - ay) * (bx_ - ax) / (by_ - ay)
        # pixel column c is inside iff crossings to its left are odd: toggle at ceil(x)
        col = np.clip(np.ceil(xx).astype(np.int64) - x0, 0, bw - 1)
        np.add.at(toggle, ((yy - y0).astype(np.int64), col), 1)
    inside = (np.cumsum(toggle, axis=1) & 1).astype(bool)[:, : x1 - x0 + 1]
    sub = img[y0:y1 + 1, x0:x1 + 1]
    sub[inside] = level


def gradient_polygons_image(height: int, width: int, n_polygons: int = 64,
                            noise_sigma: float = 15.0, seed: int = 0) -> np.ndarray:
    """Smooth bilinear gradient spanning [0,255] + ``n_polygons`` random
    sharp-edged polygons (5-8 vertices, uniform levels) + N(0, noise^2),
    clipped to [0, 255]; float32, C order."""
    rng = np.random.default_rng(seed)
    corners = rng.uniform(0.0, 255.0, size=4)
    corners[rng.integers(0, 4)] = 0.0
    corners[rng.integers(0, 4)] = 255.0
    ty = (np.arange(height, dtype=np.float64) / max(height - 1, 1))[:, None]
    tx = (np.arange(width, dtype=np.float64) / max(width - 1, 1))[None, :]
    img = (corners[0] * (1 - ty) * (1 - tx) + corners[1] * (1 - ty) * tx
           + corners[2] * ty * (1 - tx) + corners[3] * ty * tx)
    img = np.ascontiguousarray(img)
    scale = min(height, width)
    for _ in range(n_polygons):
        nv = int(rng.integers(5, 9))
        cy = rng.uniform(0, height)
        cx = rng.uniform(0, width)
        rad = rng.uniform(0.03, 0.15) * scale
        ang = np.sort(rng.uniform(0, 2 * np.pi, size=nv))
        rr = rad * rng.uniform(0.5, 1.0, size=nv)
        vy = cy + rr * np.sin(ang)
        vx = cx + rr * np.cos(ang)
        _fill_polygon(img, vx, vy, float(rng.uniform(0.0, 255.0)))
    img = img + rng.normal(0.0, noise_sigma, size=(height, width))
    return np.ascontiguousarray(np.clip(img, 0.0, 255.0).astype(np.float32))


def batch_specs(count: int = 256, seed: int = 3000, min_hw=(64, 64), max_hw=(768, 1024),
                sigma_s_range=(2.0, 15.0), sigma_r_range=(10.0, 80.0)):
    """Per-image specs for the uneven batch: height ~ U{64..768},
    width ~ U{64..1024} (independent integers), kind ~ Bernoulli(1/2)
    (0 = box, 1 = Gaussian), sigma_s ~ U[2, 15], radius = ceil(3 sigma_s),
    sigma_r ~ U[10, 80]. Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(count):
        h = int(rng.integers(min_hw[0], max_hw[0] + 1))
        w = int(rng.integers(min_hw[1], max_hw[1] + 1))
        kind = int(rng.integers(0, 2))
        ss = float(rng.uniform(*sigma_s_range))
        sr = float(rng.uniform(*sigma_r_range))
        specs.append({"height": h, "width": w, "kind": kind, "sigma_s": ss,
                      "radius": int(np.ceil(3.0 * ss - 1e-9)), "sigma_r": sr,
                      "seed": seed + 1 + k})
    return specs


def random_like(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Standard-normal float32 array (cotangents, FD directions)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray((scale * rng.standard_normal(size=shape)).astype(np.float32))
