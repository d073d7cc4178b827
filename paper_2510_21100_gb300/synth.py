"""Seeded synthetic low-light RGB images.

Stand-ins for the paper's low-light test images (ExDark, LOL, LSRW, MEF, NPE; Sec. IV),
none of which ship with this project.  The generator holds none of the enhancement
method's arithmetic: it only draws pixels.  Both the CUDA path and the CPU reference
consume the arrays it returns.

Recipe (every number is a parameter of :func:`low_light_image`):

* reflectance: Voronoi patches around ``n_cells`` uniform seeds, each patch an RGB colour
  drawn from U[0.2, 1], times a per-pixel, per-channel texture 1 + 0.1 * U[0, 1];
* illumination: sum of ``n_blobs`` Gaussian blobs (centres uniform over the image,
  sigma ~ U[40, 150] px scaled by sqrt(W*H / 240000), weights U[0.5, 1]), min-max rescaled
  into [illum_lo, illum_hi] (default [0.03, 0.35]);
* pixel = round(M * clip(illumination * reflectance + N(0, (2/255)^2), 0, 1)), M = 255 for
  8-bit data and 4095 for 12-bit data stored in uint16.
"""
from __future__ import annotations

import math

import numpy as np

try:  # scipy's k-d tree gives the exact nearest seed quickly; a numpy fallback keeps tests runnable
    from scipy.spatial import cKDTree as _KDTree
except Exception:  # pragma: no cover
    _KDTree = None


def seed_for(config_id: int, index: int) -> int:
    """Seed of image ``index`` of workload ``config_id``."""
    return int(config_id) * 1_000_000 + int(index)


def _voronoi_labels(rng: np.random.Generator, W: int, H: int, n_cells: int) -> np.ndarray:
    sx = rng.uniform(0, W, n_cells)
    sy = rng.uniform(0, H, n_cells)
    if _KDTree is not None:
        tree = _KDTree(np.stack([sx, sy], axis=1))
        labels = np.empty((H, W), dtype=np.int32)
        xs = np.arange(W, dtype=np.float64) + 0.5
        rows = max(1, (1 << 22) // max(W, 1))
        for y0 in range(0, H, rows):
            y1 = min(H, y0 + rows)
            yy, xx = np.meshgrid(np.arange(y0, y1, dtype=np.float64) + 0.5, xs, indexing="ij")
            _, lab = tree.query(np.stack([xx.ravel(), yy.ravel()], axis=1), k=1, workers=-1)
            labels[y0:y1] = lab.reshape(y1 - y0, W)
        return labels
    xs = np.arange(W, dtype=np.float64) + 0.5
    labels = np.empty((H, W), dtype=np.int32)
    for y in range(H):
        d = (xs[:, None] - sx[None, :]) ** 2 + (y + 0.5 - sy[None, :]) ** 2
        labels[y] = np.argmin(d, axis=1)
    return labels


def _scene(rng: np.random.Generator, W: int, H: int, n_cells: int, n_blobs: int):
    """Reflectance (H, W, 3) and the illumination's shape in [0, 1] (H, W) of one scene."""
    labels = _voronoi_labels(rng, W, H, n_cells)
    colours = rng.uniform(0.2, 1.0, size=(n_cells, 3)).astype(np.float32)
    refl = colours[labels]
    refl *= (1.0 + 0.1 * rng.random((H, W, 3), dtype=np.float32))

    scale = math.sqrt(W * H / 240000.0)
    illum = np.zeros((H, W), dtype=np.float32)
    xs = np.arange(W, dtype=np.float32)
    ys = np.arange(H, dtype=np.float32)
    for _ in range(n_blobs):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        sigma = rng.uniform(40.0, 150.0) * scale
        w = rng.uniform(0.5, 1.0)
        gx = np.exp(-((xs - cx) ** 2) / (2.0 * sigma * sigma)).astype(np.float32)
        gy = np.exp(-((ys - cy) ** 2) / (2.0 * sigma * sigma)).astype(np.float32)
        illum += np.float32(w) * np.outer(gy, gx)
    lo, hi = float(illum.min()), float(illum.max())
    if hi > lo:
        illum = (illum - lo) / (hi - lo)
    else:
        illum[:] = 0.5
    return refl, illum


def low_light_image(
    W: int,
    H: int,
    seed: int,
    bits: int = 8,
    n_cells: int = 64,
    n_blobs: int = 6,
    illum_lo: float = 0.03,
    illum_hi: float = 0.35,
    noise_sigma: float = 2.0 / 255.0,
) -> np.ndarray:
    """One synthetic low-light image, shape (H, W, 3), uint8 (bits <= 8) or uint16."""
    if W < 1 or H < 1:
        raise ValueError("image must be at least 1x1")
    rng = np.random.default_rng(seed)
    M = float((1 << bits) - 1)
    refl, illum = _scene(rng, W, H, n_cells, n_blobs)
    illum = illum_lo + (illum_hi - illum_lo) * illum

    img = refl * illum[:, :, None]
    img += rng.standard_normal((H, W, 3), dtype=np.float32) * np.float32(noise_sigma)
    np.clip(img, 0.0, 1.0, out=img)
    img = np.floor(img * np.float32(M) + np.float32(0.5))
    return img.astype(np.uint8 if bits <= 8 else np.uint16)


def normal_light_image(
    W: int,
    H: int,
    seed: int,
    bits: int = 8,
    n_cells: int = 64,
    n_blobs: int = 6,
    illum_lo: float = 0.45,
    illum_hi: float = 0.95,
) -> np.ndarray:
    """The scene of low_light_image(W, H, seed, ...) under normal light: the same reflectance and
    illumination shape with the illumination rescaled into [illum_lo, illum_hi], without noise (a
    reference image the generator knows, standing in for the paired normal-light images of the
    paper's datasets)."""
    if W < 1 or H < 1:
        raise ValueError("image must be at least 1x1")
    rng = np.random.default_rng(seed)
    M = float((1 << bits) - 1)
    refl, illum = _scene(rng, W, H, n_cells, n_blobs)
    illum = illum_lo + (illum_hi - illum_lo) * illum
    img = np.clip(refl * illum[:, :, None], 0.0, 1.0)
    img = np.floor(img * np.float32(M) + np.float32(0.5))
    return img.astype(np.uint8 if bits <= 8 else np.uint16)


def mixed_batch_sizes(n: int, seed: int, min_wh=(320, 240), max_wh=(1920, 1080)):
    """Image sizes with area log-uniform between two sizes and aspect 4:3, 16:9 or 3:2."""
    rng = np.random.default_rng(seed)
    a0, a1 = math.log(min_wh[0] * min_wh[1]), math.log(max_wh[0] * max_wh[1])
    aspects = [4 / 3, 16 / 9, 3 / 2]
    out = []
    for _ in range(n):
        area = math.exp(rng.uniform(a0, a1))
        ar = aspects[int(rng.integers(0, 3))]
        w = max(1, int(round(math.sqrt(area * ar))))
        h = max(1, int(round(area / w)))
        out.append((w, h))
    return out


def illumination_range(rng_seed: int, lo: float = 0.02, hi: float = 0.4):
    """Per-image illumination range: two uniform draws in [lo, hi], sorted."""
    rng = np.random.default_rng(rng_seed)
    a, b = sorted(rng.uniform(lo, hi, 2))
    return float(a), float(b)
