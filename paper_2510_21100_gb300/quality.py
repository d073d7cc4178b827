"""Image-quality measures for the gamma-sensitivity study (Sec. IV, Table III and Fig. 7 report
PSNR, SSIM, LOE and NIQE of the enhanced image for gamma from 1 to 10).  Host numpy, evaluation
only: nothing on the enhancement path uses them.

* PSNR: 10 log10(peak^2 / mean squared error) over all channels.
* SSIM: Wang, Bovik, Sheikh and Simoncelli (2004), per channel with an 11 x 11 Gaussian window of
  sigma 1.5 and constants (0.01 peak)^2, (0.03 peak)^2, averaged over the channels.
* LOE: lightness order error (Wang, Zheng, Hu and Li, 2013): with lightness L = max(r, g, b) on a
  downsampled grid, the mean over pixels of the number of pixels whose order relative to it
  differs between the input and the output.
NIQE needs a model fitted to natural images and is not computed.
"""
from __future__ import annotations

import math

import numpy as np


def psnr(a: np.ndarray, b: np.ndarray, peak: float = 255.0) -> float:
    d = a.astype(np.float64) - b.astype(np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0.0 else 10.0 * math.log10(peak * peak / mse)


def _gauss_blur(x: np.ndarray, sigma: float = 1.5, radius: int = 5) -> np.ndarray:
    """Separable Gaussian filter over the first two axes ('valid' region only)."""
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-t * t / (2.0 * sigma * sigma))
    k /= k.sum()
    H, W = x.shape[:2]
    if H <= 2 * radius or W <= 2 * radius:
        raise ValueError("image smaller than the SSIM window")
    y = sum(k[i] * x[i:H - 2 * radius + i] for i in range(2 * radius + 1))
    return sum(k[i] * y[:, i:W - 2 * radius + i] for i in range(2 * radius + 1))


def ssim(a: np.ndarray, b: np.ndarray, peak: float = 255.0) -> float:
    x = a.astype(np.float64)
    y = b.astype(np.float64)
    if x.ndim == 2:
        x, y = x[..., None], y[..., None]
    c1, c2 = (0.01 * peak) ** 2, (0.03 * peak) ** 2
    vals = []
    for ch in range(x.shape[2]):
        X, Y = x[..., ch], y[..., ch]
        mx, my = _gauss_blur(X), _gauss_blur(Y)
        sxx = _gauss_blur(X * X) - mx * mx
        syy = _gauss_blur(Y * Y) - my * my
        sxy = _gauss_blur(X * Y) - mx * my
        m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
        vals.append(float(np.mean(m)))
    return float(np.mean(vals))


def loe(inp: np.ndarray, out: np.ndarray, grid: int = 50) -> float:
    """Lightness order error on a grid x grid (at most) subsample of L = max(r, g, b)."""
    H, W = inp.shape[:2]
    sy, sx = max(1, H // grid), max(1, W // grid)
    li = inp.max(axis=2)[::sy, ::sx].astype(np.int64).ravel()
    lo = out.max(axis=2)[::sy, ::sx].astype(np.int64).ravel()
    total = 0
    for p in range(li.size):
        total += int(np.count_nonzero((li >= li[p]) != (lo >= lo[p])))
    return total / li.size


def mean_value(img: np.ndarray) -> float:
    """Mean of the HSV value channel V = max(r, g, b)."""
    return float(img.max(axis=2).mean())
