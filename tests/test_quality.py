"""Pins of the image-quality measures used by the gamma-sensitivity replica."""
import numpy as np

from paper_2510_21100_gb300 import quality


def test_psnr_closed_form():
    a = np.zeros((10, 10, 3), np.uint8)
    b = np.full((10, 10, 3), 5, np.uint8)
    assert abs(quality.psnr(a, b) - 10 * np.log10(255 ** 2 / 25)) < 1e-12
    assert quality.psnr(a, a) == float("inf")


def test_ssim_identity_and_constant_shift():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 256, size=(40, 50, 3)).astype(np.uint8)
    assert abs(quality.ssim(a, a) - 1.0) < 1e-12
    # a constant offset leaves the structure and contrast terms at 1: SSIM = luminance term only
    x = np.full((30, 30), 100.0)
    y = x + 20.0
    c1 = (0.01 * 255) ** 2
    want = (2 * 100 * 120 + c1) / (100 ** 2 + 120 ** 2 + c1)
    assert abs(quality.ssim(x, y) - want) < 1e-12
    noisy = np.clip(a.astype(int) + rng.integers(-40, 41, size=a.shape), 0, 255).astype(np.uint8)
    assert 0.0 < quality.ssim(a, noisy) < 1.0


def test_loe_zero_for_monotone_maps_and_counts_inversions():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 200, size=(20, 20, 3)).astype(np.uint8)
    assert quality.loe(a, a + 10) == 0.0                  # an order-preserving map
    b = (255 - a).astype(np.uint8)                         # reverses every strict order
    L = a.max(axis=2).astype(np.int64).ravel()
    Lb = b.max(axis=2).astype(np.int64).ravel()
    brute = np.mean([np.count_nonzero((L >= L[p]) != (Lb >= Lb[p])) for p in range(L.size)])
    assert quality.loe(a, b, grid=20) == brute > 0
