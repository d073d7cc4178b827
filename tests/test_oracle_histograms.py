"""Pins for the oracle's value channel, Eq. 3 histogram and gradient histogram."""
import numpy as np
import pytest

import brute
import oracle
from paper_2510_21100_gb300 import synth


def rand_img(H, W, K, seed, dtype=np.uint8):
    rng = np.random.default_rng(seed)
    return rng.integers(0, K, size=(H, W, 3)).astype(dtype)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 7), (7, 1), (2, 3), (5, 6), (9, 4)])
@pytest.mark.parametrize("K", [8, 256])
def test_histograms_match_brute_force(H, W, K):
    img = rand_img(H, W, K, seed=H * 100 + W + K)
    S, G = oracle.histograms(img, K)
    Sb, Gb = brute.histograms(img, K)
    assert np.array_equal(S.astype(np.int64), Sb)
    assert np.array_equal(G.astype(np.int64), Gb)


def test_histogram_mass_equals_pixel_count():
    img = synth.low_light_image(123, 77, seed=5)
    S, G = oracle.histograms(img, 256)
    assert int(S.sum()) == 123 * 77 and int(G.sum()) == 123 * 77


def test_value_channel_is_channel_max():
    img = rand_img(4, 5, 256, seed=1)
    V = oracle.value_channel(img, 256)
    assert np.array_equal(V, img.max(axis=2))


def test_constant_image_has_zero_gradient():
    img = np.full((6, 9, 3), 3, dtype=np.uint8)
    img[..., 1] = 5  # V = 5 everywhere
    S, G = oracle.histograms(img, 8)
    assert int(S[5]) == 54 and int(S.sum()) == 54
    assert int(G[0]) == 54 and int(G.sum()) == 54


def test_vertical_step_edge_closed_form():
    # left half V=a, right half V=b: at the two columns next to the edge the Sobel x-derivative is
    # (b-a)*(1+2+1) = 4(b-a) and the y-derivative is 0 (replicated rows), elsewhere both are 0.
    a, b, H, W = 10, 40, 5, 8
    img = np.zeros((H, W, 3), dtype=np.uint8)
    img[:, : W // 2, 2] = a
    img[:, W // 2:, 2] = b
    S, G = oracle.histograms(img, 256)
    assert int(G[4 * (b - a)]) == 2 * H
    assert int(G[0]) == (W - 2) * H


def test_gradient_clipped_to_top_level():
    # a single bright pixel: its 4-neighbours see |g| = 2*7 = 14 and diagonal ones 7*sqrt(2); K=8 clips to 7
    img = np.zeros((3, 3, 3), dtype=np.uint8)
    img[1, 1, 0] = 7
    S, G = oracle.histograms(img, 8)
    assert int(G[7]) == 8 and int(G[0]) == 1


def test_gradient_rounds_half_up():
    # diagonal neighbour of a bright pixel v: gx = gy = v, |g| = v*sqrt(2)
    for v in range(1, 200):
        img = np.zeros((3, 3, 3), dtype=np.uint8)
        img[1, 1, 0] = v
        _, G = oracle.histograms(img, 256)
        want = min(255, int(np.floor(v * np.sqrt(2.0) + 0.5)))
        assert int(G[want]) >= 4, v


def test_range_error_when_level_not_below_K():
    img = np.zeros((2, 2, 3), dtype=np.uint8)
    img[0, 0, 0] = 8
    with pytest.raises(oracle.OracleError) as e:
        oracle.histograms(img, 8)
    assert e.value.code == oracle.ERR_RANGE


def test_uint16_little_endian_levels():
    img = np.zeros((2, 3, 3), dtype=np.uint16)
    img[0, 0, 1] = 4095
    img[1, 2, 0] = 2048
    S, _ = oracle.histograms(img, 4096)
    assert int(S[4095]) == 1 and int(S[2048]) == 1 and int(S[0]) == 4
