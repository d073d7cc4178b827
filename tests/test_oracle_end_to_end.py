"""End-to-end pins of the oracle: brute force at K=8 on tiny images, and the gamma behaviour of Table III."""
import numpy as np
import pytest

import brute
import oracle
from paper_2510_21100_gb300 import synth


def lut_decision_margin(S, T):
    """Smallest relative distance of any LUT decision (CT(z) N vs CS(s) TT) from its threshold."""
    N = float(np.sum(S))
    CT = np.cumsum(np.asarray(T, dtype=np.float64))
    TT = CT[-1]
    CS = np.cumsum(np.asarray(S, dtype=np.float64))
    lhs = CT[None, :] * N
    rhs = CS[:, None] * TT
    return float(np.min(np.abs(lhs - rhs) / np.maximum(np.abs(rhs), 1.0)))


@pytest.mark.parametrize("seed", range(12))
def test_k8_brute_force_pipeline(seed):
    K = 8
    rng = np.random.default_rng(100 + seed)
    H, W = int(rng.integers(1, 7)), int(rng.integers(1, 7))
    img = rng.integers(0, K, size=(H, W, 3)).astype(np.uint8)
    p = oracle.Params(K=K, alpha=1e-2, beta=1e-2, gamma=2.2, max_iter=10)
    r = oracle.enhance(img, p)
    S, G = brute.histograms(img, K)
    assert np.array_equal(r.S.astype(np.int64), S) and np.array_equal(r.G.astype(np.int64), G)
    R, L = brute.solve(S, G, K, p.alpha, p.beta, p.max_iter)
    for a, b in ((r.R, R), (r.L, L)):
        nz = b != 0
        assert np.array_equal(a != 0, nz)
        assert np.max(np.abs(a[nz] - b[nz]) / b[nz], initial=0.0) < 1e-11
    N = H * W
    T = brute.target(R, L, K, p.gamma, N)
    nz = T > 0
    assert np.array_equal(r.T > 0, nz)
    assert np.max(np.abs(r.T[nz] - T[nz]) / T[nz], initial=0.0) < 1e-11
    lt = brute.lut(S, T)
    if lut_decision_margin(S, r.T) > 1e-9:  # decisions far from a tie are fixed by the mathematics
        assert np.array_equal(r.lut.astype(np.int64), lt)
    assert np.array_equal(r.out, brute.apply(img, r.lut))


def test_gamma_one_nearly_identity_and_brightness_rises_with_gamma():
    """Table III / Fig. 7: gamma = 1 gives the result closest to the input; raising gamma raises lightness."""
    img = synth.low_light_image(300, 200, seed=synth.seed_for(1, 0))
    psnr, light = [], []
    for g in (1.0, 1.5, 2.2, 5.0, 10.0):
        r = oracle.enhance(img, oracle.Params(gamma=g, alpha=1e-4, beta=1e-4))
        mse = float(((r.out.astype(np.float64) - img) ** 2).mean())
        psnr.append(10 * np.log10(255.0 ** 2 / mse))
        light.append(float(r.out.max(axis=2).mean()))
    assert psnr[0] > 28.0
    assert all(b < a for a, b in zip(psnr, psnr[1:]))
    assert all(b > a for a, b in zip(light, light[1:]))


def test_uint16_12bit_pipeline_runs_and_brightens():
    img = synth.low_light_image(64, 48, seed=3, bits=12)
    r = oracle.enhance(img, oracle.Params(K=4096, max_iter=2))
    assert r.out.dtype == np.uint16 and int(r.out.max()) < 4096
    assert r.out.max(axis=2).mean() > img.max(axis=2).mean()
    assert abs(r.T.sum() - 64 * 48) / (64 * 48) < 1e-12


@pytest.mark.parametrize("bits,K", [(8, 256), (12, 4096)])
def test_mirrored_tiling_scales_every_histogram_and_keeps_lut_and_pixels(bits, K):
    """Invariance the method implies: an image made of 2 x 2 blocks [T, T mirrored left-right; T
    mirrored top-bottom, T mirrored both ways] gives every pixel the 3 x 3 neighbourhood (mirrored) it
    has in T with the replicated border, so H_C(S) and H_C(grad S) are n times T's (n tiles); Eq. 11-15
    and Eq. 17-20 are homogeneous of degree one in (S, G, R, L, N), and with n a power of two the FP64
    scaling is exact, so R, L and the target are n times T's bit for bit, the LUT is T's, and the
    output is the same tiling of T's output.  (A border other than the replicated one, or a term of
    another degree, breaks it.)"""
    t = synth.low_light_image(37, 29, seed=5, bits=bits)
    top = np.concatenate([t, t[:, ::-1]], axis=1)
    blk = np.concatenate([top, top[::-1]], axis=0)
    big = np.ascontiguousarray(np.tile(blk, (2, 4, 1)))
    n = 32
    r = oracle.enhance(t, oracle.Params(K=K))
    rb = oracle.enhance(big, oracle.Params(K=K))
    assert np.array_equal(rb.S, n * r.S) and np.array_equal(rb.G, n * r.G)
    for a, b in ((rb.R, r.R), (rb.L, r.L), (rb.T, r.T)):
        assert np.array_equal(a / n, b)
    assert np.array_equal(rb.lut, r.lut)
    wo = np.concatenate([r.out, r.out[:, ::-1]], axis=1)
    wo = np.concatenate([wo, wo[::-1]], axis=0)
    assert np.array_equal(rb.out, np.tile(wo, (2, 4, 1)))
