"""Pins of the oracle's binned form: K bins over M > K data levels (the paper's "l levels",
Sec. II preamble, with fewer bins than levels, e.g. K = 256 on 12-bit data).  Reading: value v
falls into bin v >> log2(M / K); bin k is located at its centre value, normalised,
(k w + (w - 1) / 2) / (M - 1) with w = M / K; the class maps are the definitions' argmins over those
locations; the gradient level is clipped to M - 1 and binned likewise; the new value keeps the
pixel's place in its bin."""
from fractions import Fraction

import numpy as np
import pytest

import brute
import oracle
from paper_2510_21100_gb300 import synth


@pytest.mark.parametrize("K,M", [(8, 64), (16, 256), (256, 4096), (64, 256)])
def test_bin_locations_closed_form(K, M):
    locs = brute.bin_locations_exact(K, M)
    for k in list(range(min(K, 12))) + [K - 1]:
        assert oracle.bin_location(k, K, M) == float(locs[k])


@pytest.mark.parametrize("K", [8, 16, 256])
def test_one_bin_per_level_reduces_to_the_default(K):
    """M = K: the binned class maps equal the default closed form and index_1 table, and the whole
    pipeline gives the default's results bit for bit."""
    cm = oracle.class_table(K, K)
    ref = np.array([[oracle.class_index(K, i, j) for j in range(K)] for i in range(K)])
    assert np.array_equal(cm, ref)
    for g in (1.0, 2.2, 5.0):
        assert np.array_equal(oracle.index1_table_binned(K, K, g), oracle.index1_table(K, g))
    img = synth.low_light_image(90, 70, seed=K) if K == 256 else \
        np.random.default_rng(K).integers(0, K, size=(30, 40, 3)).astype(np.uint8)
    a = oracle.enhance(img, oracle.Params(K=K))
    b = oracle.enhance(img, oracle.Params(K=K, levels=K))
    for f in ("out", "S", "G", "R", "L", "T", "lut"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


@pytest.mark.parametrize("K,M", [(8, 64), (16, 256), (8, 32)])
def test_binned_class_maps_equal_exact_argmin(K, M):
    """The FP64 class map and index_1 (gamma = 2) against exact rational argmins: equal wherever the
    minimum is not shared by two levels."""
    locs = brute.bin_locations_exact(K, M)
    cm = oracle.class_table(K, M)
    i1 = oracle.index1_table_binned(K, M, 2.0)
    ties = 0
    for i in range(K):
        for j in range(K):
            k, tie = brute.nearest_exact(locs[i] * locs[j], locs)
            ties += tie
            if not tie:
                assert cm[i, j] == k, (i, j)
            # gamma = 2: location(j)^(1/2) is irrational in general; compare with the float argmin
    assert np.array_equal(i1, brute.class_map_binned_float(K, M, gamma=2.0))
    assert np.array_equal(cm, brute.class_map_binned_float(K, M))
    assert ties < K * K // 8


@pytest.mark.parametrize("K,M,bits", [(8, 64, 6), (64, 256, 8), (256, 4096, 12)])
def test_binned_histograms(K, M, bits):
    rng = np.random.default_rng(K)
    H, W = 23, 31
    img = rng.integers(0, M, size=(H, W, 3)).astype(np.uint8 if M <= 256 else np.uint16)
    S, G = oracle.histograms_binned(img, K, M)
    Sb, Gb = brute.histograms_binned(img, K, M)
    assert np.array_equal(S.astype(np.int64), Sb) and np.array_equal(G.astype(np.int64), Gb)
    assert S.sum() == G.sum() == H * W


def test_binned_apply_keeps_the_place_in_the_bin():
    K, M = 16, 256
    rng = np.random.default_rng(5)
    img = rng.integers(0, M, size=(9, 13, 3)).astype(np.uint8)
    lut = np.sort(rng.integers(0, K, size=K)).astype(np.uint16)
    out = oracle.apply_binned(img, lut, K, M)
    assert np.array_equal(out, brute.apply_binned(img, lut, K, M))
    V, Vo = img.max(axis=2).astype(int), out.max(axis=2).astype(int)
    nz = V > 0
    assert np.array_equal((Vo % 16)[nz], (V % 16)[nz]) and np.array_equal((Vo // 16)[nz], lut[V[nz] // 16])


@pytest.mark.parametrize("seed", range(4))
def test_binned_pipeline_at_k8_against_brute_force(seed):
    K, M = 8, 32
    rng = np.random.default_rng(300 + seed)
    img = rng.integers(0, M, size=(int(rng.integers(2, 7)), int(rng.integers(2, 7)), 3)).astype(np.uint8)
    p = oracle.Params(K=K, levels=M, alpha=1e-2, beta=1e-2)
    r = oracle.enhance(img, p)
    S, G = brute.histograms_binned(img, K, M)
    assert np.array_equal(r.S.astype(np.int64), S) and np.array_equal(r.G.astype(np.int64), G)
    idx = brute.class_map_binned_float(K, M)
    R, L = G.astype(np.float64), S.astype(np.float64)
    for _ in range(10):
        _, _, R, L, _ = brute.iterate_literal(S, G, R, L, p.alpha, p.beta, idx)
    nz = R > 0
    assert np.array_equal(r.R > 0, nz) and np.max(np.abs(r.R[nz] - R[nz]) / R[nz]) < 1e-11
    N = float(S.sum())
    idx1 = brute.class_map_binned_float(K, M, gamma=2.2)
    T = np.zeros(K)
    np.add.at(T, idx1.ravel(), (np.outer(R, L) / N).ravel())
    nz = T > 0
    assert np.array_equal(r.T > 0, nz) and np.max(np.abs(r.T[nz] - T[nz]) / T[nz]) < 1e-11
    assert np.array_equal(r.lut.astype(np.int64), brute.lut(S, r.T))
    assert np.array_equal(r.out, brute.apply_binned(img, r.lut, K, M))


def test_binned_12bit_k256_brightens():
    img = synth.low_light_image(120, 90, seed=17, bits=12)
    rb = oracle.enhance(img, oracle.Params(K=256, levels=4096))
    assert rb.out.dtype == np.uint16 and int(rb.out.max()) < 4096
    assert abs(rb.T.sum() - 120 * 90) < 1e-9 * 120 * 90
    assert rb.out.max(axis=2).astype(float).mean() > 1.5 * img.max(axis=2).astype(float).mean()
