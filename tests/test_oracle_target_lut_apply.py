"""Pins for the enhanced histogram (Eq. 17-20), histogram matching and the colour-keeping apply."""
import colorsys

import numpy as np
import pytest

import brute
import oracle
from paper_2510_21100_gb300 import synth


def solved(K=256, W=96, H=64, seed=3, gamma=2.2):
    img = synth.low_light_image(W, H, seed=seed)
    S, G = oracle.histograms(img, K)
    R, L, _ = oracle.solve(S, G, oracle.Params(K=K))
    return img, S, G, R, L


def test_target_mass_is_pixel_count():
    _, S, _, R, L = solved()
    N = int(S.sum())
    for g in (1.0, 2.2, 5.0):
        T = oracle.target(R, L, 256, g, N)
        assert abs(T.sum() - N) / N < 1e-12 and (T >= 0).all()


def test_target_matches_literal_matrices():
    _, S, _, R, L = solved()
    N = int(S.sum())
    T = oracle.target(R, L, 256, 2.2, N)
    Tb = brute.target(R, L, 256, 2.2, N)
    nz = Tb > 0
    assert np.array_equal(T > 0, nz)
    assert np.max(np.abs(T[nz] - Tb[nz]) / Tb[nz]) < 1e-12


def test_target_with_gamma_one_is_model_estimate():
    """With gamma = 1, index_1 = index, so Eq. 20 reproduces the estimate of Eq. 8."""
    _, S, _, R, L = solved()
    N = int(S.sum())
    T = oracle.target(R, L, 256, 1.0, N)
    E = np.zeros(256)
    np.add.at(E, brute.class_map(256).ravel(), (np.outer(R, L) / N).ravel())
    nz = E > 0
    assert np.array_equal(T > 0, nz) and np.max(np.abs(T[nz] - E[nz]) / E[nz]) < 1e-12


def test_gamma_moves_target_mass_to_brighter_levels():
    _, S, _, R, L = solved()
    N = int(S.sum())
    means = [float((oracle.target(R, L, 256, g, N) * np.arange(256)).sum() / N) for g in (1.0, 1.5, 2.2, 5.0, 10.0)]
    assert all(b > a for a, b in zip(means, means[1:]))


def fp64_decision_margins(S, T):
    """Per level s: relative distance of the FP64 comparison CT(z) N vs CS(s) TT from a tie, over all z."""
    N = float(np.sum(S))
    CT = np.cumsum(np.asarray(T, dtype=np.float64))
    CS = np.cumsum(np.asarray(S, dtype=np.float64))
    rhs = CS[:, None] * CT[-1]
    return np.min(np.abs(CT[None, :] * N - rhs) / np.maximum(rhs, 1.0), axis=1)


@pytest.mark.parametrize("seed", range(4))
def test_lut_matches_exact_rational_search(seed):
    """Away from FP64 near-ties the oracle's matching decisions equal the exact-arithmetic ones,
    and at the top of the source CDF (CS(s) = N) they always do."""
    _, S, _, R, L = solved(seed=seed)
    T = oracle.target(R, L, 256, 2.2, int(S.sum()))
    got = oracle.lut(S, T, 256).astype(np.int64)
    want = brute.lut(S, T)
    top = np.cumsum(S) == S.sum()
    assert np.array_equal(got[top], want[top])
    robust = fp64_decision_margins(S, T) > 1e-12
    assert np.array_equal(got[robust], want[robust])


def test_lut_top_level_survives_absorbed_tail():
    """A target whose last occupied bins are far below the running sum's ulp: the brightest source
    level still maps to the last occupied target level (exact arithmetic), not to where the FP64
    running sum stopped changing."""
    K = 16
    S = np.zeros(K, np.uint64); S[3] = 5; S[7] = 5
    T = np.zeros(K); T[2] = 6.0; T[5] = 4.0; T[9] = 1e-30; T[12] = 1e-40
    lt = oracle.lut(S, T, K).astype(np.int64)
    assert lt[7] == 12 and lt[15] == 12
    assert np.array_equal(lt, brute.lut(S, T))


def test_lut_is_monotone():
    for seed in range(3):
        _, S, _, R, L = solved(seed=seed)
        T = oracle.target(R, L, 256, 2.2, int(S.sum()))
        lt = oracle.lut(S, T, 256).astype(np.int64)
        assert (np.diff(lt) >= 0).all()


def test_lut_is_identity_on_occupied_levels_when_target_is_source():
    _, S, _, _, _ = solved()
    lt = oracle.lut(S, S.astype(np.float64), 256)
    occ = np.nonzero(S)[0]
    assert np.array_equal(lt[occ].astype(np.int64), occ)


def test_lut_flat_target_closed_form():
    """Matching to a flat histogram is equalisation: LUT[s] = ceil(K CS(s) / N) - 1 in exact integers,
    within one level of the textbook transform of Eq. 5."""
    K = 256
    _, S, _, _, _ = solved()
    N = int(S.sum())
    lt = oracle.lut(S, np.ones(K), K).astype(np.int64)
    CS = np.cumsum(S.astype(np.int64))
    want = np.maximum(-(-(K * CS) // N) - 1, 0)
    assert np.array_equal(lt, want)
    he = np.floor((K - 1) * CS / N + 0.5).astype(np.int64)  # Eq. 5 rounded to nearest
    assert np.max(np.abs(lt - he)) <= 1


def test_apply_keeps_hue_and_saturation_and_sets_value():
    img = synth.low_light_image(40, 30, seed=9)
    K = 256
    rng = np.random.default_rng(0)
    lt = np.sort(rng.integers(0, K, K)).astype(np.uint16)
    out = oracle.apply(img, lt, K)
    V = img.max(axis=2)
    assert np.array_equal(out.max(axis=2), lt[V].astype(np.uint8))
    for y in range(0, 30, 3):
        for x in range(0, 40, 3):
            c = img[y, x].astype(float) / 255
            o = out[y, x].astype(float) / 255
            if c.max() == 0 or o.max() == 0:
                continue
            h0, s0, _ = colorsys.rgb_to_hsv(*c)
            h1, s1, _ = colorsys.rgb_to_hsv(*o)
            # rounding each channel to an integer perturbs hue/saturation by at most ~1/(2 V')
            tol = 1.0 / max(1, int(out[y, x].max())) + 1e-9
            assert abs(s0 - s1) <= tol
            if s0 > 0.2 and out[y, x].max() > 20:
                dh = min(abs(h0 - h1), 1 - abs(h0 - h1))
                assert dh <= tol


def test_apply_rounds_each_channel_to_nearest_with_halves_up():
    K = 256
    lt = np.arange(K, dtype=np.uint16)[::-1].copy()  # any LUT
    V = np.arange(1, K)
    out_all = []
    # all (c, V) pairs with c <= V, laid out as one image row per V
    img = np.zeros((K - 1, K, 3), dtype=np.uint8)
    for v in V:
        img[v - 1, :, 0] = v
        img[v - 1, : v + 1, 1] = np.arange(v + 1)
    out = oracle.apply(img, lt, K)
    for v in V:
        vp = int(lt[v])
        c = np.arange(v + 1, dtype=np.int64)
        o = out[v - 1, : v + 1, 1].astype(np.int64)
        # nearest integer to c*vp/v with halves rounded up:  2 o v - v <= 2 c vp < 2 o v + v
        assert ((2 * o * v - v <= 2 * c * vp) & (2 * c * vp < 2 * o * v + v)).all()


def test_apply_black_pixel_becomes_grey_value():
    img = np.zeros((1, 2, 3), dtype=np.uint8)
    lt = np.zeros(256, dtype=np.uint16)
    lt[0] = 17
    out = oracle.apply(img, lt, 256)
    assert (out == 17).all()


def test_apply_matches_rational_brute_force():
    img = synth.low_light_image(13, 11, seed=4)
    lt = np.clip(np.arange(256) * 2, 0, 255).astype(np.uint16)
    assert np.array_equal(oracle.apply(img, lt, 256), brute.apply(img, lt))
