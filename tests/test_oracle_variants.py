"""Pins of the oracle's printed-form variants (selectable by flag, each against what the paper and
the mathematics fix): Eq. 12 / Eq. 13 as printed (the weight K_ij dividing), matching to the
nearest cumulative share, and the gradient image as forward differences."""
from fractions import Fraction

import numpy as np
import pytest

import brute
import oracle
from paper_2510_21100_gb300 import synth


# ---------------------------------------------------------------- printed Eq. 12 / Eq. 13

def tiny_case(seed, K=8, H=5, W=6):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, K, size=(H, W, 3)).astype(np.uint8)
    S, G = oracle.histograms(img, K)
    return img, S, G


@pytest.mark.parametrize("seed", range(4))
def test_printed_update_equals_exact_rational_restatement(seed):
    K = 8
    _, S, G = tiny_case(seed, K)
    idx = [[oracle.class_index(K, i, j) for j in range(K)] for i in range(K)]
    R, L = G.astype(np.float64), S.astype(np.float64)
    # one iteration from the initial histograms, then one from a perturbed, non-integer iterate
    for step in range(2):
        got = oracle.iterate(S, G, R, L, K, 1e-2, 2e-2, printed=True)
        Ru, Lu = brute.iterate_printed_exact(S, G, R, L, 1e-2, 2e-2, idx)
        for g, w, name in ((got["Ru"], Ru, "R"), (got["Lu"], Lu, "L")):
            for k in range(K):
                if w[k] == 0:
                    assert g[k] == 0, (name, k)
                else:
                    assert abs(Fraction(float(g[k])) - w[k]) / w[k] < 1e-12, (name, k, float(g[k]), float(w[k]))
        R, L = got["Rn"] * np.linspace(0.9, 1.1, K), got["Ln"] * np.linspace(1.1, 0.9, K)


def test_printed_update_closed_form():
    """With K_ij = R_i L_j / P_k the printed quotient simplifies: the R update's data term is
    sum_{j in supp L} S_k P_k / (N R_i), the L update's sum_{i in supp R} (R'_i / R_i) S_k P_k / (N L_j)."""
    K = 256
    img = synth.low_light_image(80, 60, seed=5)
    S, G = oracle.histograms(img, K)
    R, L = G.astype(np.float64), S.astype(np.float64)
    out = oracle.iterate(S, G, R, L, K, 1e-3, 1e-3, printed=True)
    N = float(S.sum())
    idx = brute.class_map(K)
    P = np.zeros(K)
    np.add.at(P, idx.ravel(), np.outer(R, L).ravel())
    q = S.astype(np.float64) * P
    sR, sL = R > 0, L > 0
    Ru = np.zeros(K)
    for i in np.nonzero(sR)[0]:
        Ru[i] = q[idx[i, sL]].sum() / (N * R[i])
    Ru = (Ru + 1e-3 * G) / ((L * L).sum() / N**2 + 1e-3)
    Lu = np.zeros(K)
    for j in np.nonzero(sL)[0]:
        Lu[j] = ((Ru[sR] / R[sR]) * q[idx[sR, j]]).sum() / (N * L[j])
    Lu = (Lu + 1e-3 * S) / ((Ru * Ru).sum() / N**2 + 1e-3)
    for got, want in ((out["Ru"], Ru), (out["Lu"], Lu)):
        nz = want != 0
        assert np.array_equal(got != 0, nz)
        assert np.max(np.abs(got[nz] - want[nz]) / want[nz]) < 1e-12


def test_printed_update_constant_image_fixed_point():
    img = np.full((7, 9, 3), 40, np.uint8)
    S, G = oracle.histograms(img, 256)
    R, L, it = oracle.solve(S, G, oracle.Params(variants=oracle.VAR_PRINTED_UPDATE))
    N = 63
    assert it == 10
    assert abs(R[0] - N) <= 1e-13 * N and np.count_nonzero(R) == 1   # N x / x: two roundings
    assert abs(L[40] - N) <= 1e-13 * N and np.count_nonzero(L) == 1


def test_printed_update_mass_supports_and_difference_from_default():
    img = synth.low_light_image(120, 90, seed=8)
    S, G = oracle.histograms(img, 256)
    N = float(S.sum())
    p = oracle.Params(variants=oracle.VAR_PRINTED_UPDATE)
    R, L, _ = oracle.solve(S, G, p)
    assert abs(R.sum() - N) / N < 1e-12 and abs(L.sum() - N) / N < 1e-12
    assert np.all((R > 0) <= (G > 0)) and np.all((L > 0) <= (S > 0))
    R0, L0, _ = oracle.solve(S, G, oracle.Params())
    assert np.max(np.abs(L - L0)) / N > 1e-3  # the printed form is a different update


# ---------------------------------------------------------------- nearest-share matching

@pytest.mark.parametrize("seed", range(5))
def test_nearest_match_equals_exact_rational_search(seed):
    rng = np.random.default_rng(seed)
    K = 16
    S = rng.integers(0, 20, size=K).astype(np.uint64)
    S[rng.integers(0, K, size=4)] = 0
    S[3] += 1
    T = rng.random(K) * float(S.sum()) / K
    T[rng.integers(0, K, size=5)] = 0.0
    T[7] += 1.0
    assert np.array_equal(oracle.lut(S, T, K, nearest=True).astype(np.int64), brute.lut_nearest(S, T))


def test_nearest_match_identity_when_target_is_source():
    img = synth.low_light_image(90, 70, seed=4)
    S, _ = oracle.histograms(img, 256)
    lt = oracle.lut(S, S.astype(np.float64), 256, nearest=True)
    occ = np.nonzero(S)[0]
    assert np.array_equal(lt[occ], occ)


@pytest.mark.parametrize("seed", range(3))
def test_nearest_match_flat_target_closed_form(seed):
    """Flat target T_z = m, N = K m: the nearest share (z + 1) / K to CS(s) / N is z + 1 = the
    integer nearest to x = K CS(s) / N, halves down (first minimum): z = ceil(x - 3/2)."""
    rng = np.random.default_rng(seed)
    K, m = 64, 37
    N = K * m
    S = np.bincount(rng.integers(0, K, size=N) ** 2 // K, minlength=K).astype(np.uint64)
    T = np.full(K, float(m))
    lt = oracle.lut(S, T, K, nearest=True).astype(np.int64)
    CS = np.cumsum(S.astype(np.int64))
    for s in range(K):
        if CS[s] == N:
            assert lt[s] == K - 1
            continue
        x = Fraction(K * int(CS[s]), N)
        z = -((-(x - Fraction(3, 2)).numerator) // (x - Fraction(3, 2)).denominator)  # ceil(x - 3/2)
        assert lt[s] == max(0, min(K - 1, z)), (s, x)


def test_nearest_match_lies_at_or_below_the_reaching_level():
    img = synth.low_light_image(200, 150, seed=9)
    S, G = oracle.histograms(img, 256)
    R, L, _ = oracle.solve(S, G, oracle.Params())
    T = oracle.target(R, L, 256, 2.2, int(S.sum()))
    a = oracle.lut(S, T, 256).astype(np.int64)
    b = oracle.lut(S, T, 256, nearest=True).astype(np.int64)
    CT = np.cumsum(T)
    for s in np.nonzero(S)[0]:
        assert b[s] <= a[s]
        if b[s] < a[s]:
            assert CT[b[s]] == CT[a[s] - 1]  # the start of the plateau just below the reaching level
    assert np.all(np.diff(b[S > 0]) >= 0)


# ---------------------------------------------------------------- forward-difference gradient

@pytest.mark.parametrize("seed", range(4))
def test_forward_gradient_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 12)), int(rng.integers(1, 12))
    img = rng.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    S, G = oracle.histograms(img, 256, forward=True)
    V = brute.value_channel(img)
    assert np.array_equal(G.astype(np.int64), np.bincount(brute.forward_levels(V, 256).ravel(), minlength=256))
    assert np.array_equal(S.astype(np.int64), np.bincount(V.ravel(), minlength=256))


def test_forward_gradient_closed_forms():
    H, W = 6, 50
    y, x = np.mgrid[0:H, 0:W]
    ramp = np.repeat(x[..., None], 3, axis=2).astype(np.uint8)  # V = x: gx = 1 except at the last column
    _, G = oracle.histograms(ramp, 256, forward=True)
    assert G[1] == H * (W - 1) and G[0] == H and G.sum() == H * W
    step = np.where((y < 4)[..., None], 10, 73).astype(np.uint8).repeat(3, axis=2)  # gy = 63 on row 3 only
    _, G = oracle.histograms(step, 256, forward=True)
    assert G[63] == W and G[0] == H * W - W
    flat = np.full((5, 5, 3), 6, np.uint8)
    _, G = oracle.histograms(flat, 8, forward=True)
    assert G[0] == 25 and G.sum() == 25


def test_variants_end_to_end_at_k8_against_brute_force():
    """All three variants together through the whole oracle pipeline at K = 8 against the literal
    restatements (histograms, the target and the LUT decided exactly)."""
    rng = np.random.default_rng(11)
    img = rng.integers(0, 8, size=(6, 7, 3)).astype(np.uint8)
    v = oracle.VAR_PRINTED_UPDATE | oracle.VAR_NEAREST_MATCH | oracle.VAR_FORWARD_GRADIENT
    p = oracle.Params(K=8, alpha=1e-2, beta=1e-2, variants=v)
    r = oracle.enhance(img, p)
    V = brute.value_channel(img)
    assert np.array_equal(r.G.astype(np.int64), np.bincount(brute.forward_levels(V, 8).ravel(), minlength=8))
    idx = [[oracle.class_index(8, i, j) for j in range(8)] for i in range(8)]
    R, L = r.G.astype(np.float64), r.S.astype(np.float64)
    N = float(r.S.sum())
    for _ in range(10):
        Ru, Lu = brute.iterate_printed_exact(r.S, r.G, R, L, 1e-2, 1e-2, idx)
        Ru = np.array([float(x) for x in Ru])
        Lu = np.array([float(x) for x in Lu])
        R, L = N * Ru / Ru.sum(), N * Lu / Lu.sum()
    nz = R > 0
    assert np.max(np.abs(r.R[nz] - R[nz]) / R[nz]) < 1e-9
    T = brute.target(r.R, r.L, 8, 2.2, N)
    assert np.max(np.abs(r.T - T) / np.maximum(T, 1e-300)) < 1e-12
    assert np.array_equal(r.lut.astype(np.int64), brute.lut_nearest(r.S, r.T))
    assert np.array_equal(r.out, brute.apply(img, r.lut))
