"""Pins for the oracle's two-level optimisation (Eq. 9-15, Algorithm 1)."""
import numpy as np
import pytest

import brute
import oracle
from paper_2510_21100_gb300 import synth


def small_case(K, seed, H=6, W=7):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, K, size=(H, W, 3)).astype(np.uint8 if K <= 256 else np.uint16)
    S, G = oracle.histograms(img, K)
    return img, S, G


def synth_case(K=256, W=96, H=64, seed=11):
    img = synth.low_light_image(W, H, seed=seed)
    S, G = oracle.histograms(img, K)
    return img, S, G


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


@pytest.mark.parametrize("K,seed", [(8, 1), (8, 2), (16, 3), (256, 4)])
@pytest.mark.parametrize("ab", [(1e-3, 1e-3), (1e-2, 1e-4), (0.5, 2.0)])
def test_one_iteration_matches_literal_matrices(K, seed, ab):
    alpha, beta = ab
    if K == 256:
        _, S, G = synth_case(K, seed=seed)
    else:
        _, S, G = small_case(K, seed)
    R = G.astype(np.float64)
    L = S.astype(np.float64)
    o = oracle.iterate(S, G, R, L, K, alpha, beta)
    Ru, Lu, Rn, Ln, _ = brute.iterate_literal(S, G, R, L, alpha, beta, brute.class_map(K))
    for a, b in ((o["Ru"], Ru), (o["Lu"], Lu), (o["Rn"], Rn), (o["Ln"], Ln)):
        nz = b != 0
        assert np.array_equal(a == 0, b == 0)
        assert rel(a[nz], b[nz]) < 1e-12


def test_solve_matches_literal_matrices_over_ten_iterations():
    K = 16
    _, S, G = small_case(K, 7, H=9, W=11)
    R, L, it = oracle.solve(S, G, oracle.Params(K=K, alpha=1e-2, beta=1e-2, max_iter=10))
    Rb, Lb = brute.solve(S, G, K, 1e-2, 1e-2, 10)
    assert it == 10
    nz = Rb != 0
    assert rel(R[nz], Rb[nz]) < 1e-11 and rel(L[Lb != 0], Lb[Lb != 0]) < 1e-11


@pytest.mark.parametrize("K,seed", [(8, 5), (16, 6)])
def test_updates_are_stationary_points_of_eq10(K, seed):
    """Eq. 13 minimises Eq. 10 in R (L and K_ij fixed); Eq. 12 then minimises it in L with the new R."""
    alpha, beta = 3e-3, 7e-3
    _, S, G = small_case(K, seed)
    idx = brute.class_map(K)
    R = G.astype(np.float64) * 1.3 + 0.5 * (G > 0)
    L = S.astype(np.float64) * 0.7 + 0.25 * (S > 0)
    o = oracle.iterate(S, G, R, L, K, alpha, beta)
    N = float(S.sum())
    Km = brute.weights(R, L, idx, N)
    J = lambda r, l: brute.objective_eq10(r, l, Km, S, G, idx, alpha, beta)
    # the objective is a strictly convex quadratic in each block, so the minimiser is unique:
    # any perturbation of the update must increase J
    Ru, Lu = o["Ru"], o["Lu"]
    base_R = J(Ru, L)
    base_L = J(Ru, Lu)
    rng = np.random.default_rng(seed)
    for _ in range(20):
        d = rng.standard_normal(K) * 1e-3 * (1 + np.abs(Ru))
        assert J(Ru + d, L) > base_R
        assert J(Ru - d, L) > base_R
        e = rng.standard_normal(K) * 1e-3 * (1 + np.abs(Lu))
        assert J(Ru, Lu + e) > base_L
        assert J(Ru, Lu - e) > base_L


def test_r_update_equals_least_squares_solution():
    """With L and K_ij fixed, Eq. 10 is a linear least-squares problem in R; numpy's lstsq solves it."""
    K, alpha, beta = 8, 1e-2, 2e-2
    _, S, G = small_case(K, 9)
    idx = brute.class_map(K)
    R = G.astype(np.float64) + 1.0 * (G > 0)
    L = S.astype(np.float64) + 2.0 * (S > 0)
    N = float(S.sum())
    Km = brute.weights(R, L, idx, N)
    Sidx = S.astype(np.float64)[idx]
    rows, rhs = [], []
    for i in range(K):
        for j in range(K):
            a = np.zeros(K)
            a[i] = L[j] / N
            rows.append(a)
            rhs.append(Km[i, j] * Sidx[i, j])
    for i in range(K):  # beta * (R_i - G_i)^2
        a = np.zeros(K)
        a[i] = np.sqrt(beta)
        rows.append(a)
        rhs.append(np.sqrt(beta) * float(G[i]))
    x, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    o = oracle.iterate(S, G, R, L, K, alpha, beta)
    assert np.allclose(o["Ru"], x, rtol=1e-9, atol=1e-9 * np.abs(x).max())


def test_class_totals_partition_all_cells():
    _, S, G = synth_case()
    R = G.astype(np.float64)
    L = S.astype(np.float64)
    o = oracle.iterate(S, G, R, L, 256, 1e-3, 1e-3)
    assert abs(o["P"].sum() - R.sum() * L.sum()) / (R.sum() * L.sum()) < 1e-12
    # q is S / P on occupied classes and 0 on empty ones
    occ = o["P"] > 0
    assert np.allclose(o["q"][occ], S[occ] / o["P"][occ], rtol=1e-15)
    assert (o["q"][~occ] == 0).all()


def test_renormalisation_and_supports_over_iterations():
    _, S, G = synth_case()
    N = float(S.sum())
    R = G.astype(np.float64)
    L = S.astype(np.float64)
    for _ in range(10):
        o = oracle.iterate(S, G, R, L, 256, 1e-3, 1e-3)
        R, L = o["Rn"], o["Ln"]
        assert abs(R.sum() - N) / N < 1e-12 and abs(L.sum() - N) / N < 1e-12
        assert np.array_equal(R > 0, G > 0) and np.array_equal(L > 0, S > 0)
        assert (R >= 0).all() and (L >= 0).all()


def test_constant_image_closed_form():
    """Constant V = a: S = N e_a, G = N e_0.  The only cell is (0, a) in class 0, so q = 0 and the
    iteration keeps R = N e_0, L = N e_a; the target is N e_0 and every level maps to 0."""
    K, a, H, W = 8, 5, 4, 6
    img = np.full((H, W, 3), a, dtype=np.uint8)
    N = H * W
    r = oracle.enhance(img, oracle.Params(K=K, gamma=2.2))
    e0 = np.zeros(K); e0[0] = N
    ea = np.zeros(K); ea[a] = N
    assert np.array_equal(r.R, e0) and np.array_equal(r.L, ea)
    assert np.array_equal(r.T, e0)
    assert (r.lut == 0).all() and (r.out == 0).all()


def test_stop_rule_stops_early_with_large_eps():
    _, S, G = synth_case()
    _, _, it = oracle.solve(S, G, oracle.Params(eps=1e30, fixed_iters=False, max_iter=10))
    assert it == 1
    _, _, it = oracle.solve(S, G, oracle.Params(eps=0.0, fixed_iters=False, max_iter=7))
    assert it == 7


def test_invalid_parameters_are_rejected():
    _, S, G = synth_case()
    for p in (oracle.Params(alpha=0.0), oracle.Params(beta=-1.0), oracle.Params(max_iter=0)):
        with pytest.raises(oracle.OracleError):
            oracle.solve(S, G, p)


def test_model_estimate_tracks_observed_histogram():
    """Fig. 3: the histogram estimated from H_C(R), H_C(L) through the class map (Eq. 8)
    approximates H_C(S) after the optimisation."""
    _, S, G = synth_case(W=160, H=120)
    R, L, _ = oracle.solve(S, G, oracle.Params(alpha=1e-4, beta=1e-4))
    N = float(S.sum())
    idx = brute.class_map(256)
    E = np.zeros(256)
    np.add.at(E, idx.ravel(), (np.outer(R, L) / N).ravel())
    R0, L0 = G.astype(np.float64), S.astype(np.float64)
    E0 = np.zeros(256)
    np.add.at(E0, idx.ravel(), (np.outer(R0, L0) / N).ravel())
    err = np.abs(E - S).sum() / N
    err0 = np.abs(E0 - S).sum() / N
    assert err < err0  # the optimisation moves the estimate towards H_C(S)
