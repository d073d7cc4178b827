"""Literal, independent restatement of the HistRetinex pipeline for pinning the oracle.

Written from the paper's equations with the matrices materialised (numpy, FP64):
the count matrix (Eq. 6), the location matrix (Eq. 7, without the printed /N),
the class map as a literal FP64 argmin (definition under Eq. 10), the weights K_ij
(Eq. 11), the minimiser of Eq. 10 in R and in L (Eq. 13, Eq. 12 with the weight
multiplying), renormalisation (Eq. 14/15), the gamma-processed location matrix and
index_1 (Eq. 17-19), the enhanced histogram (Eq. 20), histogram matching by brute-force
search and the HSV value replacement by exact rational rounding.  It shares no code with
the oracle and uses a different evaluation order (numpy reductions), so agreement is
up to rounding only.  Only suitable for small K and tiny images.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def value_channel(img):
    return img.astype(np.int64).max(axis=2)


def sobel_levels(V, K):
    P = np.pad(V.astype(np.int64), 1, mode="edge")
    H, W = V.shape
    win = lambda dy, dx: P[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
    gx = (win(-1, 1) + 2 * win(0, 1) + win(1, 1)) - (win(-1, -1) + 2 * win(0, -1) + win(1, -1))
    gy = (win(1, -1) + 2 * win(1, 0) + win(1, 1)) - (win(-1, -1) + 2 * win(-1, 0) + win(-1, 1))
    out = np.zeros_like(V, dtype=np.int64)
    for y in range(H):
        for x in range(W):
            m2 = int(gx[y, x]) ** 2 + int(gy[y, x]) ** 2
            n = math.isqrt(m2)
            g = n + 1 if 4 * m2 >= (2 * n + 1) ** 2 else n  # nearest integer to sqrt(m2), halves up
            out[y, x] = min(g, K - 1)
    return out


def histograms(img, K):
    V = value_channel(img)
    S = np.bincount(V.ravel(), minlength=K).astype(np.int64)
    G = np.bincount(sobel_levels(V, K).ravel(), minlength=K).astype(np.int64)
    return S, G


def locations(K):
    return np.arange(K, dtype=np.float64) / (K - 1)


def class_map(K):
    """index(i, j) = argmin_k |H_B(R)_i H_B(L)_j - H_B(S)_k| (first minimum)."""
    loc = locations(K)
    hlm = np.outer(loc, loc)
    return np.argmin(np.abs(hlm[:, :, None] - loc[None, None, :]), axis=2)


def class_map_gamma(K, gamma):
    """index_1(i, j) with the illumination locations raised to 1/gamma (Eq. 17-19)."""
    loc = locations(K)
    lbar = np.array([math.pow(x, 1.0 / gamma) for x in loc])
    hlm = np.outer(loc, lbar)  # rows: reflectance bin i, columns: illumination bin j
    return np.argmin(np.abs(hlm[:, :, None] - loc[None, None, :]), axis=2)


def weights(R, L, idx, N):
    """K_ij = H_C(L,R)_ij / sum over the class of idx(i,j) (Eq. 11); 0 for an empty class."""
    hcm = np.outer(R, L) / N
    K = len(R)
    tot = np.zeros(K)
    np.add.at(tot, idx.ravel(), hcm.ravel())
    den = tot[idx]
    W = np.zeros_like(hcm)
    nz = den > 0
    W[nz] = hcm[nz] / den[nz]
    return W


def iterate_literal(S, G, R, L, alpha, beta, idx):
    """One pass of Algorithm 1 with the matrices materialised; returns (Ru, Lu, Rn, Ln, Kmat)."""
    S = np.asarray(S, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    N = S.sum()
    Km = weights(R, L, idx, N)
    Sidx = S[idx]
    Ru = ((Km * Sidx * L[None, :]).sum(axis=1) / N + beta * G) / ((L * L).sum() / N**2 + beta)
    Lu = ((Km * Sidx * Ru[:, None]).sum(axis=0) / N + alpha * S) / ((Ru * Ru).sum() / N**2 + alpha)
    Rn = N * Ru / Ru.sum()
    Ln = N * Lu / Lu.sum()
    return Ru, Lu, Rn, Ln, Km


def objective_eq10(Rv, Lv, Km, S, G, idx, alpha, beta):
    """J of Eq. 10 (all bins) for given histograms and fixed weights."""
    S = np.asarray(S, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    N = S.sum()
    data = (np.outer(Rv, Lv) / N - Km * S[idx]) ** 2
    return data.sum() + alpha * ((Lv - S) ** 2).sum() + beta * ((Rv - G) ** 2).sum()


def solve(S, G, K, alpha, beta, T):
    idx = class_map(K)
    R = np.asarray(G, dtype=np.float64).copy()
    L = np.asarray(S, dtype=np.float64).copy()
    for _ in range(T):
        _, _, R, L, _ = iterate_literal(S, G, R, L, alpha, beta, idx)
    return R, L


def target(R, L, K, gamma, N):
    idx1 = class_map_gamma(K, gamma)
    hcm = np.outer(R, L) / N
    T = np.zeros(K)
    np.add.at(T, idx1.ravel(), hcm.ravel())
    return T


def lut(S, T):
    """Smallest z whose target CDF reaches the source CDF: CT(z) / CT(K-1) >= CS(s) / N, decided
    in exact rational arithmetic over the given (double) target values."""
    K = len(S)
    N = int(np.sum(S))
    CT, acc = [], Fraction(0)
    for t in T:
        acc += Fraction(float(t))
        CT.append(acc)
    TT = CT[-1]
    CS = np.cumsum(np.asarray(S, dtype=np.int64))
    out = np.zeros(K, dtype=np.int64)
    for s in range(K):
        z = 0
        while z < K - 1 and not (CT[z] * N >= int(CS[s]) * TT):
            z += 1
        out[s] = z
    return out


def apply(img, lut_):
    """Replace V by V' = LUT[V] keeping hue and saturation: c -> nearest integer to c V'/V (halves up)."""
    H, W, _ = img.shape
    out = np.zeros_like(img)
    for y in range(H):
        for x in range(W):
            c = [int(v) for v in img[y, x]]
            V = max(c)
            Vp = int(lut_[V])
            if V == 0:
                out[y, x] = (Vp, Vp, Vp)
            else:
                out[y, x] = [math.floor(Fraction(ch * Vp, V) + Fraction(1, 2)) for ch in c]
    return out


# ---- printed forms of three readings (selectable variants) ----

def forward_levels(V, K):
    """Gradient levels from forward differences gx = V(x+1,y) - V(x,y), gy = V(x,y+1) - V(x,y)
    (replicate border: zero at the last column / row), magnitude rounded half up, clipped."""
    P = np.pad(V.astype(np.int64), ((0, 1), (0, 1)), mode="edge")
    H, W = V.shape
    gx = P[:H, 1:W + 1] - P[:H, :W]
    gy = P[1:H + 1, :W] - P[:H, :W]
    out = np.zeros_like(V, dtype=np.int64)
    for y in range(H):
        for x in range(W):
            m2 = int(gx[y, x]) ** 2 + int(gy[y, x]) ** 2
            n = math.isqrt(m2)
            out[y, x] = min(n + 1 if 4 * m2 >= (2 * n + 1) ** 2 else n, K - 1)
    return out


def iterate_printed_exact(S, G, R, L, alpha, beta, idx):
    """One pass of Algorithm 1 with Eq. 13 and Eq. 12 exactly as printed (the weight K_ij divides),
    in exact rational arithmetic over the given double inputs: K_ij = HCM_ij / class total
    (Eq. 11, HCM_ij = R_i L_j / N by Eq. 6); a cell with zero weight contributes nothing.
    Returns (Ru, Lu) as lists of Fractions."""
    K = len(S)
    N = Fraction(int(np.sum(S)))
    Rf = [Fraction(float(x)) for x in R]
    Lf = [Fraction(float(x)) for x in L]
    Sf = [Fraction(int(x)) for x in S]
    Gf = [Fraction(int(x)) for x in G]
    hcm = [[Rf[i] * Lf[j] / N for j in range(K)] for i in range(K)]
    tot = [Fraction(0)] * K
    for i in range(K):
        for j in range(K):
            tot[idx[i][j]] += hcm[i][j]
    W = [[(hcm[i][j] / tot[idx[i][j]]) if tot[idx[i][j]] != 0 else Fraction(0) for j in range(K)] for i in range(K)]
    dR = sum(x * x for x in Lf) / (N * N) + Fraction(beta)
    Ru = []
    for i in range(K):
        a = sum((Lf[j] * Sf[idx[i][j]] / (N * W[i][j]) for j in range(K) if W[i][j] != 0), Fraction(0))
        Ru.append((a + Fraction(beta) * Gf[i]) / dR)
    dL = sum(x * x for x in Ru) / (N * N) + Fraction(alpha)
    Lu = []
    for j in range(K):
        b = sum((Ru[i] * Sf[idx[i][j]] / (N * W[i][j]) for i in range(K) if W[i][j] != 0), Fraction(0))
        Lu.append((b + Fraction(alpha) * Sf[j]) / dL)
    return Ru, Lu


def lut_nearest(S, T):
    """Target level whose cumulative share is nearest to the source level's: the first z minimising
    |CT(z) N - CS(s) TT| in exact rational arithmetic over the given (double) target values; the
    last occupied target level where CS(s) = N."""
    K = len(S)
    N = int(np.sum(S))
    CT, acc = [], Fraction(0)
    for t in T:
        acc += Fraction(float(t))
        CT.append(acc)
    TT = CT[-1]
    top = max(z for z in range(K) if T[z] > 0)
    CS = np.cumsum(np.asarray(S, dtype=np.int64))
    out = np.zeros(K, dtype=np.int64)
    for s in range(K):
        if int(CS[s]) == N:
            out[s] = top
            continue
        d = [abs(CT[z] * N - int(CS[s]) * TT) for z in range(K)]
        out[s] = d.index(min(d))
    return out


# ---- binned data: K bins over M data levels ----

def bin_locations_exact(K, M):
    """Bin centre values normalised to [0, 1], as exact rationals: (k w + (w - 1)/2) / (M - 1)."""
    w = M // K
    return [Fraction(2 * k * w + w - 1, 2 * (M - 1)) for k in range(K)]


def nearest_exact(p, locs):
    """(first k minimising |p - loc_k|, whether the minimum is shared by two levels), exactly."""
    d = [abs(p - x) for x in locs]
    m = min(d)
    ks = [k for k, v in enumerate(d) if v == m]
    return ks[0], len(ks) > 1


def class_map_binned_float(K, M, gamma=None):
    """Class map (gamma None) or index_1 map over the bin locations by a literal FP64 argmin."""
    w = M // K
    loc = np.array([(2 * k * w + w - 1) / (2.0 * (M - 1)) for k in range(K)])
    lj = loc if gamma is None else np.array([math.pow(x, 1.0 / gamma) for x in loc])
    hlm = np.outer(loc, lj)
    return np.argmin(np.abs(hlm[:, :, None] - loc[None, None, :]), axis=2)


def histograms_binned(img, K, M):
    V = value_channel(img)
    sh = int(round(math.log2(M // K)))
    S = np.bincount((V >> sh).ravel(), minlength=K).astype(np.int64)
    G = np.bincount((sobel_levels(V, M) >> sh).ravel(), minlength=K).astype(np.int64)
    return S, G


def apply_binned(img, lut_, K, M):
    """V' = LUT[s] w + (V - s w) (s = V >> log2 w); channels c -> nearest integer to c V'/V, halves up."""
    sh = int(round(math.log2(M // K)))
    H, W, _ = img.shape
    out = np.zeros_like(img)
    for y in range(H):
        for x in range(W):
            c = [int(v) for v in img[y, x]]
            V = max(c)
            s = V >> sh
            Vp = (int(lut_[s]) << sh) + (V - (s << sh))
            if V == 0:
                out[y, x] = (Vp, Vp, Vp)
            else:
                out[y, x] = [math.floor(Fraction(ch * Vp, V) + Fraction(1, 2)) for ch in c]
    return out
