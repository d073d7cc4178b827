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
