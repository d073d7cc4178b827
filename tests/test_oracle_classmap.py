"""Pins for the class maps: index(i,j) (definition under Eq. 10) and index_1 (Eq. 17-19)."""
import math

import numpy as np
import pytest

import brute
import oracle


@pytest.mark.parametrize("K", [8, 16, 256])
def test_closed_form_class_index_equals_fp64_argmin(K):
    want = brute.class_map(K)
    got = np.array([[oracle.class_index(K, i, j) for j in range(K)] for i in range(K)])
    assert np.array_equal(got, want)


def test_class_index_has_no_ties_and_partitions_cells():
    for K in (8, 256, 4096):
        km1 = K - 1
        i = np.arange(K)[:, None]
        j = np.arange(K)[None, :]
        two_ij = 2 * i * j
        # a tie would need 2ij = (2k+1)(K-1): even vs odd
        assert (two_ij % 2 == 0).all() and km1 % 2 == 1
        cls = (two_ij + km1) // (2 * km1)
        assert np.bincount(cls.ravel(), minlength=K).sum() == K * K
        assert cls.max() == K - 1 and cls.min() == 0


def test_class_index_large_K_sampled():
    K = 4096
    rng = np.random.default_rng(0)
    loc = np.arange(K) / (K - 1)
    for _ in range(2000):
        i, j = (int(v) for v in rng.integers(0, K, 2))
        p = loc[i] * loc[j]
        k = int(np.argmin(np.abs(p - loc)))
        assert oracle.class_index(K, i, j) == k


@pytest.mark.parametrize("K,gamma", [(8, 2.2), (16, 1.5), (256, 2.2), (256, 5.0)])
def test_index1_equals_literal_argmin(K, gamma):
    assert np.array_equal(oracle.index1_table(K, gamma), brute.class_map_gamma(K, gamma))


def test_index1_large_K_sampled():
    K, gamma = 4096, 2.2
    t = oracle.index1_table(K, gamma)
    rng = np.random.default_rng(1)
    loc = np.arange(K) / (K - 1)
    for _ in range(2000):
        i, j = (int(v) for v in rng.integers(0, K, 2))
        p = math.pow(j / (K - 1), 1 / gamma) * loc[i]
        assert t[i, j] == int(np.argmin(np.abs(p - loc)))


@pytest.mark.parametrize("K", [8, 256])
def test_index1_with_gamma_one_is_index(K):
    t = oracle.index1_table(K, 1.0)
    assert np.array_equal(t, brute.class_map(K))


def test_index1_monotone_in_each_argument():
    t = oracle.index1_table(256, 2.2).astype(np.int64)
    assert (np.diff(t, axis=0) >= 0).all() and (np.diff(t, axis=1) >= 0).all()
    # gamma > 1 raises every illumination location, so no cell moves to a darker class than index(i,j)
    assert (t >= brute.class_map(256)).all()
