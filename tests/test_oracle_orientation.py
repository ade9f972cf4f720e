"""Orientation averaging (Eqs. 5-6) in the oracle's sampler.

The quadrature form of Eq. 5 puts trajectory j at the node j mod K of a
K-point Gauss-Legendre rule in x = cos(theta) on [0, 1] and scales its weight
by K W_k.  Pinned here against numpy's Gauss-Legendre rule, polynomial
exactness, and trajectory by trajectory against the fixed-angle sampler at
the node's angle (the same random draws, so the same t0, k_perp and exit).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W


@pytest.mark.parametrize("K", [1, 2, 5, 10, 64])
def test_nodes_are_gauss_legendre_on_unit_interval(K):
    x, w = O.quad_nodes(K)
    X, Wt = np.polynomial.legendre.leggauss(K)
    assert np.all(np.diff(x) < 0)                        # descending
    assert np.allclose(np.sort(x), np.sort(0.5 * (X + 1.0)), rtol=0, atol=1e-15)
    assert np.allclose(np.sort(w), np.sort(0.5 * Wt), rtol=0, atol=1e-14)
    # exact for polynomials up to degree 2K - 1 on [0, 1]
    for m in range(2 * K):
        assert abs(np.dot(w, x ** m) - 1.0 / (m + 1)) <= 1e-14


def test_quadrature_sample_is_the_fixed_sample_at_the_node():
    t, p, K, n, seed, inst = W.TARGETS["H2"], W.PULSE_800, 5, 40, 9, 2
    soa, _, bad = O.sample(t, p, W.quadrature(K), seed=seed, instance=inst, n=n)
    x, w = O.quad_nodes(K)
    for j in range(n):
        k = j % K
        nh = soa[7:10, j]
        assert abs(nh[2] - x[k]) <= 1e-15
        phi = math.atan2(nh[1], nh[0])
        one, _, _ = O.sample(t, p, (W.ALIGN_FIXED, math.acos(x[k]), phi), seed=seed,
                             instance=inst, j_begin=j, n=1)
        assert np.array_equal(one[0:7, 0], soa[0:7, j])          # birth, exit, momentum
        assert np.allclose(one[7:10, 0], nh, rtol=0, atol=1e-15)
        wq = soa[10, j] + 1j * soa[11, j]
        wf = one[10, 0] + 1j * one[11, 0]
        assert abs(wq - K * w[k] * wf) <= 1e-12 * abs(wf) + 1e-300


def test_bad_node_count_is_refused():
    t, p = W.TARGETS["H2"], W.PULSE_800
    for K in (0, 65):
        with pytest.raises(ValueError):
            O.sample(t, p, W.quadrature(K), n=4)
