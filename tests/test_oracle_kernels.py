"""Pins for the oracle's kernel-descriptor weighted covariance (Sec. III-C1,
Table I), against facts fixed outside it.

* constant weights (RBF with sigma = 0; a constant polynomial) reduce it to
  the plain neighbourhood covariance;
* two neighbours with known weights have the closed form
  C = w1 w2 / (w1 + w2)^2 (p1 - p2)(p1 - p2)^T; the weights themselves are
  chosen where each kernel of Table I takes a value fixed by its definition
  (1/2 at unit distance for RBF, Gaussian and Laplacian with sigma picked
  for it; exact integers and fractions for Polynomial and HI);
* scaling every weight by the same factor changes nothing;
* a zero total weight gives NaN.
The paper gives no formula for how the kernel enters the covariance and no
worked example, so the weighted form itself is a reading (parity with the
paper unpinned); these pins fix the oracle to that reading.
"""
import math

import numpy as np
import pytest

import oracle


def test_constant_weights_reduce_to_the_plain_covariance():
    rng = np.random.default_rng(1)
    p = (rng.random((200, 3)) * 5).astype(np.float32)
    q = (rng.random((30, 3)) * 5).astype(np.float32)
    idx, _ = oracle.knn_brute(q, p, 12)
    plain = oracle.cov(p, idx, -1.0)
    a = oracle.cov_weighted(p, q, idx, -1.0, "rbf", sigma=0.0)
    b = oracle.cov_weighted(p, q, idx, -1.0, "polynomial", alpha=0.0, c=2.0, d=3.0)
    np.testing.assert_allclose(a, plain, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b, plain, rtol=1e-12, atol=1e-15)
    reg = oracle.cov(p, idx, 1e-3)
    np.testing.assert_allclose(oracle.cov_weighted(p, q, idx, 1e-3, "rbf", sigma=0.0), reg, rtol=1e-12,
                               atol=1e-12)


def _two_point(kernel, q, p1, p2, w1, w2, **kw):
    p = np.array([p1, p2], np.float32)
    C = oracle.cov_weighted(p, np.array([q], np.float32), np.array([[0, 1]], np.int32), -1.0, kernel, **kw)[0]
    dl = np.asarray(p1, np.float64) - np.asarray(p2, np.float64)
    want = w1 * w2 / (w1 + w2) ** 2 * np.outer(dl, dl)
    got = oracle.unpack6(C)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


def test_two_neighbours_closed_form_per_kernel():
    q, p1, p2 = [1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [1.0, 1.0, 0.0]  # distances 0 and 1
    _two_point("rbf", q, p1, p2, 1.0, 0.5, sigma=math.log(2.0))
    _two_point("gaussian", q, p1, p2, 1.0, 0.5, sigma=1.0 / math.sqrt(2.0 * math.log(2.0)))
    _two_point("laplacian", q, p1, p2, 1.0, 0.5, sigma=1.0 / math.log(2.0))
    # Polynomial (alpha <x', y'> + c)^d, origin 0: <q, p1> = 1, <q, p2'> = 2
    _two_point("polynomial", [1.0, 0, 0], [1.0, 0, 0], [2.0, 0.5, 0], 1.0, 4.0, alpha=1.0, c=0.0, d=2.0)
    # HI: q' = (1,1,1); p1' = q' -> 3/3; p2' = (0,1,3) -> (0+1+1)/3 (the sum
    # of q', not of p2', is the denominator)
    _two_point("hi", [1.0, 1, 1], [1.0, 1, 1], [0.0, 1, 3], 1.0, 2.0 / 3.0)
    # the origin shifts Polynomial/HI coordinates: the same points 10 m away
    # from an origin placed 10 m away give the same answer
    o = (10.0, -3.0, 2.0)
    sh = lambda v: [v[0] + o[0], v[1] + o[1], v[2] + o[2]]
    _two_point("hi", sh([1.0, 1, 1]), sh([1.0, 1, 1]), sh([0.0, 1, 3]), 1.0, 2.0 / 3.0, origin=o)


def test_common_weight_scale_cancels_and_zero_weight_is_nan():
    rng = np.random.default_rng(2)
    p = (rng.random((100, 3)) * 4 + 1).astype(np.float32)
    q = (rng.random((10, 3)) * 4 + 1).astype(np.float32)
    idx, _ = oracle.knn_brute(q, p, 9)
    a = oracle.cov_weighted(p, q, idx, -1.0, "polynomial", alpha=1.0, c=0.5, d=1.0)
    b = oracle.cov_weighted(p, q, idx, -1.0, "polynomial", alpha=7.0, c=3.5, d=1.0)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)
    z = oracle.cov_weighted(p, q, idx, -1.0, "polynomial", alpha=0.0, c=0.0, d=1.0)
    assert np.isnan(z).all()


def test_bad_arguments():
    p = np.zeros((3, 3), np.float32)
    with pytest.raises(ValueError):
        oracle.cov_weighted(p, np.zeros((1, 3), np.float32), np.array([[0, 5]], np.int32), -1.0, "rbf")
