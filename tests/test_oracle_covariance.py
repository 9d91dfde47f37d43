"""Pins for the particle covariance and the Cholesky factor."""
import numpy as np
import pytest

import inputs
from oracle import covariance


def test_sample_covariance_matches_numpy_cov_and_two_point_case():
    X = inputs.fields(50, 7, seed=2)
    mu, S = covariance.sample_covariance(X)
    np.testing.assert_allclose(mu, X.mean(0), rtol=1e-14)
    np.testing.assert_allclose(S, np.cov(X, rowvar=False), rtol=1e-12, atol=1e-14)
    # two particles a, b: Sigma = (a - b)(a - b)^T / 2
    a, b = np.array([1.0, 2.0, -1.0]), np.array([0.0, -1.0, 3.0])
    _, S2 = covariance.sample_covariance(np.stack([a, b]))
    np.testing.assert_allclose(S2, np.outer(a - b, a - b) / 2, rtol=1e-15)


def test_cholesky_known_factor():
    for D in (1, 5, 64):
        B = inputs.lower_factor(D, seed=D)
        L = covariance.cholesky_lower(B @ B.T)
        np.testing.assert_allclose(L, B, rtol=1e-10, atol=1e-12)


def test_regularised_cholesky_rank_deficient():
    X = inputs.fields(5, 12, seed=1)  # N < D: rank 4
    _, S = covariance.sample_covariance(X)
    L, delta, tries, level = covariance.regularised_cholesky(S, 1e-8)
    assert delta > 0 and tries >= 1 and level == tries - 1
    np.testing.assert_allclose(L @ L.T, S + delta * np.eye(12), rtol=1e-8, atol=1e-10 * np.trace(S))
    assert delta == pytest.approx(1e-8 * np.trace(S) / 12 * 10 ** (tries - 1), rel=1e-12)
    # a later step starts from the level that worked
    L2, delta2, tries2, level2 = covariance.regularised_cholesky(S, 1e-8, start_level=level)
    assert tries2 == 1 and level2 == level and delta2 == pytest.approx(delta, rel=1e-12)
    # an SPD matrix at a raised level keeps that level and its larger ridge
    A = inputs.spd_matrix(6, seed=2)
    _, d3, t3, l3 = covariance.regularised_cholesky(A, 1e-8, start_level=3)
    assert t3 == 1 and l3 == 3 and d3 == pytest.approx(1e-5 * np.trace(A) / 6, rel=1e-12)
