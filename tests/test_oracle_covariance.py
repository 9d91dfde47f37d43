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


@pytest.mark.parametrize("L,beta,keep", [(1, 0.5, False), (2, 0.3, False), (3, 1.0, False), (4, 0.7, True),
                                         (5, 0.0, False)])
def test_gaussian_part_covariance_inverts_the_hessian_of_the_tempered_target(L, beta, keep):
    # P = Sigma^{-1} must be the Hessian of beta S + a |phi|^2 / 2 (lambda = 0), here taken by
    # second differences of the oracle's own action (exact for a quadratic up to rounding)
    from oracle import lattice
    m2, c_kin, c_mass = 1.3, 0.7, 0.9
    D = L * L
    a = 1.0 if keep else 1.0 - beta

    def f(x):
        S = lattice.action(x[None, :], L, m2, 0.0, c_kin, c_mass)[0]
        return beta * S + 0.5 * a * float(x @ x)
    E = np.eye(D)
    H = np.array([[f(E[i] + E[j]) - f(E[i]) - f(E[j]) + f(np.zeros(D)) for j in range(D)] for i in range(D)])
    Sigma = covariance.gaussian_part_covariance(L, beta, m2, c_kin, c_mass, keep)
    np.testing.assert_allclose(Sigma @ H, np.eye(D), atol=1e-11)


def test_gaussian_part_covariance_spectrum_is_the_closed_form():
    # eigenvalues 1 / (a + 2 beta p_k), p_k = c_mass m2 + c_kin sum_mu 4 sin^2(pi k_mu / L)
    import closed_forms as cf
    L, beta, m2 = 6, 0.4, 0.8
    Sigma = covariance.gaussian_part_covariance(L, beta, m2)
    p = m2 + cf.lattice_laplacian_eigs(L)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(Sigma)), np.sort(1.0 / (1.0 - beta + 2.0 * beta * p)),
                               rtol=1e-12)
    np.testing.assert_allclose(Sigma, cf.free_field_covariance(L, m2, beta), rtol=1e-12, atol=1e-15)
