"""Pins for the independent Metropolis-Hastings sweep (SMC-IRMH): its acceptance ratio
against the densities written out with scipy, exact acceptance when the proposal is the
target, the whitened norm against a direct solve, invariance of the tempered free field
under sweeps with a mismatched proposal, and the free-field evidence."""
import math

import numpy as np
import pytest
import scipy.stats

import closed_forms as cf
from oracle import irmh, lattice, mutation, philox
from oracle.smc import SMC, SMCConfig


def _spd(D, seed):
    g = np.random.default_rng(seed)
    B = g.standard_normal((D, D)) / math.sqrt(D)
    return B @ B.T + 0.5 * np.eye(D)


@pytest.mark.parametrize("keep_reference", [False, True])
def test_log_alpha_is_the_metropolis_hastings_ratio(keep_reference):
    L, N = 3, 40
    D = L * L
    g = np.random.default_rng(1)
    Sigma = _spd(D, 2)
    Lc = np.linalg.cholesky(Sigma)
    mu = 0.3 * g.standard_normal(D)
    phi = mu + g.standard_normal((N, D)) @ Lc.T * 1.3
    beta = 0.37
    S, sq = lattice.action(phi, L, -4.0, 8.0), lattice.sq_norm(phi)
    r = irmh.whitened_sq_norm(phi, mu, Lc)
    _, _, _, _, _, la = irmh.irmh_sweep(phi, S, sq, r, Lc, mu, beta, L, -4.0, 8.0, 1.0, 1.0, keep_reference,
                                        7, 0, 3, 1)
    Z = philox.normals(7, 0, philox.KIND_PROPOSE, 3, 1, N, D, bits=32)
    prop = mu + Z @ Lc.T

    def log_gamma(x):  # tempered target up to its constant
        Sx, qx = lattice.action(x, L, -4.0, 8.0), lattice.sq_norm(x)
        return -beta * Sx - 0.5 * qx if keep_reference else -beta * Sx - (1 - beta) * 0.5 * qx
    q = scipy.stats.multivariate_normal(mean=mu, cov=Sigma)
    want = log_gamma(prop) - log_gamma(phi) + q.logpdf(phi) - q.logpdf(prop)
    np.testing.assert_allclose(la, want, rtol=1e-9, atol=1e-9)


def test_exact_proposal_is_always_accepted():
    # beta = 0 without the reference kept: the target is N(0, I); with q = N(0, I) too,
    # log alpha is zero up to rounding and every proposal is accepted
    L, N = 2, 64
    D = L * L
    phi = np.random.default_rng(3).standard_normal((N, D))
    S, sq = lattice.action(phi, L, -4.0, 8.0), lattice.sq_norm(phi)
    r = irmh.whitened_sq_norm(phi, np.zeros(D), np.eye(D))
    _, _, _, _, acc, la = irmh.irmh_sweep(phi, S, sq, r, np.eye(D), np.zeros(D), 0.0, L, -4.0, 8.0, 1.0, 1.0,
                                          False, 1, 0, 1, 0)
    assert np.abs(la).max() < 1e-12 and acc.all()


def test_whitened_norm_is_the_mahalanobis_distance():
    D = 6
    Sigma = _spd(D, 4)
    Lc = np.linalg.cholesky(Sigma)
    g = np.random.default_rng(5)
    mu, phi = g.standard_normal(D), g.standard_normal((5, D))
    Xc = phi - mu
    want = np.einsum("nd,de,ne->n", Xc, np.linalg.inv(Sigma), Xc)
    np.testing.assert_allclose(irmh.whitened_sq_norm(phi, mu, Lc), want, rtol=1e-12)


def test_irmh_free_field_evidence():
    # free field lambda = 0, m2 = 1 on the 2 x 2 torus: closed form; the Gaussian proposal
    # fits a Gaussian target, so the estimate is tight
    lz = np.array([SMC(SMCConfig(L=2, N=2048, m2=1.0, lam=0.0, rho=0.9, n_mcmc=5, seed=s, inner="irmh")).run()["logz"]
                   for s in range(6)])
    ref = cf.free_field_logz(2, 1.0)
    se = lz.std(ddof=1) / math.sqrt(len(lz))
    assert abs(lz.mean() + 0.5 * lz.var(ddof=1) - ref) < 4.0 * se + 0.01


@pytest.mark.parametrize("keep_reference", [False, True])
def test_invariance_free_field(keep_reference):
    # exact draws from gamma_beta of the free field stay distributed as gamma_beta under
    # independence sweeps whose Gaussian proposal is shifted and 1.5 x too wide: only the
    # Hastings factor q(phi) / q(phi') keeps E|phi|^2 and Var M where they are
    L, m2, beta, N = 3, 1.0, 0.6, 20000
    D = L * L
    g = np.random.default_rng(22)
    C = cf.free_field_covariance(L, m2, beta, keep_reference)
    phi = g.standard_normal((N, D)) @ np.linalg.cholesky(C).T
    want_sq, want_varM = float(np.trace(C)), float(C.sum()) / D ** 2
    S, sq = lattice.action(phi, L, m2, 0.0), lattice.sq_norm(phi)
    mu = 0.1 * np.ones(D)
    Lc = np.linalg.cholesky(1.5 * C)
    r = irmh.whitened_sq_norm(phi, mu, Lc)
    accs = []
    for s in range(6):
        phi, S, sq, r, acc, _ = irmh.irmh_sweep(phi, S, sq, r, Lc, mu, beta, L, m2, 0.0, 1.0, 1.0, keep_reference,
                                                4, 0, 1, s)
        accs.append(acc.mean())
    assert 0.2 < min(accs) and max(accs) < 0.95, accs
    assert abs(sq.mean() - want_sq) < 4 * math.sqrt(np.var(sq) / N), (sq.mean(), want_sq)
    varM = phi.mean(axis=1).var()
    assert abs(varM - want_varM) < 4 * want_varM * math.sqrt(2.0 / N), (varM, want_varM)
    np.testing.assert_allclose(r, irmh.whitened_sq_norm(phi, mu, Lc), rtol=1e-10)
