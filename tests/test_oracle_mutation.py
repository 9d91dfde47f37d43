"""Pins for the random-walk Metropolis step: proposal covariance, accept rule
and invariance of the tempered free-field target."""
import math

import numpy as np
import pytest

import closed_forms as cf
import inputs
from oracle import lattice, mutation, philox


def test_proposal_increment_covariance_is_s2_LLT():
    # catches a transposed factor: Cov(phi' - phi) must be s^2 L L^T, not s^2 L^T L
    D, N, s = 3, 200000, 0.7
    Lc = np.array([[1.0, 0.0, 0.0], [0.8, 0.5, 0.0], [-0.3, 0.9, 0.2]])
    Z = philox.normals(5, 0, philox.KIND_PROPOSE, 1, 0, N, D)
    inc = mutation.propose(np.zeros((N, D)), Z, Lc, s)
    C = np.cov(inc, rowvar=False)
    want = s * s * Lc @ Lc.T
    assert np.abs(C - want).max() < 0.02
    assert np.abs(C - s * s * Lc.T @ Lc).max() > 0.1


def test_accept_rule_signs():
    L, m2, lam = 2, -4.0, 8.0
    phi = np.full((1, 4), 0.9)          # far outside the wells: high action
    prop = np.full((1, 4), 0.5)         # at the well bottom, lower action and norm
    S = lattice.action(phi, L, m2, lam)
    sq = lattice.sq_norm(phi)
    for beta in (0.0, 0.3, 1.0):
        _, _, _, acc, S2, sq2, la = mutation.accept(phi, S, sq, prop, np.log(np.array([1.0 - 1e-12])), beta,
                                                   L, m2, lam, 1.0, 1.0)
        assert la[0] > 0 and acc[0]
        want = -beta * (S2[0] - S[0]) - (1 - beta) * 0.5 * (sq2[0] - sq[0])
        assert la[0] == pytest.approx(want, rel=1e-14)
    # the reverse move is rejected when log u is below zero but above log alpha
    _, _, _, acc, _, _, la = mutation.accept(prop, lattice.action(prop, L, m2, lam), lattice.sq_norm(prop), phi,
                                             np.array([-1e-9]), 1.0, L, m2, lam, 1.0, 1.0)
    assert la[0] < -1e-9 and not acc[0]


@pytest.mark.parametrize("keep_reference", [False, True])
def test_invariance_free_field(keep_reference):
    # exact draws from gamma_beta stay distributed as gamma_beta under the sweep
    L, m2, beta, N = 4, 1.0, 0.6, 20000
    D = L * L
    g = inputs.rng(12)
    if keep_reference:
        # gamma_beta = N(0, I) exp(-beta S): quadratic form 1/2 + beta P, i.e. the free field of
        # "beta" -> treat via explicit covariance
        A = np.linalg.inv(2 * (0.5 * np.eye(D) + beta * free_field_matrix(L, m2)))
        phi = g.standard_normal((N, D)) @ np.linalg.cholesky(A).T
        want_sq = np.trace(A)
    else:
        phi = cf.free_field_sample(L, m2, beta, N, g)
        want_sq = cf.free_field_sq_mean(L, m2, beta)
    S = lattice.action(phi, L, m2, 0.0)
    sq = lattice.sq_norm(phi)
    Lc = np.linalg.cholesky(np.cov(phi, rowvar=False))
    for s in range(8):
        phi, S, sq, acc = mutation.rw_sweep(phi, S, sq, Lc, 2.38 / math.sqrt(D), beta, L, m2, 0.0, 1.0, 1.0,
                                            keep_reference, 3, 0, 1, s)
    assert 0.1 < acc.mean() < 0.6
    se = math.sqrt(np.var(sq) / N) * 3.0   # chains are correlated with their start; generous factor
    assert abs(sq.mean() - want_sq) < 4 * se
    # cached S and |phi|^2 are those of the current fields
    np.testing.assert_allclose(S, lattice.action(phi, L, m2, 0.0), rtol=1e-12)
    np.testing.assert_allclose(sq, lattice.sq_norm(phi), rtol=1e-12)


def free_field_matrix(L, m2):
    D = L * L
    A = np.zeros((D, D))
    for r in range(L):
        for c in range(L):
            x = r * L + c
            A[x, x] += 4.0 + m2
            for (rr, cc) in ((r, (c + 1) % L), (r, (c - 1) % L), ((r + 1) % L, c), ((r - 1) % L, c)):
                A[x, rr * L + cc] -= 1.0
    return A
