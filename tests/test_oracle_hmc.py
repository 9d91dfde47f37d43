"""Pins for the HMC transition (SMC-HMC): the gradients of the action and of the tempered
log-target against finite differences of the independently written action and target,
leapfrog reversibility and its second-order energy error,
near-certain acceptance for small steps, invariance of the tempered free field under the
transition, and the free-field evidence."""
import math

import numpy as np
import pytest

import closed_forms as cf
from oracle import hmc, lattice
from oracle.smc import SMC, SMCConfig


@pytest.mark.parametrize("L,c", [(3, (1.0, 1.0)), (4, (0.5, 0.5)), (2, (1.0, 1.0)), (1, (1.0, 1.0))])
def test_gradient_matches_finite_differences(L, c):
    g = np.random.default_rng(L)
    phi = g.standard_normal((3, L * L))
    grad = hmc.grad_action(phi, L, -4.0, 8.0, *c)
    h = 1e-6
    for x in range(L * L):
        e = np.zeros(L * L)
        e[x] = h
        fd = (lattice.action(phi + e, L, -4.0, 8.0, *c) - lattice.action(phi - e, L, -4.0, 8.0, *c)) / (2 * h)
        np.testing.assert_allclose(grad[:, x], fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("keep_reference", [False, True])
def test_target_gradient_matches_finite_differences(keep_reference):
    # the force of the leapfrog map is the gradient of the tempered log-target as a whole,
    # reference term included: -beta grad S - a phi with a = 1 - beta (1 with the reference kept)
    L, beta = 3, 0.37
    phi = np.random.default_rng(4).standard_normal((2, L * L))
    grad = hmc.grad_log_target(phi, beta, L, -4.0, 8.0, 1.0, 1.0, keep_reference)

    def log_gamma(q):
        return lattice.log_target(lattice.action(q, L, -4.0, 8.0), lattice.sq_norm(q), beta, keep_reference)
    h = 1e-6
    for x in range(L * L):
        e = np.zeros(L * L)
        e[x] = h
        fd = (log_gamma(phi + e) - log_gamma(phi - e)) / (2 * h)
        np.testing.assert_allclose(grad[:, x], fd, rtol=1e-6, atol=1e-6)


def test_leapfrog_is_reversible_and_second_order():
    L = 4
    g = np.random.default_rng(2)
    phi, p = 0.5 * g.standard_normal((5, 16)), g.standard_normal((5, 16))
    v = 0.5 + g.random(16)
    args = (0.6, L, -4.0, 8.0, 1.0, 1.0, False)
    phi1, p1 = hmc.leapfrog(phi, p, v, 0.05, 20, *args)
    phi0, p0 = hmc.leapfrog(phi1, -p1, v, 0.05, 20, *args)
    np.testing.assert_allclose(phi0, phi, atol=1e-11)
    np.testing.assert_allclose(-p0, p, atol=1e-11)

    def dH(eps, n):
        a, b = hmc.leapfrog(phi, p, v, eps, n, *args)
        H = lambda f, q: (0.6 * lattice.action(f, L, -4.0, 8.0) + 0.4 * 0.5 * lattice.sq_norm(f)  # noqa: E731
                          + 0.5 * (v * q * q).sum(axis=1))
        return np.abs(H(a, b) - H(phi, p))
    ratio = dH(0.01, 20) / dH(0.005, 40)  # same trajectory length, half the step
    assert np.all((ratio > 3.0) & (ratio < 5.0)), ratio


def test_small_steps_are_accepted():
    L, N = 3, 64
    g = np.random.default_rng(3)
    phi = 0.7 + 0.2 * g.standard_normal((N, L * L))
    S, sq = lattice.action(phi, L, -4.0, 8.0), lattice.sq_norm(phi)
    out = hmc.hmc_sweep(phi, S, sq, np.full(L * L, 0.05), 1e-3, 0.5, L, -4.0, 8.0, 1.0, 1.0, False, 1, 0, 1, 0)
    assert np.abs(out[4]).max() < 1e-4 and out[3].all()


def test_hmc_free_field_evidence():
    lz = np.array([SMC(SMCConfig(L=2, N=2048, m2=1.0, lam=0.0, rho=0.9, n_mcmc=3, seed=s, inner="hmc")).run()["logz"]
                   for s in range(6)])
    ref = cf.free_field_logz(2, 1.0)
    se = lz.std(ddof=1) / math.sqrt(len(lz))
    assert abs(lz.mean() + 0.5 * lz.var(ddof=1) - ref) < 4.0 * se + 0.01


@pytest.mark.parametrize("keep_reference", [False, True])
def test_invariance_free_field(keep_reference):
    # exact draws from gamma_beta of the free field stay distributed as gamma_beta under HMC
    # transitions with an inverse mass deliberately off the exact variances: a wrong kinetic
    # or potential term in the Hamiltonian of the accept test moves E|phi|^2 and Var M (or
    # starves the acceptance); a wrong force leaves the transition exact and only lowers the
    # acceptance, which the gradient pins above cover
    L, m2, beta, N = 4, 1.0, 0.6, 20000
    D = L * L
    g = np.random.default_rng(21)
    C = cf.free_field_covariance(L, m2, beta, keep_reference)
    phi = g.standard_normal((N, D)) @ np.linalg.cholesky(C).T
    want_sq, want_varM = float(np.trace(C)), float(C.sum()) / D ** 2
    S, sq = lattice.action(phi, L, m2, 0.0), lattice.sq_norm(phi)
    v = np.diag(C) * (0.5 + g.random(D))
    accs = []
    for s in range(4):
        phi, S, sq, acc, _ = hmc.hmc_sweep(phi, S, sq, v, hmc.default_step(D), beta, L, m2, 0.0, 1.0, 1.0,
                                           keep_reference, 3, 0, 1, s)
        accs.append(acc.mean())
    assert min(accs) > 0.6, accs
    assert abs(sq.mean() - want_sq) < 4 * math.sqrt(np.var(sq) / N), (sq.mean(), want_sq)
    varM = phi.mean(axis=1).var()
    assert abs(varM - want_varM) < 4 * want_varM * math.sqrt(2.0 / N), (varM, want_varM)
    np.testing.assert_allclose(S, lattice.action(phi, L, m2, 0.0), rtol=1e-12)
    np.testing.assert_allclose(sq, lattice.sq_norm(phi), rtol=1e-12)
