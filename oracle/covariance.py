"""Particle covariance, its regularisation and Cholesky factor (App. A: one
Gaussian covariance estimated from the particle population at every outer step).

Test infrastructure (see ``oracle/__init__``).

Reading where the paper is silent: the covariance is the unweighted sample
covariance of the (already resampled) population with divisor N - 1; a ridge
delta * I with delta = jitter_rel * 10^level * trace / D is added before
factorising, and the ridge is multiplied by 10 (up to ``max_tries`` times) while
the matrix is not numerically positive definite. A run starts at level 0 and each
outer step starts from the level that succeeded at the previous one.
"""
import numpy as np


def sample_covariance(X):
    """mean and Sigma = Xc^T Xc / (N - 1) with Xc = X - mean (rows are particles)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    mu = X.mean(axis=0)
    Xc = X - mu
    return mu, (Xc.T @ Xc) / (n - 1)


def cholesky_lower(A):
    """Lower factor of A = L L^T (library routine; raises LinAlgError when not PD)."""
    return np.linalg.cholesky(np.asarray(A, dtype=np.float64))


def regularised_cholesky(Sigma, jitter_rel=1e-8, max_tries=6, start_level=0):
    """Returns (L, delta, tries, level) with L L^T = Sigma + delta I and
    delta = jitter_rel 10^level trace / D."""
    D = Sigma.shape[0]
    delta = jitter_rel * np.trace(Sigma) / D
    for _ in range(start_level):
        delta *= 10.0
    for tries in range(1, max_tries + 1):
        try:
            return cholesky_lower(Sigma + delta * np.eye(D)), delta, tries, start_level + tries - 1
        except np.linalg.LinAlgError:
            delta *= 10.0
    raise np.linalg.LinAlgError("covariance not positive definite after %d ridge increases" % max_tries)


def gaussian_part_covariance(L, beta, m2, c_kin=1.0, c_mass=1.0, keep_reference=False):
    """Covariance of the Gaussian part of the tempered target gamma_beta (Sec. 2 tempering
    path), a kernel covariance that does not depend on the particles.

    log gamma_beta = -beta S - (1 - beta) |phi|^2 / 2 (with the reference kept:
    -|phi|^2 / 2 - beta S); its quadratic part is -(1/2) phi^T P phi with
    P = a I + 2 beta (c_kin K + c_mass m2 I), K the form of Eq. (1)'s kinetic term,
    phi^T K phi = sum_x sum_mu phi_x (2 phi_x - phi_{x+mu} - phi_{x-mu}), and a = 1 - beta
    (1 with the reference kept). Returns P^{-1}; for lambda = 0 it is the target's
    covariance. K is assembled term by term from that sum (on L <= 2 several
    neighbour terms land on the same entry)."""
    D = L * L
    K = np.zeros((D, D))
    for r in range(L):
        for c in range(L):
            x = r * L + c
            for rr, cc in (((r + 1) % L, c), ((r - 1) % L, c), (r, (c + 1) % L), (r, (c - 1) % L)):
                K[x, x] += 1.0           # phi_x * phi_x, once per neighbour term (2 per direction)
                K[x, rr * L + cc] -= 1.0
    a = 1.0 if keep_reference else 1.0 - beta
    P = a * np.eye(D) + 2.0 * beta * (c_kin * K + c_mass * m2 * np.eye(D))
    return np.linalg.inv(P)
