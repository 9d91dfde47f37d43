"""Hamiltonian Monte Carlo sweep with a diagonal mass matrix (Sec. 2 sampler (iii)
"SMC-HMC"; App. A: a fixed trajectory of 20 leapfrog steps, a diagonal mass matrix).

Test infrastructure (see ``oracle/__init__``).

Reading (the paper tunes the mass matrix in a warm-up with window adaptation and then
freezes it; it states neither the step size nor a tuning rule): the inverse mass of site
x is the population's variance at the refit, v_x = Sigma_xx + delta (delta the ridge of
the factorisation), so that the momenta p ~ N(0, diag(1/v)) move every site on its own
scale; the step size is fixed per run (eps = 0.8 D^(-1/4) unless given).

The target of a temperature is gamma_beta (the random-walk sweep's), with
    log gamma_beta(phi) = -beta S(phi) - a |phi|^2 / 2,   a = 1 - beta (a = 1 when the
    reference is kept at beta = 1),
    grad log gamma_beta = -beta grad S - a phi,
    grad S_x = c_kin (8 phi_x - 2 sum of the four neighbours) + 2 c_mass m2 phi_x + 4 lam phi_x^3
(the kinetic term of Eq. (1) in the form c_kin phi^T (4 I - A) phi, A the periodic
adjacency). One transition: p = z / sqrt(v) with z the normals of the random-walk sweep's
counters; leapfrog p += eps/2 g, then n times {phi += eps v p; g = grad; p += eps g}, the
last momentum step a half step; accept when log u < H(phi, p) - H(phi', p'),
H = -log gamma_beta + sum_x v_x p_x^2 / 2.
"""
import numpy as np

from . import lattice, mutation, philox

N_LEAPFROG = 20


def default_step(D):
    return 0.8 * float(D) ** -0.25


def grad_action(phi, L, m2, lam, c_kin=1.0, c_mass=1.0):
    """dS/dphi for every site, written with np.roll neighbours (rows are fields)."""
    phi = np.asarray(phi, np.float64)
    f = phi.reshape(phi.shape[:-1] + (L, L))
    nb = np.roll(f, 1, -1) + np.roll(f, -1, -1) + np.roll(f, 1, -2) + np.roll(f, -1, -2)
    g = c_kin * (8.0 * f - 2.0 * nb) + 2.0 * c_mass * m2 * f + 4.0 * lam * f ** 3
    return g.reshape(phi.shape)


def grad_log_target(phi, beta, L, m2, lam, c_kin, c_mass, keep_reference):
    a = 1.0 if keep_reference else 1.0 - beta
    return -beta * grad_action(phi, L, m2, lam, c_kin, c_mass) - a * np.asarray(phi, np.float64)


def leapfrog(phi, p, v, eps, n, beta, L, m2, lam, c_kin, c_mass, keep_reference):
    """n leapfrog steps of (phi, p) for H = -log gamma_beta + p^T diag(v) p / 2."""
    phi = np.array(phi, np.float64)
    p = np.array(p, np.float64)
    p = p + 0.5 * eps * grad_log_target(phi, beta, L, m2, lam, c_kin, c_mass, keep_reference)
    for i in range(n):
        phi = phi + eps * v * p
        g = grad_log_target(phi, beta, L, m2, lam, c_kin, c_mass, keep_reference)
        p = p + (eps if i + 1 < n else 0.5 * eps) * g
    return phi, p


def hmc_sweep(phi, S, sq, v, eps, beta, L, m2, lam, c_kin, c_mass, keep_reference, seed, stream, step, sweep,
              n_leapfrog=N_LEAPFROG):
    N, D = phi.shape
    Z = philox.normals(seed, stream, philox.KIND_PROPOSE, step, sweep, N, D, bits=32)
    p0 = Z / np.sqrt(v)[None, :]
    prop, p1 = leapfrog(phi, p0, v[None, :], eps, n_leapfrog, beta, L, m2, lam, c_kin, c_mass, keep_reference)
    S_new = lattice.action(prop, L, m2, lam, c_kin, c_mass)
    sq_new = lattice.sq_norm(prop)
    kin0 = 0.5 * (v[None, :] * p0 * p0).sum(axis=1)
    kin1 = 0.5 * (v[None, :] * p1 * p1).sum(axis=1)
    log_alpha = mutation.log_accept_ratio(S_new, sq_new, S, sq, beta, keep_reference) - (kin1 - kin0)
    u = philox.uniform53(seed, stream, philox.KIND_ACCEPT, step, sweep, np.arange(N))
    acc = np.log(u) < log_alpha
    phi = np.where(acc[:, None], prop, phi)
    return phi, np.where(acc, S_new, S), np.where(acc, sq_new, sq), acc, log_alpha
