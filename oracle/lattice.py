"""Lattice phi^4 action, tempering log-weight and magnetisation (Sec. 2, Eq. (1)).

Test infrastructure (see ``oracle/__init__``).

Fields are arrays whose last axis holds the D = L*L sites of a periodic L x L
lattice in row-major order, site x = r*L + c; direction mu=1 moves along c,
mu=2 along r, both with periodic wrap.

Action reading. Eq. (1) writes S = sum_x [1/2 sum_mu (phi_{x+mu}-phi_x)^2
+ 1/2 m0^2 phi_x^2 + lambda phi_x^4]. The workloads this library is built for
use the unhalved site form
    S = sum_x [ sum_mu phi_x (2 phi_x - phi_{x+mu} - phi_{x-mu}) + m^2 phi_x^2 + lambda phi_x^4 ],
whose kinetic part equals sum_{x,mu} (phi_{x+mu}-phi_x)^2. Both are covered by
two coefficients:
    S = sum_x [ c_kin * K_x + c_mass * m2 * phi_x^2 + lam * phi_x^4 ],
    K_x = sum_mu phi_x (2 phi_x - phi_{x+mu} - phi_{x-mu}),
with (c_kin, c_mass) = (1, 1) for the unhalved form and (1/2, 1/2) for Eq. (1).
"""
import math

import numpy as np


def as_lattice(phi, L):
    phi = np.asarray(phi, dtype=np.float64)
    return phi.reshape(phi.shape[:-1] + (L, L))


def kinetic_site_terms(phi, L):
    """K_x for every site, from the 4-neighbour periodic stencil."""
    f = as_lattice(phi, L)
    nb = (np.roll(f, 1, axis=-1) + np.roll(f, -1, axis=-1)
          + np.roll(f, 1, axis=-2) + np.roll(f, -1, axis=-2))
    return f * (4.0 * f - nb)


def action(phi, L, m2, lam, c_kin=1.0, c_mass=1.0):
    """S(phi) of Eq. (1) in the coefficient form above; one value per field."""
    f = as_lattice(phi, L)
    site = c_kin * kinetic_site_terms(phi, L) + c_mass * m2 * f * f + lam * f ** 4
    return site.sum(axis=(-1, -2))


def sq_norm(phi):
    phi = np.asarray(phi, dtype=np.float64)
    return (phi * phi).sum(axis=-1)


def log_gauss_const(D):
    """(D/2) log(2 pi): minus the log-normaliser of the N(0, I_D) reference."""
    return 0.5 * D * math.log(2.0 * math.pi)


def tempering_loglik(S, sq, D, keep_reference=False):
    """Incremental tempering log-weight ell = log gamma_1 - log gamma_0.

    Tempering path (Sec. 2): gamma_beta(phi) = N(phi; 0, I)^(1-beta) exp(-beta S)
    (reference dropped at beta = 1) gives ell = -S + |phi|^2 / 2 + (D/2) log 2 pi.
    With ``keep_reference`` the path is N(phi; 0, I) exp(-beta S), i.e.
    exp(-[U_0 + beta S]) normalised by the reference, and ell = -S.
    """
    if keep_reference:
        return -np.asarray(S, dtype=np.float64)
    return -np.asarray(S, dtype=np.float64) + 0.5 * np.asarray(sq, dtype=np.float64) + log_gauss_const(D)


def log_target(S, sq, beta, keep_reference=False):
    """log gamma_beta up to a beta-dependent constant, the MCMC target at beta."""
    if keep_reference:
        return -beta * np.asarray(S) - 0.5 * np.asarray(sq)
    return -beta * np.asarray(S) - (1.0 - beta) * 0.5 * np.asarray(sq)


def magnetisation(phi):
    """M = (1/V) sum_x phi_x (Sec. 2, order parameter)."""
    phi = np.asarray(phi, dtype=np.float64)
    return phi.mean(axis=-1)
