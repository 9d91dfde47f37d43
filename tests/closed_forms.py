"""Closed forms and quadratures that pin the oracle (and, through it, the kernels).

None of this is the sampler: these are exact results for special cases of the
phi^4 model of Eq. (1), in the coefficient form
    S = sum_x [ c_kin * sum_mu phi_x (2 phi_x - phi_{x+mu} - phi_{x-mu}) + c_mass m2 phi_x^2 + lam phi_x^4 ].

* Free field (lam = 0, c_mass m2 > 0): S = phi^T P phi with P diagonal in the
  lattice Fourier basis, p_k = c_mass m2 + c_kin sum_mu 4 sin^2(pi k_mu / L).
  Along the tempering path gamma_beta = N(0, I)^(1-beta) exp(-beta S):
      log Z_beta = (beta D / 2) log(2 pi) - 1/2 sum_k log(1 - beta + 2 beta p_k).
  At beta = 1 this is (D/2) log pi - 1/2 sum_k log p_k.
  M = mean field has Var M = 1/(2 D p_0) with p_0 = c_mass m2 (k = 0 mode).
* One site (L = 1): the kinetic term vanishes, Z = int exp(-c_mass m2 c^2 - lam c^4) dc.
* 2 x 2 torus: each nearest-neighbour pair appears twice, so the kinetic term is
  a 4-cycle with coupling 2 c_kin; Z = tr(T^4) for the symmetric transfer kernel
  T(x, y) = exp(-V(x)/2 - 2 c_kin (x - y)^2 - V(y)/2), V = c_mass m2 phi^2 + lam phi^4.
"""
import math

import numpy as np
from scipy import integrate


def lattice_laplacian_eigs(L):
    k = np.arange(L)
    s = 4.0 * np.sin(np.pi * k / L) ** 2
    return (s[:, None] + s[None, :]).ravel()


def free_field_logz(L, m2, beta=1.0, c_kin=1.0, c_mass=1.0, keep_reference=False):
    """log Z_beta of the free field along the tempering path."""
    D = L * L
    p = c_mass * m2 + c_kin * lattice_laplacian_eigs(L)
    if keep_reference:
        # gamma_beta = N(0, I) exp(-beta S): quadratic form 1/2 + beta p_k.
        return -0.5 * D * math.log(2.0 * math.pi) + 0.5 * D * math.log(math.pi) \
            - 0.5 * float(np.log(0.5 + beta * p).sum())
    return 0.5 * beta * D * math.log(2.0 * math.pi) - 0.5 * float(np.log(1.0 - beta + 2.0 * beta * p).sum())


def free_field_moments(L, m2, c_mass=1.0):
    """(Var M, <|M|>, chi) of the free field at beta = 1."""
    D = L * L
    var = 1.0 / (2.0 * D * c_mass * m2)
    return var, math.sqrt(2.0 * var / math.pi), D * var


def free_field_sq_mean(L, m2, beta=1.0, c_kin=1.0, c_mass=1.0):
    """E |phi|^2 under gamma_beta: sum_k 1 / (2 q_k), q_k = (1-beta)/2 + beta p_k."""
    p = c_mass * m2 + c_kin * lattice_laplacian_eigs(L)
    q = 0.5 * (1.0 - beta) + beta * p
    return float((0.5 / q).sum())


def free_field_sample(L, m2, beta, n, rng, c_kin=1.0, c_mass=1.0):
    """Exact draws from gamma_beta of the free field (eigenbasis of the quadratic form)."""
    D = L * L
    p = c_mass * m2 + c_kin * lattice_laplacian_eigs(L)
    # Build the real quadratic form explicitly and diagonalise it.
    idx = np.arange(D).reshape(L, L)
    A = np.zeros((D, D))
    for r in range(L):
        for c in range(L):
            x = idx[r, c]
            A[x, x] += c_kin * 4.0 + c_mass * m2
            for (rr, cc) in ((r, (c + 1) % L), (r, (c - 1) % L), ((r + 1) % L, c), ((r - 1) % L, c)):
                A[x, idx[rr, cc]] -= c_kin
    Q = 0.5 * (1.0 - beta) * np.eye(D) + beta * A
    evals, evecs = np.linalg.eigh(Q)
    assert np.allclose(np.sort(evals), np.sort(0.5 * (1.0 - beta) + beta * p), atol=1e-9)
    xi = rng.standard_normal((n, D))
    return (xi / np.sqrt(2.0 * evals)) @ evecs.T


def free_field_covariance(L, m2, beta, keep_reference=False, c_kin=1.0, c_mass=1.0):
    """Covariance of gamma_beta for the free field, from the quadratic form written out site
    by site: precision a I + 2 beta A with a = 1 - beta (1 with the reference kept) and
    S = phi^T A phi."""
    D = L * L
    A = np.zeros((D, D))
    for r in range(L):
        for c in range(L):
            x = r * L + c
            A[x, x] += c_kin * 4.0 + c_mass * m2
            for (rr, cc) in ((r, (c + 1) % L), (r, (c - 1) % L), ((r + 1) % L, c), ((r - 1) % L, c)):
                A[x, rr * L + cc] -= c_kin
    a = 1.0 if keep_reference else 1.0 - beta
    return np.linalg.inv(a * np.eye(D) + 2.0 * beta * A)


def one_site_logz(m2, lam, c_mass=1.0):
    f = lambda c: math.exp(-c_mass * m2 * c * c - lam * c ** 4)
    val, err = integrate.quad(f, -np.inf, np.inf, epsabs=0, epsrel=1e-13, limit=200)
    return math.log(val)


def one_site_information(m2, lam, c_mass=1.0):
    """Information H = E_post[log L] - log Z of the one-site problem as nested sampling
    sets it up: prior N(0, 1), likelihood L(c) = exp(-S(c)) / N(c; 0, 1), posterior
    exp(-S) / Z (adaptive quadrature)."""
    logz = one_site_logz(m2, lam, c_mass)
    S = lambda c: c_mass * m2 * c * c + lam * c ** 4  # noqa: E731
    f = lambda c: math.exp(-S(c) - logz) * (-S(c) + 0.5 * c * c + 0.5 * math.log(2.0 * math.pi))  # noqa: E731
    val, _ = integrate.quad(f, -np.inf, np.inf, epsabs=0, epsrel=1e-12, limit=200)
    return val - logz


def two_by_two_logz(m2, lam, c_kin=1.0, c_mass=1.0, half_width=8.0, n=4001):
    """log Z of the 2 x 2 torus by the transfer matrix on a uniform grid
    (trapezoid rule; the integrand decays like a Gaussian or faster)."""
    x = np.linspace(-half_width, half_width, n)
    h = x[1] - x[0]
    V = c_mass * m2 * x * x + lam * x ** 4
    T = np.exp(-0.5 * V[:, None] - 2.0 * c_kin * (x[:, None] - x[None, :]) ** 2 - 0.5 * V[None, :])
    ev = np.linalg.eigvalsh(h * T)
    top = ev.max()
    return 4.0 * math.log(top) + math.log(float(((ev / top) ** 4).sum()))
