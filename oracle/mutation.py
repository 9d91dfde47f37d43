"""Covariance-preconditioned random-walk Metropolis sweep (Sec. 2 sampler (i);
App. A: Gaussian random-walk proposal from the particle covariance, scaled by
2.38^2 / V in variance, i.e. 2.38 / sqrt(D) on the Cholesky factor).

Test infrastructure (see ``oracle/__init__``).

One sweep moves every particle jointly in all D sites:
    phi' = phi + s * L z,   z ~ N(0, I_D)      (row form: Phi' = Phi + s Z L^T)
    log alpha = log gamma_beta(phi') - log gamma_beta(phi)
              = -beta (S' - S) - (1 - beta) (|phi'|^2 - |phi|^2) / 2
    accept when log u < log alpha, u uniform on (0, 1].
(With the reference kept at beta = 1 the second term is -(|phi'|^2 - |phi|^2)/2.)
"""
import numpy as np

from . import lattice, philox


def rw_scale_default(D):
    return 2.38 / np.sqrt(D)


def log_accept_ratio(S_new, sq_new, S_old, sq_old, beta, keep_reference=False):
    dS = np.asarray(S_new) - np.asarray(S_old)
    dsq = np.asarray(sq_new) - np.asarray(sq_old)
    if keep_reference:
        return -beta * dS - 0.5 * dsq
    return -beta * dS - (1.0 - beta) * 0.5 * dsq


def propose(phi, Z, Lchol, scale):
    """phi' = phi + scale * Z L^T (rows are particles)."""
    return np.asarray(phi, np.float64) + scale * (np.asarray(Z, np.float64) @ np.asarray(Lchol, np.float64).T)


def accept(phi, S, sq, prop, log_u, beta, L, m2, lam, c_kin, c_mass, keep_reference=False):
    """Metropolis decision per particle. Returns (phi, S, sq, accepted mask,
    S_prop, sq_prop, log_alpha)."""
    S_new = lattice.action(prop, L, m2, lam, c_kin, c_mass)
    sq_new = lattice.sq_norm(prop)
    log_alpha = log_accept_ratio(S_new, sq_new, S, sq, beta, keep_reference)
    acc = log_u < log_alpha
    phi = np.where(acc[:, None], prop, phi)
    S = np.where(acc, S_new, S)
    sq = np.where(acc, sq_new, sq)
    return phi, S, sq, acc, S_new, sq_new, log_alpha


def rw_sweep(phi, S, sq, Lchol, scale, beta, L, m2, lam, c_kin, c_mass, keep_reference,
             seed, stream, step, sweep, normal_bits=32):
    """One full sweep with the random numbers of the shared counter layout:
    normals (KIND_PROPOSE, step, sweep, particle, block) and the accept uniform
    (KIND_ACCEPT, step, sweep, particle, 0)."""
    N, D = phi.shape
    Z = philox.normals(seed, stream, philox.KIND_PROPOSE, step, sweep, N, D, bits=normal_bits)
    prop = propose(phi, Z, Lchol, scale)
    u = philox.uniform53(seed, stream, philox.KIND_ACCEPT, step, sweep, np.arange(N))
    phi, S, sq, acc, _, _, _ = accept(phi, S, sq, prop, np.log(u), beta, L, m2, lam, c_kin, c_mass,
                                      keep_reference)
    return phi, S, sq, acc
