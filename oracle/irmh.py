"""Independent Metropolis-Hastings sweep tuned to the particle covariance (Sec. 2
sampler (ii) "SMC-IRMH"): every particle proposes a fresh draw from the Gaussian of the
population's mean and covariance, independently of where it is.

Test infrastructure (see ``oracle/__init__``).

With q = N(mu, Sigma), Sigma = L L^T (the refit of this temperature):
    phi' = mu + L z,   z ~ N(0, I_D)      (row form: Phi' = 1 mu^T + Z L^T)
    log alpha = log gamma_beta(phi') - log gamma_beta(phi) + log q(phi) - log q(phi')
              = [tempered-target term of the random-walk sweep] + (|z|^2 - r) / 2,
    r = |L^{-1}(phi - mu)|^2, the current particle's whitened squared norm (log q up to
    its constant is -r/2 at the particle and -|z|^2/2 at the proposal).
r is computed for every particle after the refit and becomes |z|^2 when a proposal is
accepted. The random numbers are those of the random-walk sweep: normals (KIND_PROPOSE,
step, sweep, particle, block), the uniform (KIND_ACCEPT, step, sweep, particle, 0).
"""
import numpy as np
import scipy.linalg

from . import lattice, mutation, philox


def whitened_sq_norm(phi, mu, Lchol):
    """r_n = |L^{-1}(phi_n - mu)|^2 by forward substitution."""
    X = (np.asarray(phi, np.float64) - np.asarray(mu, np.float64)[None, :]).T
    W = scipy.linalg.solve_triangular(np.asarray(Lchol, np.float64), X, lower=True)
    return (W * W).sum(axis=0)


def irmh_sweep(phi, S, sq, r, Lchol, mu, beta, L, m2, lam, c_kin, c_mass, keep_reference, seed, stream, step,
               sweep):
    N, D = phi.shape
    Z = philox.normals(seed, stream, philox.KIND_PROPOSE, step, sweep, N, D, bits=32)
    prop = np.asarray(mu, np.float64)[None, :] + Z @ np.asarray(Lchol, np.float64).T
    zz = (Z * Z).sum(axis=1)
    S_new = lattice.action(prop, L, m2, lam, c_kin, c_mass)
    sq_new = lattice.sq_norm(prop)
    log_alpha = mutation.log_accept_ratio(S_new, sq_new, S, sq, beta, keep_reference) + 0.5 * (zz - r)
    u = philox.uniform53(seed, stream, philox.KIND_ACCEPT, step, sweep, np.arange(N))
    acc = np.log(u) < log_alpha
    phi = np.where(acc[:, None], prop, phi)
    return phi, np.where(acc, S_new, S), np.where(acc, sq_new, sq), np.where(acc, zz, r), acc, log_alpha
