"""Seeded synthetic inputs shared by the oracle-side and the GPU-side tests.

This module only draws numbers (numpy's PCG64 streams) with the shapes and
value ranges of the sampler's data; it contains none of the method's
arithmetic, so it can feed both implementations without coupling them.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(int(seed))


def fields(N, D, seed, scale=1.0, dtype=np.float64):
    """N fields of D sites, i.i.d. normal with the given scale."""
    return (scale * rng(seed).standard_normal((N, D))).astype(dtype)


def broken_phase_fields(N, D, seed, amplitude=0.5, noise=0.3, dtype=np.float64):
    """Fields near one of the two minima +-amplitude plus noise (bimodal population)."""
    g = rng(seed)
    sign = np.where(g.random(N) < 0.5, -1.0, 1.0)
    return (sign[:, None] * amplitude + noise * g.standard_normal((N, D))).astype(dtype)


def log_weights(N, seed, spread=50.0, offset=-1000.0):
    """Tempering log-likelihood values with a wide spread (like -S + |phi|^2/2)."""
    g = rng(seed)
    return offset + spread * g.standard_normal(N)


def positive_weights(N, seed, zeros=0, heavy=False):
    """Positive weights with max 1 (optionally some exact zeros, or a heavy tail)."""
    g = rng(seed)
    w = np.exp(-3.0 * g.random(N)) if not heavy else np.exp(-30.0 * g.random(N))
    if zeros:
        w[g.choice(N, size=zeros, replace=False)] = 0.0
    w[g.integers(N)] = 1.0
    return w / w.max()


def spd_matrix(D, seed, cond=100.0):
    """A symmetric positive-definite D x D matrix with the given condition number."""
    g = rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((D, D)))
    ev = np.geomspace(1.0, 1.0 / cond, D)
    return (Q * ev) @ Q.T


def lower_factor(D, seed):
    """A random lower-triangular matrix with a positive diagonal."""
    g = rng(seed)
    B = np.tril(g.standard_normal((D, D)) * 0.3)
    B[np.diag_indices(D)] = 0.5 + g.random(D)
    return B


def word32(seed):
    return int(rng(seed).integers(0, 2 ** 32))
