"""Adaptive tempering: ESS, bisection for the next temperature, reweighting and
the running log Z (Sec. 2 sampler (i); App. A, target ESS).

Test infrastructure (see ``oracle/__init__``).

Readings where the paper is silent: the ESS of the incremental weights
w_i = exp(dbeta * ell_i) is (sum w)^2 / sum w^2; the next increment dbeta in
(0, 1 - beta] solves ESS(dbeta) = rho * N and is found by bisection on
[0, 1 - beta], halving until ``iters`` steps are done or the bracket stops
shrinking; the returned value is the lower end (its ESS is >= rho N). If
ESS(1 - beta) >= rho N the run steps straight to beta = 1. Particles are
resampled at every temperature, so the log Z increment is
log mean_i exp(dbeta ell_i), accumulated over temperatures with Kahan
compensation.
"""
import math

import numpy as np


def shifted(ell):
    """a_i = ell_i - max_j ell_j (all <= 0, the maximiser gives exactly 0)."""
    ell = np.asarray(ell, dtype=np.float64)
    return ell - ell.max()


def ess(ell, dbeta):
    """Effective sample size of the weights exp(dbeta * ell_i)."""
    w = np.exp(dbeta * shifted(ell))
    return w.sum() ** 2 / (w * w).sum()


def bisect_dbeta(ell, beta, rho, iters=64):
    """Next temperature increment. Returns (dbeta, n_iterations_used)."""
    n = len(ell)
    target = rho * n
    hi = 1.0 - beta
    if ess(ell, hi) >= target:
        return hi, 0
    lo = 0.0
    used = 0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        used += 1
        if ess(ell, mid) >= target:
            lo = mid
        else:
            hi = mid
    if lo == 0.0:
        # No positive increment keeps the ESS above target at this resolution:
        # take the smallest bracket end so the run still advances.
        return hi, used
    return lo, used


def reweight(ell, dbeta):
    """Normalised-by-max weights w_i = exp(dbeta (ell_i - ell_max)) (max weight 1)
    and the log Z increment log mean_i exp(dbeta ell_i)."""
    ell = np.asarray(ell, dtype=np.float64)
    w = np.exp(dbeta * shifted(ell))
    inc = dbeta * ell.max() + math.log(w.sum()) - math.log(len(ell))
    return w, inc


class KahanSum:
    """Compensated running sum (Kahan) of the per-temperature log Z increments."""

    def __init__(self):
        self.s = 0.0
        self.c = 0.0

    def add(self, x):
        y = x - self.c
        t = self.s + y
        self.c = (t - self.s) - y
        self.s = t
        return self.s
