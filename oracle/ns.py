"""Nested sampling with slice-sampling rejuvenation (Sec. 2 sampler (iv) "NS";
App. A: a fraction of the live points is deleted per iteration, and the new
points come from slice sampling along directions drawn from the live-point
covariance, subject to the current likelihood constraint).

Test infrastructure (see ``oracle/__init__``).

Prior N(0, I_D); likelihood log L = ell = -S + |phi|^2/2 + (D/2) log 2 pi, so
that prior x likelihood = exp(-S) and Z = int exp(-S) (the same target and
evidence as the tempered SMC).

Readings where the paper is silent (it defers to the nested-slice-sampling
reference):
* iteration it deletes the k = n_delete lowest-likelihood live points (stable
  order); L* is the largest deleted log L;
* the prior volume shrinks by the expected factor of removing points one at a
  time: log X_j = log X_{j-1} - 1/(N - j + 1) for the j-th deleted point of the
  batch, whose weight is X_{j-1} - X_j;
* the covariance (and Cholesky factor) is that of the N - k surviving points;
* each new point starts from a survivor chosen uniformly (word-0 uniform of
  (KIND_NS_START, it, 0, slot, 0)) and takes ``slice_steps`` slice steps; a step
  draws d = L z (z: KIND_NS_DIRECTION, it, step, slot, block), a slice height on
  the prior log N(x) - E with E = -log u (u: block 0 of KIND_NS_SLICE, it, step,
  slot), brackets the whole prior slice along the line exactly (the roots of
  |x + t d|^2 = |x|^2 + 2E), and shrinks the bracket towards t = 0 with uniforms
  from blocks 1, 2, ... until log L(x + t d) > L*; after ``max_shrink`` failed
  tries the point stays where it is (counted as capped);
* stop when log(X mean_live L) - log Z < log(stop_frac); the final evidence
  adds X mean_live L; the error bar is sqrt(H / N) with H the information.
"""
import dataclasses
import math

import numpy as np

from . import covariance, lattice, philox


def logaddexp(a, b):
    if a == -math.inf:
        return b
    if b == -math.inf:
        return a
    m = max(a, b)
    return m + math.log(math.exp(a - m) + math.exp(b - m))


def logsumexp(v):
    v = np.asarray(v, dtype=np.float64)
    if v.size == 0:
        return -math.inf
    m = float(v.max())
    return m + math.log(float(np.exp(v - m).sum()))


@dataclasses.dataclass
class NSConfig:
    L: int
    N: int
    m2: float
    lam: float
    c_kin: float = 1.0
    c_mass: float = 1.0
    n_delete: int = 1
    slice_steps: int = 0           # <= 0: 3 * D
    stop_frac: float = 1e-3
    max_shrink: int = 64
    jitter_rel: float = 1e-8
    seed: int = 0
    stream: int = 0
    normal_bits: int = 32
    max_iters: int = 1000000

    @property
    def D(self):
        return self.L * self.L

    @property
    def steps(self):
        return self.slice_steps if self.slice_steps > 0 else 3 * self.D


def loglik(phi, cfg):
    S = lattice.action(phi, cfg.L, cfg.m2, cfg.lam, cfg.c_kin, cfg.c_mass)
    return lattice.tempering_loglik(S, lattice.sq_norm(phi), cfg.D)


def prior_bracket(x, d, E):
    """Roots t- < 0 < t+ of |x + t d|^2 = |x|^2 + 2E (the exact prior slice)."""
    a = float(d @ d)
    b = float(x @ d)
    disc = math.sqrt(b * b + 2.0 * E * a)
    return (-b - disc) / a, (-b + disc) / a


def slice_chain(x, logl_x, Lchol, lstar, cfg, it, slot):
    """Slice steps for one new point. Returns (x, log L(x), n_capped)."""
    capped = 0
    D = cfg.D
    for s in range(cfg.steps):
        z = philox.normals(cfg.seed, cfg.stream, philox.KIND_NS_DIRECTION, it, s, 1, D,
                           bits=cfg.normal_bits, row0=slot)[0]
        d = Lchol @ z
        w = philox.words(cfg.seed, cfg.stream, philox.KIND_NS_SLICE, it, s, [slot],
                         np.arange(cfg.max_shrink + 1))[0]
        E = -math.log(float(philox.uniform53_words(w[0, 0], w[0, 1])))
        t_lo, t_hi = prior_bracket(x, d, E)
        moved = False
        for r in range(cfg.max_shrink):
            u = float(philox.uniform53_words(w[1 + r, 0], w[1 + r, 1]))
            t = t_lo + u * (t_hi - t_lo)
            y = x + t * d
            ly = float(loglik(y[None, :], cfg)[0])
            if ly > lstar:
                x, logl_x, moved = y, ly, True
                break
            if t < 0.0:
                t_lo = t
            else:
                t_hi = t
        if not moved:
            capped += 1
    return x, logl_x, capped


class NS:
    def __init__(self, cfg: NSConfig):
        self.cfg = cfg
        c = cfg
        self.live = philox.normals(c.seed, c.stream, philox.KIND_INIT, 0, 0, c.N, c.D, bits=c.normal_bits)
        self.logl = loglik(self.live, c)
        self.logX = 0.0
        self.logZ = -math.inf
        self.dead_logl = []
        self.dead_logw = []
        self.it = 0
        self.capped = 0
        self.ridge_level = 0
        self.done = False

    def remaining_log_evidence(self):
        return self.logX + logsumexp(self.logl) - math.log(self.cfg.N)

    def replace_step(self):
        c = self.cfg
        self.it += 1
        it = self.it
        N, k = c.N, c.n_delete
        order = np.argsort(self.logl, kind="stable")
        dead, survivors = order[:k], order[k:]
        lstar = float(self.logl[dead[-1]])
        logX = self.logX
        for j in range(1, k + 1):
            shrink = 1.0 / (N - j + 1)
            logw = logX + math.log(-math.expm1(-shrink))
            logX = logX - shrink
            lj = float(self.logl[dead[j - 1]])
            self.dead_logl.append(lj)
            self.dead_logw.append(logw)
            self.logZ = logaddexp(self.logZ, lj + logw)
        self.logX = logX
        _, Sigma = covariance.sample_covariance(self.live[survivors])
        Lc, _, _, self.ridge_level = covariance.regularised_cholesky(Sigma, c.jitter_rel,
                                                                     start_level=self.ridge_level)
        new_pts = []
        for slot in range(k):
            w = philox.words(c.seed, c.stream, philox.KIND_NS_START, it, 0, [slot], [0])[0, 0]
            u = float(w[0]) * 2.0 ** -32
            start = int(survivors[int(math.floor(u * (N - k)))])
            x, lx, cap = slice_chain(self.live[start].copy(), float(self.logl[start]), Lc, lstar, c, it, slot)
            self.capped += cap
            new_pts.append((x, lx))
        for slot in range(k):
            self.live[dead[slot]] = new_pts[slot][0]
            self.logl[dead[slot]] = new_pts[slot][1]
        if self.remaining_log_evidence() - self.logZ < math.log(c.stop_frac):
            self.done = True
        return self.done

    def run(self):
        while not self.done and self.it < self.cfg.max_iters:
            self.replace_step()
        return self.result()

    def final(self):
        """(log Z, information H, error sqrt(H/N)) including the live points."""
        c = self.cfg
        logw_live = self.logX - math.log(c.N)
        all_l = np.concatenate([np.asarray(self.dead_logl), self.logl])
        all_w = np.concatenate([np.asarray(self.dead_logw), np.full(c.N, logw_live)])
        logZ = logsumexp(all_l + all_w)
        p = np.exp(all_l + all_w - logZ)
        H = float((p * all_l).sum()) - logZ
        return logZ, H, math.sqrt(max(H, 0.0) / c.N)

    def result(self):
        logZ, H, err = self.final()
        return {"logz": logZ, "logz_err": err, "H": H, "n_iter": self.it, "capped": self.capped}
