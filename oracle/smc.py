"""Adaptive tempered SMC with covariance-preconditioned random-walk moves
(Sec. 2 sampler (i) "SMC-RW"; App. A parameters).

Test infrastructure (see ``oracle/__init__``).

Outer step at temperature index t (t = 1, 2, ...), in the paper's order:
  1. choose dbeta by ESS bisection (``tempering.bisect_dbeta``);
  2. reweight, log Z += log mean exp(dbeta ell) (Kahan);
  3. systematic resampling with offset word (KIND_RESAMPLE, t, 0, 0, 0)[0];
  4. re-estimate the particle covariance and its Cholesky factor (ridge level
     carried over from the previous step); with kernel_cov = "gaussian_part" the
     covariance is instead the exact one of the Gaussian part of the new tempered
     target (a particle-independent control for the free field's closed form);
  5. n_mcmc random-walk Metropolis sweeps targeting gamma_{beta + dbeta} (or, with
     inner = "irmh", independent Metropolis-Hastings sweeps, oracle.irmh; with inner = "hmc",
     HMC transitions with the covariance diagonal as inverse mass, oracle.hmc);
  5'. optionally (z2_flip) the global move phi -> -phi per particle with a Philox bit
     (KIND_FLIP, t, 0, particle, 0), bit 0 of word 0;
  6. refresh ell from the cached S and |phi|^2.
Initial particles are N(0, I_D) draws (KIND_INIT, 0, 0, particle, block).
"""
import dataclasses
import math

import numpy as np

from . import covariance, hmc, irmh, lattice, mutation, observables, philox, resample, tempering


@dataclasses.dataclass
class SMCConfig:
    L: int
    N: int
    m2: float
    lam: float
    c_kin: float = 1.0
    c_mass: float = 1.0
    keep_reference: bool = False
    rho: float = 0.5
    n_mcmc: int = 10
    rw_scale: float = 0.0          # <= 0: 2.38 / sqrt(D)
    jitter_rel: float = 1e-8
    bisect_iters: int = 64
    seed: int = 0
    stream: int = 0
    normal_bits: int = 32          # 32: double-precision draws; 24: single-precision draws
    max_steps: int = 100000
    z2_flip: bool = False          # global phi -> -phi move after each temperature's sweeps
    inner: str = "rw"              # "rw": random-walk sweeps; "irmh": independent MH sweeps (oracle.irmh);
                                   # "hmc": HMC transitions (oracle.hmc)
    hmc_step: float = 0.0          # <= 0: oracle.hmc.default_step(D)
    kernel_cov: str = "population"  # "population": the resampled population's covariance (App. A);
                                    # "gaussian_part": covariance.gaussian_part_covariance at the new beta

    @property
    def D(self):
        return self.L * self.L

    @property
    def scale(self):
        return self.rw_scale if self.rw_scale > 0 else mutation.rw_scale_default(self.D)


def z2_flip(phi, seed, stream, t):
    """Global symmetry move: particle n is negated when bit 0 of the first Philox word of
    counter (KIND_FLIP << 24 | t, 0, n, 0) is set. The tempered targets are even in phi
    (the action is a sum of even terms and the reference N(0, I) is symmetric), so the
    move is a Metropolis proposal with acceptance ratio 1; S, |phi|^2 and the
    log-weights are unchanged. (The paper gives such moves to its AHMC control only.)"""
    w = philox.words(seed, stream, philox.KIND_FLIP, t, 0, np.arange(phi.shape[0]), [0])[:, 0, 0]
    flip = (w & np.uint64(1)) == np.uint64(1)
    out = phi.copy()
    out[flip] = -out[flip]
    return out


class SMC:
    def __init__(self, cfg: SMCConfig):
        self.cfg = cfg
        c = cfg
        self.phi = philox.normals(c.seed, c.stream, philox.KIND_INIT, 0, 0, c.N, c.D, bits=c.normal_bits)
        self.S = lattice.action(self.phi, c.L, c.m2, c.lam, c.c_kin, c.c_mass)
        self.sq = lattice.sq_norm(self.phi)
        self.ell = lattice.tempering_loglik(self.S, self.sq, c.D, c.keep_reference)
        self.beta = 0.0
        self.logz = tempering.KahanSum()
        self.t = 0
        self.ridge_level = 0
        self.history = []

    @property
    def done(self):
        return self.beta >= 1.0

    def choose_dbeta(self):
        c = self.cfg
        dbeta, _ = tempering.bisect_dbeta(self.ell, self.beta, c.rho, c.bisect_iters)
        return dbeta

    def temper_step(self):
        c = self.cfg
        if self.done:
            raise RuntimeError("beta already 1")
        self.t += 1
        t = self.t
        dbeta = self.choose_dbeta()
        beta_new = 1.0 if dbeta >= 1.0 - self.beta else self.beta + dbeta
        w, inc = tempering.reweight(self.ell, dbeta)
        ess = w.sum() ** 2 / (w * w).sum()
        self.logz.add(inc)
        U = philox.word32(c.seed, c.stream, philox.KIND_RESAMPLE, t)
        anc = resample.systematic(w, U)
        self.phi, self.S, self.sq = self.phi[anc], self.S[anc], self.sq[anc]
        if c.kernel_cov == "gaussian_part":
            mu = self.phi.mean(axis=0)
            Sigma = covariance.gaussian_part_covariance(c.L, beta_new, c.m2, c.c_kin, c.c_mass, c.keep_reference)
        else:
            mu, Sigma = covariance.sample_covariance(self.phi)
        Lc, delta, _, self.ridge_level = covariance.regularised_cholesky(Sigma, c.jitter_rel,
                                                                         start_level=self.ridge_level)
        n_acc = 0
        if c.inner == "hmc":
            v = np.diag(Sigma) + delta
            eps = c.hmc_step if c.hmc_step > 0 else hmc.default_step(c.D)
            for s in range(c.n_mcmc):
                self.phi, self.S, self.sq, acc, _ = hmc.hmc_sweep(
                    self.phi, self.S, self.sq, v, eps, beta_new, c.L, c.m2, c.lam, c.c_kin, c.c_mass,
                    c.keep_reference, c.seed, c.stream, t, s)
                n_acc += int(acc.sum())
        elif c.inner == "irmh":
            r = irmh.whitened_sq_norm(self.phi, mu, Lc)
            for s in range(c.n_mcmc):
                self.phi, self.S, self.sq, r, acc, _ = irmh.irmh_sweep(
                    self.phi, self.S, self.sq, r, Lc, mu, beta_new, c.L, c.m2, c.lam, c.c_kin, c.c_mass,
                    c.keep_reference, c.seed, c.stream, t, s)
                n_acc += int(acc.sum())
        else:
            for s in range(c.n_mcmc):
                self.phi, self.S, self.sq, acc = mutation.rw_sweep(
                    self.phi, self.S, self.sq, Lc, c.scale, beta_new, c.L, c.m2, c.lam, c.c_kin, c.c_mass,
                    c.keep_reference, c.seed, c.stream, t, s, c.normal_bits)
                n_acc += int(acc.sum())
        if c.z2_flip:
            self.phi = z2_flip(self.phi, c.seed, c.stream, t)
        self.ell = lattice.tempering_loglik(self.S, self.sq, c.D, c.keep_reference)
        self.beta = beta_new
        rec = {"t": t, "beta": beta_new, "dbeta": dbeta, "ess": ess, "logz_inc": inc,
               "logz": self.logz.s, "acc_rate": n_acc / float(c.N * max(c.n_mcmc, 1))}
        self.history.append(rec)
        return rec

    def run(self):
        while not self.done and self.t < self.cfg.max_steps:
            self.temper_step()
        return self.result()

    def result(self):
        obs = observables.summary(self.phi)
        obs.update({"logz": self.logz.s, "beta": self.beta, "n_steps": self.t})
        return obs


def run(cfg: SMCConfig):
    return SMC(cfg).run()
