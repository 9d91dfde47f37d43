"""Bias of the SMC evidence from the population-estimated proposal covariance (oracle study).

Test infrastructure, like the rest of ``tests/``: it runs the FP64 oracle only. The
random-walk kernel of a temperature uses the covariance of the population it is about
to move (App. A). On the free field (lam = 0, m2 = 1), where log Z has a closed form,
this prints log Zhat - log Z over a few seeds

* against the number of sweeps per temperature and the target ESS (population
  covariance),
* against the number of particles at the workload's 10 sweeps and ESS 0.5 N,
* with the exact covariance of the tempered free field in place of the population's
  (the control: the driver is then exact and only the usual -Var/2 remains),
* the final population's mean |phi|^2 against its exact value (the contraction),
* with three other estimates of the covariance: each half of the resampled population
  moved with the other half's covariance, the importance-weighted covariance of the
  population before resampling, and the covariance of an independent replica population
  on the same temperature schedule,
* optionally (--L32) one run of the 32 x 32 precision-check workload
  (N = 4096, ESS 0.5 N, 10 sweeps or --L32-sweeps) with each covariance (about 10
  minutes at 10 sweeps, two hours at 100),
* optionally (--L16) the 16 x 16 free field at the same D/N = 1/4 as the 32 x 32 run
  (N = 1024, 10 and 100 sweeps, two seeds),
* optionally (--broken) the interacting 8 x 8 workload (m2 = -4, lam = 8, N = 1024),
  which has no closed form, as the sweeps per temperature grow.

    python tests/study_covariance_bias.py [--L16] [--L32 [--L32-sweeps 100]] [--broken]
"""
import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
for p in (os.path.dirname(HERE), HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import numpy as np  # noqa: E402

import closed_forms as cf  # noqa: E402
from oracle import covariance, lattice, mutation, philox, resample, tempering  # noqa: E402
from oracle.smc import SMC, SMCConfig  # noqa: E402


def broken_phase(seeds):
    # (sweeps, ESS target, seeds) in increasing cost
    for n_mcmc, rho, ns in ((10, 0.5, seeds), (50, 0.9, seeds), (200, 0.9, 2), (800, 0.9, 1)):
        t0 = time.time()
        lz = np.array([SMC(SMCConfig(L=8, N=1024, m2=-4.0, lam=8.0, rho=rho, n_mcmc=n_mcmc, seed=s)).run()["logz"]
                       for s in range(ns)])
        sd = lz.std(ddof=1) if ns > 1 else float("nan")
        print("%-46s log Zhat = %8.3f  (sd %.3f, %d seeds, %.0f s)"
              % ("L=8 m2=-4 lam=8 N=1024 sweeps=%d ESS=%.1fN" % (n_mcmc, rho), lz.mean(), sd, ns, time.time() - t0),
              flush=True)


def variant_logz(L, N, seed, mode, rho=0.5, n_mcmc=10):
    """The SMC driver's temperature step written out with another covariance estimate:
    mode "split" moves each half of the resampled population with the covariance of the
    other half; mode "weighted" uses the importance-weighted covariance of the population
    before resampling."""
    c = SMCConfig(L=L, N=N, m2=1.0, lam=0.0, rho=rho, n_mcmc=n_mcmc, seed=seed)
    s = SMC(c)
    while not s.done:
        s.t += 1
        t = s.t
        dbeta = s.choose_dbeta()
        beta_new = 1.0 if dbeta >= 1.0 - s.beta else s.beta + dbeta
        w, inc = tempering.reweight(s.ell, dbeta)
        s.logz.add(inc)
        if mode == "weighted":
            wn = w / w.sum()
            Xc = s.phi - wn @ s.phi
            Sig = (Xc * wn[:, None]).T @ Xc / (1.0 - (wn * wn).sum())
        anc = resample.systematic(w, philox.word32(c.seed, c.stream, philox.KIND_RESAMPLE, t))
        s.phi, s.S, s.sq = s.phi[anc], s.S[anc], s.sq[anc]
        if mode == "weighted":
            groups = [(np.arange(N), Sig, 0)]
        else:
            perm = np.random.default_rng([seed, t]).permutation(N)
            A, B = perm[: N // 2], perm[N // 2:]
            groups = [(A, covariance.sample_covariance(s.phi[B])[1], 0), (B, covariance.sample_covariance(s.phi[A])[1], 1)]
        for own, Sig_g, stream in groups:
            Lc = covariance.regularised_cholesky(Sig_g, c.jitter_rel)[0]
            ph, S, sq = s.phi[own], s.S[own], s.sq[own]
            for k in range(n_mcmc):
                ph, S, sq, _ = mutation.rw_sweep(ph, S, sq, Lc, c.scale, beta_new, L, 1.0, 0.0, 1.0, 1.0, False,
                                                 seed, stream, t, k)
            s.phi[own], s.S[own], s.sq[own] = ph, S, sq
        s.ell = lattice.tempering_loglik(s.S, s.sq, c.D)
        s.beta = beta_new
    return s.logz.s


def replica_logz(L, N, seed, rho=0.5, n_mcmc=10):
    """Two independent populations on one temperature schedule (the first's adaptive
    one): each is moved with the covariance of the other, so no kernel depends on the
    particles it moves or on their copies. Returns the first population's log Zhat."""
    cA = SMCConfig(L=L, N=N, m2=1.0, lam=0.0, rho=rho, n_mcmc=n_mcmc, seed=seed)
    cB = SMCConfig(L=L, N=N, m2=1.0, lam=0.0, rho=rho, n_mcmc=n_mcmc, seed=seed + 7919)
    A, B = SMC(cA), SMC(cB)
    while not A.done:
        A.t += 1
        B.t += 1
        dbeta = A.choose_dbeta()
        beta_new = 1.0 if dbeta >= 1.0 - A.beta else A.beta + dbeta
        for r, c in ((A, cA), (B, cB)):
            w, inc = tempering.reweight(r.ell, dbeta)
            r.logz.add(inc)
            anc = resample.systematic(w, philox.word32(c.seed, c.stream, philox.KIND_RESAMPLE, r.t))
            r.phi, r.S, r.sq = r.phi[anc], r.S[anc], r.sq[anc]
        LA = covariance.regularised_cholesky(covariance.sample_covariance(B.phi)[1], cA.jitter_rel)[0]
        LB = covariance.regularised_cholesky(covariance.sample_covariance(A.phi)[1], cB.jitter_rel)[0]
        for r, c, Lc in ((A, cA, LA), (B, cB, LB)):
            for k in range(n_mcmc):
                r.phi, r.S, r.sq, _ = mutation.rw_sweep(r.phi, r.S, r.sq, Lc, c.scale, beta_new, L, 1.0, 0.0, 1.0,
                                                        1.0, False, c.seed, c.stream, r.t, k)
            r.ell = lattice.tempering_loglik(r.S, r.sq, c.D)
            r.beta = beta_new
    return A.logz.s


def logz_seeds(L, N, rho, n_mcmc, seeds, exact_covariance=False):
    """log Zhat of the free field for seeds 0..seeds-1; with ``exact_covariance`` the
    kernel covariance at each new temperature is the tempered free field's own."""
    saved = (tempering.bisect_dbeta, covariance.sample_covariance)
    if exact_covariance:
        state = {}

        def recording_bisect(ell, beta, rho_, iters=64):
            d, used = saved[0](ell, beta, rho_, iters)
            state["beta"] = min(1.0, beta + d)
            return d, used
        tempering.bisect_dbeta = recording_bisect
        covariance.sample_covariance = lambda X: (X.mean(axis=0), cf.free_field_covariance(L, 1.0, state["beta"]))
    try:
        return np.array([SMC(SMCConfig(L=L, N=N, m2=1.0, lam=0.0, rho=rho, n_mcmc=n_mcmc, seed=s)).run()["logz"]
                         for s in range(seeds)])
    finally:
        tempering.bisect_dbeta, covariance.sample_covariance = saved


def report(label, L, lz, t0):
    ref = cf.free_field_logz(L, 1.0)
    sd = lz.std(ddof=1) if len(lz) > 1 else float("nan")
    print("%-46s log Zhat - log Z = %+8.3f  (sd %.3f, %d seeds, %.0f s)"
          % (label, lz.mean() - ref, sd, len(lz), time.time() - t0), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L32", action="store_true", help="also run the 32 x 32, N = 4096 workload once (minutes)")
    ap.add_argument("--L16", action="store_true", help="also the 16 x 16 free field at N = 1024, 10 and 100 sweeps")
    ap.add_argument("--broken", action="store_true", help="also the interacting 8 x 8 workload (minutes)")
    ap.add_argument("--L32-sweeps", type=int, default=10, help="sweeps per temperature of the --L32 runs")
    ap.add_argument("--seeds", type=int, default=4)
    a = ap.parse_args()
    L = 8
    for n_mcmc in (10, 50, 200):
        for rho in (0.5, 0.9):
            t0 = time.time()
            report("L=8 N=1024 sweeps=%d ESS=%.1fN" % (n_mcmc, rho), L, logz_seeds(L, 1024, rho, n_mcmc, a.seeds), t0)
    for N in (256, 4096):
        t0 = time.time()
        report("L=8 N=%d sweeps=10 ESS=0.5N" % N, L, logz_seeds(L, N, 0.5, 10, a.seeds), t0)
    # the controls have a large spread: 32 seeds
    n_ctl = max(a.seeds, 32)
    t0 = time.time()
    lz = logz_seeds(L, 1024, 0.5, 10, n_ctl, exact_covariance=True)
    report("L=8 N=1024 sweeps=10 ESS=0.5N exact covariance", L, lz, t0)
    print("%-46s mean + var/2 - log Z = %+.3f" % ("", lz.mean() + 0.5 * lz.var(ddof=1) - cf.free_field_logz(L, 1.0)))
    t0 = time.time()
    report("L=8 N=1024 sweeps=10 ESS=0.5N replica", L, np.array([replica_logz(L, 1024, s) for s in range(n_ctl)]), t0)
    for n_mcmc in (10, 200):
        r = SMC(SMCConfig(L=L, N=1024, m2=1.0, lam=0.0, rho=0.5, n_mcmc=n_mcmc, seed=0))
        r.run()
        print("%-46s mean |phi|^2 of the final population %.3f (exact %.3f)"
              % ("L=8 N=1024 sweeps=%d ESS=0.5N seed 0" % n_mcmc, float((r.phi ** 2).sum(axis=1).mean()),
                 cf.free_field_sq_mean(L, 1.0)), flush=True)
    for mode in ("split", "weighted"):
        t0 = time.time()
        report("L=8 N=1024 sweeps=10 ESS=0.5N %s" % mode, L,
               np.array([variant_logz(L, 1024, s, mode) for s in range(a.seeds)]), t0)
    if a.L16:
        for n_mcmc in (10, 100):
            t0 = time.time()
            report("L=16 N=1024 sweeps=%d ESS=0.5N" % n_mcmc, 16, logz_seeds(16, 1024, 0.5, n_mcmc, 2), t0)
    if a.broken:
        broken_phase(a.seeds)
    if a.L32:
        m = a.L32_sweeps
        t0 = time.time()
        report("L=32 N=4096 sweeps=%d ESS=0.5N" % m, 32, logz_seeds(32, 4096, 0.5, m, 1), t0)
        t0 = time.time()
        report("L=32 N=4096 sweeps=%d ESS=0.5N exact covariance" % m, 32,
               logz_seeds(32, 4096, 0.5, m, 1, exact_covariance=True), t0)
    print("closed forms: L=8 %.10f  L=32 %.10f" % (cf.free_field_logz(8, 1.0), cf.free_field_logz(32, 1.0)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
