"""Target-ESS sweep of the SMC-RW sampler in the paper's own setting (Sec. 3, App. A and
App. E): the 10 x 10 lattice with the action of Eq. (1) (kinetic and mass terms with
factor 1/2), m^2 = -4, lambda = 1, the target exp(-U_0 - S) that keeps the Gaussian
reference at beta = 1, N = 5000 particles and n_MCMC = 3 V random-walk sweeps per
temperature (App. E uses 500). For each target ESS it runs several seeds through the
library and reports the mean and spread of log Z, the number of temperatures and
likelihood evaluations, the acceptance rate, the mode balance and the wall time per run.
The library's log Z in this mode is log E_{N(0,I)}[exp(-S_E)]; the values the paper prints
(Tables 1, 3 and 4: about -65.3 at L = 10, -146 at 15, -210 at 18) equal it minus
(V/4) log(pi) at all three sizes, so `logz_paper_convention` reports that difference too.

    python -m paper_2511_15196_gb300.ess_sweep [--ess 0.9 0.99 0.999] [--seeds 4] [--n-mcmc 300] [--L 10]
                                               [--irmh | --hmc] [--fp32]
"""
import argparse
import json
import math
import time


def paper_config(ess, seed, n_mcmc=300, N=5000, precision=None, L=10, kind=None):
    from . import FP64, SMC_RW, Config
    return Config(L=L, N=N, m2=-4.0, lam=1.0, c_kin=0.5, c_mass=0.5, keep_reference=True,
                  precision=FP64 if precision is None else precision, n_mcmc=n_mcmc, ess_target=ess, seed=seed,
                  kind=SMC_RW if kind is None else kind)


def run_one(cfg):
    """One run to beta = 1: (observables, GPU milliseconds)."""
    import torch
    from . import Run
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run = Run(cfg)
    obs = run.run()
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    run.close()
    return obs, ms


def sweep(ess_targets, seeds, n_mcmc=None, N=5000, L=10, kind=None, precision=None):
    """n_mcmc defaults to 3 V (App. A); kind: SMC_RW (default), SMC_IRMH or SMC_HMC;
    precision: FP64 (default), FP32 or MIXED_BF16."""
    if n_mcmc is None:
        n_mcmc = 3 * L * L
    rows = []
    for ess in ess_targets:
        res = [run_one(paper_config(ess, s, n_mcmc=n_mcmc, N=N, L=L, kind=kind, precision=precision))
               for s in range(seeds)]
        lz = [o["logz"] for o, _ in res]
        m = sum(lz) / len(lz)
        sd = math.sqrt(sum((x - m) ** 2 for x in lz) / max(len(lz) - 1, 1))
        rows.append({"ess_target": ess, "seeds": seeds, "logz_mean": m, "logz_sd": sd,
                     "L": L, "kind": {2: "irmh", 3: "hmc"}.get(kind, "rw"),
                     "precision": {1: "fp32", 2: "mixed_bf16"}.get(precision, "fp64"),
                     "logz_paper_convention": m - L * L / 4 * math.log(math.pi),
                     "temperatures": sum(o["n_steps"] for o, _ in res) / len(res),
                     "likelihood_evals": sum(o["n_likelihood_evals"] for o, _ in res) / len(res),
                     "acc_rate": sum(o["acc_rate"] for o, _ in res) / len(res),
                     "mode_balance": sum(o["mode_balance"] for o, _ in res) / len(res),
                     "ms_per_run": sum(t for _, t in res) / len(res)})
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--ess", type=float, nargs="+", default=[0.9, 0.99, 0.999])
    ap.add_argument("--seeds", type=int, default=4)
    ap.add_argument("--n-mcmc", type=int, default=None, help="sweeps per temperature (default 3 V)")
    ap.add_argument("--N", type=int, default=5000)
    ap.add_argument("--L", type=int, default=10)
    ap.add_argument("--irmh", action="store_true", help="independent Metropolis-Hastings sweeps (SMC-IRMH)")
    ap.add_argument("--hmc", action="store_true", help="HMC transitions, 20 leapfrog steps (SMC-HMC)")
    ap.add_argument("--fp32", action="store_true", help="the float arithmetic form")
    a = ap.parse_args()
    kind = 2 if a.irmh else 3 if a.hmc else None
    for row in sweep(a.ess, a.seeds, n_mcmc=a.n_mcmc, N=a.N, L=a.L, kind=kind, precision=1 if a.fp32 else None):
        print(json.dumps(row))


if __name__ == "__main__":
    main()
