"""Scan of the kappa-parameterised phi^4 action (App. G) with the SMC-RW sampler: for each
nearest-neighbour coupling kappa at fixed lambda, one run per seed to beta = 1 on the
target exp(-S_kappa) (the Gaussian reference tempered away), reporting log Z of the kappa
form (the library's log Z plus the -lambda V of the dropped constant), <|M|>, the
susceptibility chi = V (<M^2> - <M>^2), the mode balance and the acceptance rate. With the
global Z2 move (flags) the two modes stay balanced, so <M> ~ 0 and chi measures the
fluctuation of M across both modes.

    python -m paper_2511_15196_gb300.scans [--L 16] [--lam 1.0] [--kappa 0.1 0.2 0.3 0.4]
"""
import argparse
import json


def scan(kappas, lam=1.0, L=16, N=4096, n_mcmc=20, seeds=2, z2_flip=True, precision=None):
    from . import FLAG_Z2_FLIP, MIXED_BF16, FP64, Run, kappa_config, kappa_logz_shift
    if precision is None:
        precision = MIXED_BF16 if L % 4 == 0 else FP64
    D = L * L
    rows = []
    for kappa in kappas:
        res = []
        for seed in range(seeds):
            cfg = kappa_config(kappa, lam, L=L, N=N, n_mcmc=n_mcmc, ess_target=0.5, precision=precision, seed=seed,
                               flags=FLAG_Z2_FLIP if z2_flip else 0)
            run = Run(cfg)
            o = run.run()
            run.close()
            res.append(o)
        mean = lambda k: sum(o[k] for o in res) / len(res)  # noqa: E731
        rows.append({"kappa": kappa, "lambda": lam, "L": L, "seeds": seeds,
                     "logz_kappa": mean("logz") + kappa_logz_shift(lam, D), "mean_absM": mean("mean_absM"),
                     "chi": mean("chi"), "mode_balance": mean("mode_balance"), "acc_rate": mean("acc_rate"),
                     "temperatures": mean("n_steps")})
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--lam", type=float, default=1.0)
    ap.add_argument("--kappa", type=float, nargs="+", default=[0.1, 0.2, 0.3, 0.4, 0.5])
    ap.add_argument("--seeds", type=int, default=2)
    ap.add_argument("--no-flip", action="store_true")
    a = ap.parse_args()
    for row in scan(a.kappa, a.lam, a.L, seeds=a.seeds, z2_flip=not a.no_flip):
        print(json.dumps(row))


if __name__ == "__main__":
    main()
