"""Time to a log Z within +-tol (the evidence estimate of Sec. 2 and App. E, as a cost):
for each arithmetic form, the wall time of one run at the cheapest (N, rho, sweeps) cell
of a grid whose seeds' mean log Z lies within tol of a reference value and whose
seed-to-seed standard deviation is at most tol. The reference is the pooled mean of the
reference form's runs at the grid's most expensive cell.

Workload: broken-phase phi^4 (m2 = -4, lambda = 8), n_mcmc random-walk sweeps per
temperature, runs from beta = 0 to 1. The number of sweeps is a grid axis because the
estimate's bias depends on it: the proposal covariance is estimated from the population
it moves, and with few sweeps per temperature that biases log Z upwards by far more than
the tolerance at large D.

    python -m paper_2511_15196_gb300.time_to_logz [--L 64] [--N 8192 16384 32768 65536]
        [--rho 0.5 0.9] [--n-mcmc 20] [--seeds 32] [--forms mixed fp32] [--ref-form fp64]
        [--tol 0.05]
"""
import argparse
import json
import math
import statistics
import time

FORMS = {"fp64": 0, "fp32": 1, "mixed": 2}


def cells(Ns, rhos, sweeps=(20,)):
    """Grid cells (N, rho, n_mcmc) in increasing cost: by the mutation work per
    temperature N * n_mcmc, then by rho (a higher ESS target means more temperatures),
    then by N."""
    return sorted(((N, rho, m) for N in Ns for rho in rhos for m in sweeps),
                  key=lambda c: (c[0] * c[2], c[1], c[0]))


def summarise(logz, ms):
    m = sum(logz) / len(logz)
    sd = statistics.stdev(logz) if len(logz) > 1 else math.inf
    return {"logz_mean": m, "logz_sd": sd, "ms_per_run": statistics.median(ms), "seeds": len(logz)}


def first_within(rows, ref, tol):
    """The first row (rows in increasing cost) with |mean - ref| <= tol and sd <= tol."""
    for r in rows:
        if abs(r["logz_mean"] - ref) <= tol and r["logz_sd"] <= tol:
            return r
    return None


def gpu_runner(L, N, rho, form, seed, n_mcmc):
    """One run to beta = 1 on the GPU: (log Z, wall milliseconds)."""
    import torch
    from . import Config, Run
    cfg = Config(L=L, N=N, m2=-4.0, lam=8.0, precision=FORMS[form], n_mcmc=n_mcmc, ess_target=rho, seed=seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run = Run(cfg)
    obs = run.run()
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    run.close()
    return obs["logz"], ms


def run_cell(L, N, rho, form, seeds, n_mcmc, runner=gpu_runner, seed0=0):
    res = [runner(L, N, rho, form, seed0 + s, n_mcmc) for s in range(seeds)]
    row = summarise([r[0] for r in res], [r[1] for r in res])
    row.update({"L": L, "N": N, "rho": rho, "form": form, "n_mcmc": n_mcmc})
    return row


def measure(L, Ns, rhos, forms, ref_form, seeds, tol, n_mcmc, runner=gpu_runner, emit=print):
    """n_mcmc: sweeps per temperature, one value or a list of them (a grid axis)."""
    sweeps = [n_mcmc] if isinstance(n_mcmc, int) else list(n_mcmc)
    grid = cells(Ns, rhos, sweeps)
    N_ref, rho_ref, m_ref = grid[-1]
    ref_row = run_cell(L, N_ref, rho_ref, ref_form, seeds, m_ref, runner, seed0=10000)
    ref = ref_row["logz_mean"]
    emit(json.dumps({"reference": ref_row}))
    out = {}
    for form in forms:
        rows = []
        hit = None
        for N, rho, m in grid:
            row = run_cell(L, N, rho, form, seeds, m, runner)
            rows.append(row)
            emit(json.dumps(row))
            hit = first_within(rows, ref, tol)
            if hit is not None:
                break
        out[form] = {"time_to_logz_s": hit["ms_per_run"] * 1e-3 if hit else None,
                     "cell": {"N": hit["N"], "rho": hit["rho"], "n_mcmc": hit["n_mcmc"]} if hit else None,
                     "logz_ref": ref, "tol": tol}
        emit(json.dumps({"form": form, **out[form]}))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--L", type=int, default=64)
    ap.add_argument("--N", type=int, nargs="+", default=[8192, 16384, 32768, 65536])
    ap.add_argument("--rho", type=float, nargs="+", default=[0.5, 0.9])
    ap.add_argument("--seeds", type=int, default=32)
    ap.add_argument("--forms", nargs="+", default=["mixed", "fp32"], choices=list(FORMS))
    ap.add_argument("--ref-form", default="fp64", choices=list(FORMS))
    ap.add_argument("--tol", type=float, default=0.05)
    ap.add_argument("--n-mcmc", type=int, nargs="+", default=[20])
    a = ap.parse_args()
    measure(a.L, a.N, a.rho, a.forms, a.ref_form, a.seeds, a.tol, a.n_mcmc)


if __name__ == "__main__":
    main()
