"""Time to a log Z within +-tol (the evidence estimate of Sec. 2 and App. E, as a cost):
for each arithmetic form, the wall time of one run at the cheapest (N, rho, sweeps) cell
of a grid whose seeds' mean log Z lies within tol of a reference value and whose
seed-to-seed standard deviation is at most tol. The reference is the pooled mean of the
reference form's runs at the grid's most expensive cell.

Workloads: broken-phase phi^4 (m2 = -4, lambda = 8; default), or with --free the free
field (m2 = 1, lambda = 0), whose log Z has a closed form that then serves as the
reference (no reference runs). n_mcmc random-walk sweeps per temperature, runs from
beta = 0 to 1. The number of sweeps is a grid axis because the estimate's bias depends on
it: the proposal covariance is estimated from the population it moves, and with few
sweeps per temperature that biases log Z upwards by far more than the tolerance at large
D. --kernel-cov gaussian replaces that covariance by the exact one of the tempered
Gaussian part (PHI4_FLAG_FREE_KERNEL_COV; the target's own for the free field), which
does not depend on the particles.

    python -m paper_2511_15196_gb300.time_to_logz [--L 64] [--N 8192 16384 32768 65536]
        [--rho 0.5 0.9] [--n-mcmc 20] [--seeds 32] [--forms mixed fp32] [--ref-form fp64]
        [--tol 0.05] [--free] [--kernel-cov population|gaussian] [--confirm-seeds 8]
"""
import argparse
import json
import math
import statistics
import time

FORMS = {"fp64": 0, "fp32": 1, "mixed": 2}


def free_field_logz(L, m2):
    """log Z = (D/2) log pi - (1/2) sum_k log(m2 + sum_mu 4 sin^2(pi k_mu / L)) of the free
    field with the unhalved action (the closed form of the workload statement)."""
    s = [4.0 * math.sin(math.pi * k / L) ** 2 for k in range(L)]
    return 0.5 * L * L * math.log(math.pi) - 0.5 * sum(math.log(m2 + a + b) for a in s for b in s)


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
        if "given_up_after" not in r and abs(r["logz_mean"] - ref) <= tol and r["logz_sd"] <= tol:
            return r
    return None


MODEL = {"m2": -4.0, "lam": 8.0, "flags": 0}


def gpu_runner(L, N, rho, form, seed, n_mcmc):
    """One run to beta = 1 on the GPU: (log Z, wall milliseconds)."""
    import torch
    from . import Config, Run
    cfg = Config(L=L, N=N, m2=MODEL["m2"], lam=MODEL["lam"], flags=MODEL["flags"], precision=FORMS[form],
                 n_mcmc=n_mcmc, ess_target=rho, seed=seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run = Run(cfg)
    obs = run.run()
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    run.close()
    return obs["logz"], ms


def run_cell(L, N, rho, form, seeds, n_mcmc, runner=gpu_runner, seed0=0, ref=None, tol=None, early=0):
    """Runs `seeds` seeds of a cell. With early > 1 and a reference, the cell is given up
    after its first `early` seeds when their mean lies more than tol + 5 standard errors
    from the reference (it cannot end within tol); the row then says so."""
    res = [runner(L, N, rho, form, seed0 + s, n_mcmc) for s in range(min(seeds, early) if early > 1 else seeds)]
    if early > 1 and ref is not None and len(res) < seeds:
        head = summarise([r[0] for r in res], [r[1] for r in res])
        if abs(head["logz_mean"] - ref) > tol + 5.0 * head["logz_sd"] / math.sqrt(len(res)):
            head.update({"L": L, "N": N, "rho": rho, "form": form, "n_mcmc": n_mcmc, "given_up_after": len(res)})
            return head
        res += [runner(L, N, rho, form, seed0 + s, n_mcmc) for s in range(len(res), seeds)]
    row = summarise([r[0] for r in res], [r[1] for r in res])
    row.update({"L": L, "N": N, "rho": rho, "form": form, "n_mcmc": n_mcmc})
    return row


def measure(L, Ns, rhos, forms, ref_form, seeds, tol, n_mcmc, runner=gpu_runner, emit=print, exact=None,
            confirm_seeds=0, early=0):
    """n_mcmc: sweeps per temperature, one value or a list of them (a grid axis).
    exact: a known log Z (closed form) used as the reference instead of reference runs.
    confirm_seeds > 0: only the first form scans the grid; every other form is run at the
    first form's cell (and at the cell before it in cost order, when there is one) with
    that many seeds, its time there reported (the forms run the same sampler, so they reach
    the tolerance at the same cell; the rows show whether they do)."""
    sweeps = [n_mcmc] if isinstance(n_mcmc, int) else list(n_mcmc)
    grid = cells(Ns, rhos, sweeps)
    if exact is None:
        N_ref, rho_ref, m_ref = grid[-1]
        ref_row = run_cell(L, N_ref, rho_ref, ref_form, seeds, m_ref, runner, seed0=10000)
        ref = ref_row["logz_mean"]
        emit(json.dumps({"reference": ref_row}))
    else:
        ref = exact
        emit(json.dumps({"reference": {"closed_form": exact}}))
    out = {}
    for fi, form in enumerate(forms):
        if confirm_seeds > 0 and fi > 0:
            first = out[forms[0]]["cell"]
            if first is None:
                out[form] = {"time_to_logz_s": None, "cell": None, "logz_ref": ref, "tol": tol}
                emit(json.dumps({"form": form, **out[form]}))
                continue
            idx = grid.index((first["N"], first["rho"], first["n_mcmc"]))
            rows = []
            for N, rho, m in grid[max(0, idx - 1):idx + 1]:
                row = run_cell(L, N, rho, form, confirm_seeds, m, runner)
                rows.append(row)
                emit(json.dumps(row))
            hit = rows[-1]
            ok = abs(hit["logz_mean"] - ref) <= tol and hit["logz_sd"] <= tol
            out[form] = {"time_to_logz_s": hit["ms_per_run"] * 1e-3, "cell": first, "logz_ref": ref, "tol": tol,
                         "within_tol_at_cell": ok, "seeds": confirm_seeds}
            emit(json.dumps({"form": form, **out[form]}))
            continue
        rows = []
        hit = None
        for N, rho, m in grid:
            row = run_cell(L, N, rho, form, seeds, m, runner, ref=ref, tol=tol, early=early)
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
    ap.add_argument("--free", action="store_true", help="free field m2 = 1, lambda = 0 against its closed form")
    ap.add_argument("--kernel-cov", default="population", choices=["population", "gaussian"])
    ap.add_argument("--confirm-seeds", type=int, default=0)
    ap.add_argument("--early-seeds", type=int, default=0,
                    help="give a cell up after this many seeds when it cannot end within the tolerance")
    a = ap.parse_args()
    exact = None
    if a.free:
        MODEL.update(m2=1.0, lam=0.0)
        exact = free_field_logz(a.L, 1.0)
    if a.kernel_cov == "gaussian":
        from . import FLAG_FREE_KERNEL_COV
        MODEL["flags"] = FLAG_FREE_KERNEL_COV
    measure(a.L, a.N, a.rho, a.forms, a.ref_form, a.seeds, a.tol, a.n_mcmc, exact=exact,
            confirm_seeds=a.confirm_seeds, early=a.early_seeds)


if __name__ == "__main__":
    main()
