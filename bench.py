"""Benchmark of the SMC temperature step on GB300.

Workload (default): adaptive tempered SMC with random-walk moves on the broken
phase of lattice phi^4, L = 64 (D = 4096 sites), N = 8192 particles, m2 = -4,
lambda = 8, 20 Metropolis sweeps per temperature, target ESS 0.5 N, proposal and
covariance GEMMs on the tcgen05 tensor cores in bf16 with fp32 accumulation,
FP64 Cholesky, acceptance test and compensated log Z.

One step = one temperature: ESS bisection and reweighting, systematic
resampling, particle gather, covariance, Cholesky, 20 x (normals, proposal GEMM,
stencil accept). Metric: site updates per second = N * D * n_mcmc per step over
the whole step's device time (K steps timed with CUDA events on the run's stream,
barrier + synchronize on both sides, max over ranks). The state (fields,
proposals, normals: about 320 MiB per sweep) is larger than L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp32|fp64]
  python bench.py --sampler hmc --precision fp32   # SMC-HMC steps (20 leapfrog steps per transition)
  python bench.py --impl reference     # the FP64 CPU oracle on a bounded sample

With --gpus N > 1 (torchrun) each rank advances its own independent replica
(the sampler has no data-parallel exchange at this size: "replicas only").
"""
import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PREC = {"mixed": 2, "fp32": 1, "fp64": 0}
PREC_DTYPE = {"mixed": "bf16-gemm/fp32-state/fp64-accept", "fp32": "fp32 (fp64 log Z)", "fp64": "fp64"}
METRIC = "site-updates/s in mutation; time-to-logZ(±0.05) mixed vs FP32 at L=64, 1 GB300"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=list(PREC))
    ap.add_argument("--L", type=int, default=64)
    ap.add_argument("--N", type=int, default=8192)
    ap.add_argument("--n-mcmc", type=int, default=20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=2048, help="particles in the oracle's bounded sample")
    ap.add_argument("--sampler", default="rw", choices=["rw", "hmc"],
                    help="rw: random-walk sweeps (default); hmc: HMC transitions (fp32 or fp64)")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "kernels"],
                    help="single: one L=64 run; batch: 64 independent runs of mixed lattice sizes")
    ap.add_argument("--batch-runs", type=int, default=64)
    ap.add_argument("--fp32-steps", type=int, default=3,
                    help="temperatures of the plain FP32 comparator timed after the mixed form (0: skip)")
    return ap.parse_args()


def batch_configs(p, n_runs, n_mcmc):
    """64 independent runs: L in {8,12,16,24,32} round-robin, N in {1024,2048,4096} by seed,
    lambda in {4,8,16} by (run // 3), m2 = -4, float fields with bf16 tensor-core GEMMs."""
    cfgs = []
    for r in range(n_runs):
        cfgs.append(p.Config(L=[8, 12, 16, 24, 32][r % 5], N=[1024, 2048, 4096][r % 3], m2=-4.0,
                             lam=[4.0, 8.0, 16.0][(r // 3) % 3], precision=p.MIXED_BF16, n_mcmc=n_mcmc,
                             ess_target=0.5, seed=r))
    return cfgs


def run_batch(a):
    import torch
    import paper_2511_15196_gb300 as p
    rank, world, dist = dist_setup(a)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    n_mcmc = a.n_mcmc if a.n_mcmc != 20 else 10
    cfgs = batch_configs(p, a.batch_runs, n_mcmc)
    for c in cfgs:
        c.seed += 100000 * rank
    stream = torch.cuda.current_stream()
    units = lambda b: sum(c.N * c.L * c.L * c.n_mcmc for c, m in zip(b.cfgs, b.members) if m.observables()["beta"] < 1.0)
    b = p.Batch(cfgs)
    for _ in range(a.warmup):
        if b.temper_step() == 0:
            b = p.Batch(cfgs)
    l0 = sum(m.kernel_launches() for m in b.members)
    total_units = 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    elapsed = 0.0
    with Clocks(local) as clk:
        for _ in range(a.steps):
            u = units(b)
            if u == 0:
                b = p.Batch(cfgs)
                u = units(b)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            b.temper_step()
            ev1.record(stream)
            torch.cuda.synchronize()
            elapsed += ev0.elapsed_time(ev1)
            total_units += u
    launches = sum(m.kernel_launches() for m in b.members) - l0 + 2 * a.steps
    elapsed = max_over_ranks(elapsed, dist)
    value = world * total_units / (elapsed * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": elapsed / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": PREC_DTYPE["mixed"], "data": "synthetic (Philox N(0,I) initial fields)",
            "config": {"workload": "batched SMC-RW: %d independent runs, L in {8,12,16,24,32} round-robin, "
                                   "N in {1024,2048,4096} by seed, lambda in {4,8,16}, m2=-4, %d RWM sweeps, "
                                   "ESS 0.5N, bf16 tensor-core GEMMs" % (a.batch_runs, n_mcmc),
                       "runs": a.batch_runs, "l2": "per-step working set of all runs (~1.5 GB) larger than L2"},
            "gpu_launches": launches, "clocks": clk.summary(), "tuning": b.tuning()}
    if rank == 0:
        print(json.dumps(line))
    b.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_kernels(a):
    """The hot kernels one by one at the benchmark size, through the kernel-level C ABI, for
    ncu captures (no timing, no JSON line): two proposal GEMMs, two fused accepts, two FP64
    Cholesky factorisations of a 4096 x 4096 SPD matrix, three bf16 normal draws, two mixed
    covariances (exact Gram of fixed-point digits) of the 8192 x 4096 population."""
    import torch
    import paper_2511_15196_gb300 as p
    N, L = 8192, 64
    D = L * L
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    phi = 0.5 * torch.randn(N, D, device="cuda", generator=g)
    Lc = torch.tril(0.02 * torch.randn(D, D, device="cuda", dtype=torch.float64, generator=g)) + \
        0.3 * torch.eye(D, device="cuda", dtype=torch.float64)
    Lb = Lc.to(torch.bfloat16)
    for i in range(2):
        p.rw_propose(phi, Lb, p.MIXED_BF16, 2.38 / L, 1, 0, 1, i)
    S, sq = p.action(phi, L, -4.0, 8.0)
    ell = -S + 0.5 * sq
    delta = (0.01 * torch.randn(N, D, device="cuda", generator=g)).half()
    for i in range(2):
        p.rw_accept_delta(phi.clone(), delta, L, -4.0, 8.0, S.clone(), sq.clone(), ell.clone(), 0.02, 1, 0, 1, i)
    A = torch.randn(D, D, device="cuda", dtype=torch.float64, generator=g) * 0.01
    A = A @ A.T + torch.eye(D, device="cuda", dtype=torch.float64)
    for i in range(2):
        p.cholesky(A.clone(), 1e-8)
    Zb = torch.empty(N, D, dtype=torch.bfloat16, device="cuda")
    for i in range(3):
        p.philox_normals(Zb, 7, 0, p.RNG_PROPOSE, 1, i)
    for i in range(2):
        p.covariance(phi, p.MIXED_BF16)
    torch.cuda.synchronize()
    print("kernels workload done")
    return 0


HMC_LEAPFROG = 20
# algorithmic work of one HMC transition per site: 21 momentum kicks (gradient: 3 adds for
# the neighbour sum, 2 multiplies for x^3, A x + B nb + C x^3 as a multiply and 2 FMAs, then
# the FMA y += h e g: 12 flop) and 20 drifts (one FMA: 2 flop); shared-memory traffic: 4
# neighbour loads per kick and one store per drift
HMC_FLOP_PER_SITE = (HMC_LEAPFROG + 1) * 12 + HMC_LEAPFROG * 2


def hmc_smem_bytes_per_site(prec):
    return ((HMC_LEAPFROG + 1) * 4 + HMC_LEAPFROG) * (8 if prec == 0 else 4)


def workload(a):
    D = a.L * a.L
    if a.sampler == "hmc":
        return {"workload": "SMC-HMC tempering step, broken-phase phi^4 L=%d (D=%d), N=%d, m2=-4, lambda=8, "
                            "%d HMC transitions/temperature (%d leapfrog steps, covariance-diagonal inverse mass), "
                            "ESS 0.5N, %s" % (a.L, D, a.N, a.n_mcmc, HMC_LEAPFROG, a.precision),
                "sampler": "hmc", "L": a.L, "D": D, "N": a.N, "n_mcmc": a.n_mcmc, "m2": -4.0, "lambda": 8.0,
                "ess_target": 0.5, "precision": a.precision,
                "l2": "inputs larger than L2 (fields %d MiB + normals per transition)"
                      % (a.N * D * (8 if a.precision == "fp64" else 4) >> 20)}
    return {"workload": "SMC-RW tempering step, broken-phase phi^4 L=%d (D=%d), N=%d, m2=-4, lambda=8, "
                        "%d RWM sweeps/temperature, ESS 0.5N, %s" % (a.L, D, a.N, a.n_mcmc, a.precision),
            "L": a.L, "D": D, "N": a.N, "n_mcmc": a.n_mcmc, "m2": -4.0, "lambda": 8.0, "ess_target": 0.5,
            "precision": a.precision,
            "l2": "inputs larger than L2 (fields %d MiB + proposals + normals per sweep)" % (a.N * D * 4 >> 20)}


def dist_setup(a):
    if a.gpus <= 1 and "WORLD_SIZE" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    dist.init_process_group("gloo")
    return dist.get_rank(), dist.get_world_size(), dist


def max_over_ranks(x, dist):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return None
        try:
            rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
            os.unlink(self.f.name)
        except Exception:
            return None
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        if not sm:
            return None
        mx = max(float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit())
        load = [x for x in sm if x > 0.5 * mx] or sm
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for k, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6786.6), d.get("bf16_tflops", 1897.7), d.get("bf16_tflops_sustained", 1683.6), \
            "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


def kernel_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None when the
    kernel's source changed since the counters were taken (the hash covers the source
    section that holds the kernel: from the line `section_begin` to `section_end`)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(kernel)
    if not d:
        return None
    src = os.path.join(ROOT, d["source"])
    if not os.path.exists(src):
        return None
    text = open(src, "rb").read()
    if "section_begin" in d:
        a = text.find(d["section_begin"].encode())
        b = text.find(d["section_end"].encode(), a + 1)
        if a < 0 or b < 0:
            return None
        text = text[a:b]
    if hashlib.sha256(text).hexdigest()[:16] != d["sha256_16"]:
        return None
    return d["bytes_per_launch"]


def cpu_sample(a):
    """Particles in the oracle's bounded sample (an HMC transition costs about 21 gradient
    evaluations, so its sample is smaller)."""
    return a.cpu_sample if a.sampler == "rw" else min(a.cpu_sample, 128)


def cpu_baseline(a, sample):
    """The FP64 oracle (test infrastructure, untuned) on a bounded sample of the workload:
    one temperature step from beta = 0 with `sample` particles of the same lattice."""
    import numpy as np
    from oracle.smc import SMC, SMCConfig
    cfg = SMCConfig(L=a.L, N=sample, m2=-4.0, lam=8.0, rho=0.5, n_mcmc=a.n_mcmc, seed=0,
                    normal_bits=32 if a.precision == "fp64" else 24,
                    inner="hmc" if a.sampler == "hmc" else "rw")
    smc = SMC(cfg)
    t0 = time.perf_counter()
    smc.temper_step()
    dt = time.perf_counter() - t0
    D = a.L * a.L
    try:
        import threadpoolctl
        cores = max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()) or os.cpu_count()
    except Exception:
        cores = os.cpu_count()
    del np
    return {"value": sample * D * a.n_mcmc / dt, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
            "sample": "one temperature step (ESS bisection, resampling, covariance + Cholesky of the D x D "
                      "covariance, %d %s) with N=%d of the %d particles, L=%d; %.1f s"
                      % (a.n_mcmc, "HMC transitions" if a.sampler == "hmc" else "RWM sweeps", sample, a.N, a.L, dt)}


def run_reference(a):
    rank, world, dist = dist_setup(a)
    if rank != 0:
        return 0
    res = []
    for _ in range(a.warmup):
        pass
    for _ in range(max(1, a.steps)):
        res.append(cpu_baseline(a, cpu_sample(a)))
    v = statistics.median(r["value"] for r in res)
    cb = dict(res[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "site-updates/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * cpu_sample(a) * a.L ** 2 * a.n_mcmc / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp64",
            "data": "synthetic (Philox N(0,I) initial fields)", "config": workload(a), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def time_steps(p, cfg, steps, warmup, stream, dist, local):
    """Times `steps` temperatures of a run of `cfg` after `warmup` untimed ones (CUDA events on
    the run's stream, barrier and synchronize on both sides). A run that reaches beta = 1
    is continued by a fresh replica of the same configuration. Returns the elapsed device
    milliseconds, the stage timers, the kernel launches, the last run, the sampler's state
    over the timed temperatures and the clock sampler."""
    import torch

    def fresh():
        r = p.Run(cfg)
        r.set_stage_timing(True)
        return r

    run = fresh()
    for _ in range(warmup):
        if run.temper_step() >= 1.0:
            run = fresh()
    run.stage_times(reset=True)
    l0 = run.kernel_launches()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage_acc = {}
    launches = 0
    betas, accs, esss, replicas = [], [], [], 1

    def bank(r):
        for k, (ms, n) in r.stage_times(reset=True).items():
            s = stage_acc.setdefault(k, [0.0, 0])
            s[0] += ms
            s[1] += n

    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(steps):
            b = run.temper_step()
            betas.append(b)
            if b >= 1.0:
                # the run reached beta = 1: account and continue on a fresh replica
                bank(run)
                launches += run.kernel_launches() - l0
                ev1.record(stream)
                torch.cuda.synchronize()
                partial = ev0.elapsed_time(ev1)
                o = run.observables()  # outside the timed interval
                accs.append(o["acc_rate"])
                esss.append(o["ess"])
                run = fresh()
                replicas += 1
                l0 = run.kernel_launches()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                stage_acc.setdefault("_partial_ms", [0.0, 0])[0] += partial
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed_ms = ev0.elapsed_time(ev1) + stage_acc.pop("_partial_ms", [0.0, 0])[0]
    if dist is not None:
        dist.barrier()
    launches += run.kernel_launches() - l0
    bank(run)
    if betas and betas[-1] < 1.0:
        o = run.observables()
        accs.append(o["acc_rate"])
        esss.append(o["ess"])
    finite = [x for x in accs if x == x]
    telemetry = {"temperatures_timed": steps, "replicas": replicas, "beta_after_each_step": betas,
                 "acc_rate_last_step_per_replica": accs, "ess_last_step_per_replica": esss,
                 "acc_rate_mean": sum(finite) / len(finite) if finite else float("nan")}
    return elapsed_ms, stage_acc, launches, run, telemetry, clk


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "kernels":
        return run_kernels(a)
    if a.workload == "batch":
        return run_batch(a)
    import torch
    import paper_2511_15196_gb300 as p
    rank, world, dist = dist_setup(a)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    D = a.L * a.L
    prec = PREC[a.precision]
    hmc = a.sampler == "hmc"
    if hmc and prec == 2:
        raise SystemExit("--sampler hmc runs in the fp32 or fp64 form")
    cfg = p.Config(L=a.L, N=a.N, m2=-4.0, lam=8.0, precision=prec, n_mcmc=a.n_mcmc, ess_target=0.5,
                   seed=1000 + rank, kind=p.SMC_HMC if hmc else p.SMC_RW)
    stream = torch.cuda.current_stream()

    elapsed_ms, stage_acc, launches, run, telemetry, clk = time_steps(p, cfg, a.steps, a.warmup, stream, dist,
                                                                      local)
    elapsed_ms = max_over_ranks(elapsed_ms, dist)
    units_per_step = a.N * D * a.n_mcmc
    value = world * units_per_step * a.steps / (elapsed_ms * 1e-3)
    # wall time of the sweeps (their normals, proposal and accept overlap on three streams)
    mutation_ms = stage_acc.get("mutation", [0, 0])[0] or \
        sum(stage_acc.get(k, [0, 0])[0] for k in ("normals", "propose", "accept"))

    # roofline of the dominant kernel (kernel-level timers only: the Cholesky stage is
    # many kernels on two streams, its tensor-core trailing update is timed per launch)
    hbm, bf16, bf16_s, src = peaks()
    dom = max(("chol_update", "propose", "accept", "normals"), key=lambda k: stage_acc.get(k, [0, 0])[0])
    ms_tot, n_l = stage_acc[dom]
    avg_s = ms_tot / max(n_l, 1) * 1e-3
    acc = telemetry["acc_rate_mean"] if telemetry["acc_rate_mean"] == telemetry["acc_rate_mean"] else 0.25
    extra = {}
    if dom == "chol_update":
        # exact digit emulation of the FP64 update A22 -= P P^T: 36 bf16 digit-plane products
        # (pairs k + l <= 9 of eight 7-bit digits) of the 64-wide panel per lower element;
        # the timed launches are the bulk of each panel's update (the trailing matrix
        # without the next block column, (m - 64)(m - 63)/2 lower elements)
        nb = (D + 63) // 64
        elems = sum((D - 64 * (kb + 2)) * (D - 64 * (kb + 2) + 1) // 2 for kb in range(nb - 2))
        # one Cholesky stage per factorisation attempt
        n_fact = stage_acc.get("cholesky", [0, 0])[1]
        units = 36 * 2 * 64 * elems * n_fact / max(n_l, 1)
        work = ("tensor", units, "TFLOP/s")
        extra = {"fp64_equivalent_tflops": 2 * 64 * elems * n_fact / (ms_tot * 1e-3) / 1e12,
                 "factorizations": n_fact}
    elif hmc and dom == "accept":
        # the HMC transition kernel (timed as the accept stage): FMA-unit work of the
        # leapfrog trajectory; its shared-memory traffic against the derived shared-memory
        # bandwidth (128 B per SM per cycle) is reported beside it
        work = ("alu", a.N * D * HMC_FLOP_PER_SITE, "TFLOP/s")
        smem = a.N * D * hmc_smem_bytes_per_site(prec)
        smem_peak = 152 * 2070e6 * 128 / 1e9
        extra = {"kernel_name": "hmc_kernel", "smem_bytes_per_launch": smem,
                 "smem_gbs": smem / avg_s / 1e9, "smem_peak_gbs": smem_peak,
                 "smem_frac": smem / avg_s / 1e9 / smem_peak}
    else:
        work = {
            # the mixed form's proposal runs on the tensor cores, the FP32 / FP64 forms' on the
            # SIMT FMA units
            "propose": ("tensor" if prec == 2 else "alu", a.N * D * (D + 1), "TFLOP/s"),
            "accept": ("hbm", a.N * D * ((4 + 2) if prec == 2 else (8 if prec == 0 else 4)) + a.N * D * acc *
                       (8 if prec == 0 else 4), "GB/s"),
            "normals": ("hbm", a.N * D * (2 if prec == 2 else 4 * (2 if prec == 0 else 1)), "GB/s"),
        }[dom]
    bound, units, unit = work
    if unit == "TFLOP/s" and bound == "alu":
        # derived from unit counts and the maximum SM clock (2070 MHz, 152 SMs): FP32, 128 FMA
        # lanes per SM per cycle; FP64, one warp instruction per 64 cycles on each of the four
        # sub-partitions (measured issue cost on this part), i.e. 2 lanes per SM per cycle
        achieved = units / avg_s / 1e12
        peak = 152 * 2070e6 * 2 * (128 if prec == 1 else 2) / 1e12
        peak_src = "derived %s FMA peak (152 SMs x %s lanes/cycle x 2 flop x 2070 MHz)" % (
            "FP32" if prec == 1 else "FP64", "128" if prec == 1 else "2")
    elif unit == "TFLOP/s":
        achieved = units / avg_s / 1e12
        peak = bf16_s
        peak_src = "%s bf16 sustained (kernel timed inside a long step)" % src
    else:
        achieved = units / avg_s / 1e9
        peak = hbm
        peak_src = "%s HBM copy" % src
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "peak_source": peak_src, "traffic": kernel_traffic(dom),
                "work_per_launch": units, "avg_launch_ms": avg_s * 1e3, **extra}
    stages = {k: {"ms_per_step": v[0] / a.steps, "launches": v[1]} for k, v in stage_acc.items() if v[1]}
    line = {"metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": elapsed_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": PREC_DTYPE[a.precision],
            "data": "synthetic (Philox N(0,I) initial fields, random-init sampler state)",
            "config": workload(a), "gpu_launches": launches,
            "mutation_only": {"value": world * units_per_step * a.steps / (mutation_ms * 1e-3) if mutation_ms else None,
                              "unit": "site-updates/s", "ms_per_step": mutation_ms / a.steps},
            "roofline": roofline, "stages": stages, "clocks": clk.summary(), "sampler": telemetry}
    run.close()
    if prec == 2 and not hmc and a.fp32_steps > 0:
        # the plain FP32 form (SIMT float GEMMs, float covariance and Cholesky, FP64 log Z)
        # on the same workload and seed, timed the same way: the comparator of the metric
        cfg32 = dataclasses.replace(cfg, precision=p.FP32)
        ms32, acc32, l32, r32, tel32, clk32 = time_steps(p, cfg32, a.fp32_steps, 3, stream, dist, local)
        ms32 = max_over_ranks(ms32, dist)
        mut32 = acc32.get("mutation", [0, 0])[0] or \
            sum(acc32.get(k, [0, 0])[0] for k in ("normals", "propose", "accept"))
        r32.close()
        line["fp32_comparator"] = {
            "value": world * units_per_step * a.fp32_steps / (ms32 * 1e-3), "unit": "site-updates/s",
            "steps": a.fp32_steps, "warmup": 3, "ms_per_step": ms32 / a.fp32_steps,
            "mutation_only": world * units_per_step * a.fp32_steps / (mut32 * 1e-3) if mut32 else None,
            "dtype": PREC_DTYPE["fp32"], "gpu_launches": l32, "sampler": tel32, "clocks": clk32.summary(),
            "stages": {k: {"ms_per_step": v[0] / a.fp32_steps, "launches": v[1]} for k, v in acc32.items() if v[1]},
            "speedup_of_mixed": (ms32 / a.fp32_steps) / (elapsed_ms / a.steps)}

    if not a.no_e2e:
        # the same metric through the public API with the population held in pinned host
        # memory: the same run (seed, warm-up steps) as the device-timed one, and every
        # timed step copies the population in (H2D), advances one temperature, copies the
        # new population out (D2H) and reads log Z back
        r2 = p.Run(cfg)
        for _ in range(a.warmup):
            if r2.temper_step() >= 1.0:
                r2 = p.Run(cfg)
        host = torch.empty((a.N, D), dtype=torch.float64 if prec == 0 else torch.float32).pin_memory()
        r2.copy_particles(host)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        n_done = 0
        for _ in range(a.steps):
            r2.load_particles(host)
            b = r2.temper_step()
            r2.copy_particles(host)
            lz = r2.log_evidence()
            n_done += 1
            if b >= 1.0:
                break
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
        nbytes = host.numel() * host.element_size()
        line["e2e"] = {"value": world * units_per_step * n_done / e2e_s, "unit": "site-updates/s",
                       "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 16, "steps": n_done,
                       "ms_per_step": e2e_s * 1e3 / n_done}
        del lz
        r2.close()
    if rank == 0 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, cpu_sample(a))
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
