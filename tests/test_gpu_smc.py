"""Whole-step and whole-run parity of the GPU SMC (through the C ABI) with the
FP64 oracle: the same Philox streams make FP64 runs agree step by step; the
float and bf16 forms and longer runs are compared statistically (32 seeds,
3 standard errors) on log Z, <|M|> and the susceptibility."""
import math

import numpy as np
import pytest

import closed_forms as cf
from oracle.smc import SMC, SMCConfig

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2511_15196_gb300 as p  # noqa: E402


def gpu_cfg(**kw):
    base = dict(L=8, N=1024, m2=-4.0, lam=8.0, n_mcmc=10, ess_target=0.5, precision=p.FP64, seed=0)
    base.update(kw)
    return p.Config(**base)


def oracle_cfg(**kw):
    base = dict(L=8, N=1024, m2=-4.0, lam=8.0, n_mcmc=10, rho=0.5, seed=0)
    base.update(kw)
    return SMCConfig(**base)


@pytest.mark.parametrize("L,N", [(8, 1024), (1, 64), (2, 256), (12, 300), (16, 512), (20, 300)])
def test_fp64_steps_match_oracle(L, N):
    # L = 16, 20 (D = 256, 400): the factorisation uses the tensor-core trailing update and
    # the look-ahead schedule (D = 400 with a ragged last block)
    run = p.Run(gpu_cfg(L=L, N=N, n_mcmc=4, seed=3))
    ref = SMC(oracle_cfg(L=L, N=N, n_mcmc=4, seed=3))
    for _ in range(3):
        if ref.done:
            break
        beta = run.temper_step()
        rec = ref.temper_step()
        assert beta == pytest.approx(rec["beta"], rel=1e-10, abs=1e-13)
        lz, _ = run.log_evidence()
        assert lz == pytest.approx(rec["logz"], rel=1e-10, abs=1e-9)
        phi = run.particles().cpu().numpy()
        assert np.abs(phi - ref.phi).max() < 1e-8
    obs = run.observables()
    ro = ref.result()
    assert obs["mean_absM"] == pytest.approx(ro["mean_absM"], rel=1e-8, abs=1e-12)
    run.close()


@pytest.mark.parametrize("precision", [p.FP64, p.FP32], ids=["fp64", "fp32"])
def test_z2_flip_matches_oracle(precision):
    # the same particles flip on both sides (one Philox bit per particle and temperature)
    L, N = 8, 512
    run = p.Run(gpu_cfg(L=L, N=N, n_mcmc=3, seed=4, precision=precision, flags=p.FLAG_Z2_FLIP))
    ref = SMC(oracle_cfg(L=L, N=N, n_mcmc=3, seed=4, z2_flip=True,
                         normal_bits=32 if precision == p.FP64 else 24))
    for _ in range(2):
        run.temper_step()
        ref.temper_step()
        phi = run.particles().cpu().numpy().astype(np.float64)
        if precision == p.FP64:
            assert np.abs(phi - ref.phi).max() < 1e-8
        else:
            # float fields: the signs of the row means agree wherever the row mean is clear
            Mg, Mo = phi.mean(axis=1), ref.phi.mean(axis=1)
            clear = np.abs(Mo) > 1e-3
            assert (np.sign(Mg[clear]) == np.sign(Mo[clear])).mean() > 0.99
    run.close()


def test_z2_flip_balances_the_modes_mixed():
    # broken phase on the pipelined mixed path (L % 4 == 0)
    run = p.Run(gpu_cfg(L=16, N=2048, n_mcmc=4, seed=6, precision=p.MIXED_BF16, flags=p.FLAG_Z2_FLIP))
    for _ in range(4):
        run.temper_step()
    M = run.particles().cpu().numpy().mean(axis=1)
    assert abs((M > 0).mean() - 0.5) < 4 * math.sqrt(0.25 / 2048)
    run.close()


@pytest.mark.parametrize("L,N", [(4, 512), (8, 1024), (2, 300)])
def test_irmh_fp64_steps_match_oracle(L, N):
    # SMC-IRMH: the same proposals (mean + L z), Hastings terms and decisions as the oracle
    run = p.Run(gpu_cfg(L=L, N=N, n_mcmc=3, seed=9, kind=p.SMC_IRMH))
    ref = SMC(oracle_cfg(L=L, N=N, n_mcmc=3, seed=9, inner="irmh"))
    for _ in range(3):
        if ref.done:
            break
        beta = run.temper_step()
        rec = ref.temper_step()
        assert beta == pytest.approx(rec["beta"], rel=1e-10, abs=1e-13)
        lz, _ = run.log_evidence()
        assert lz == pytest.approx(rec["logz"], rel=1e-10, abs=1e-9)
        phi = run.particles().cpu().numpy()
        assert np.abs(phi - ref.phi).max() < 1e-8
        assert run.observables()["acc_rate"] == pytest.approx(rec["acc_rate"], abs=1e-12)
    run.close()


def test_irmh_configuration_checks():
    with pytest.raises(RuntimeError):
        p.Run(gpu_cfg(L=8, N=64, kind=p.SMC_IRMH, precision=p.MIXED_BF16))
    with pytest.raises(RuntimeError):
        p.Run(gpu_cfg(L=40, N=64, kind=p.SMC_IRMH))


@pytest.mark.parametrize("L,N,keep", [(4, 512, False), (8, 1024, False), (3, 300, True), (16, 256, False),
                                      (20, 128, False), (24, 128, False), (40, 64, False), (46, 64, True)])
def test_hmc_fp64_steps_match_oracle(L, N, keep):
    # SMC-HMC: the same momenta, leapfrog trajectories (20 steps, covariance-diagonal inverse
    # mass), energies and decisions as the oracle; the sizes cover every thread layout
    # (32 to 512 threads per particle) and a last CTA with idle particle slots
    run = p.Run(gpu_cfg(L=L, N=N, n_mcmc=2, seed=5, kind=p.SMC_HMC, keep_reference=keep))
    ref = SMC(oracle_cfg(L=L, N=N, n_mcmc=2, seed=5, inner="hmc", keep_reference=keep))
    for _ in range(3):
        if ref.done:
            break
        beta = run.temper_step()
        rec = ref.temper_step()
        assert beta == pytest.approx(rec["beta"], rel=1e-10, abs=1e-13)
        lz, _ = run.log_evidence()
        assert lz == pytest.approx(rec["logz"], rel=1e-10, abs=1e-9)
        phi = run.particles().cpu().numpy()
        assert np.abs(phi - ref.phi).max() < 1e-8
        assert run.observables()["acc_rate"] == pytest.approx(rec["acc_rate"], abs=1e-12)
    run.close()


@pytest.mark.parametrize("L,N", [(8, 1024), (10, 250), (12, 256), (18, 300), (24, 256), (40, 128), (64, 64)],
                         ids=["D64", "D100_ragged_cta", "D144", "D324", "D576", "D1600", "D4096"])
def test_hmc_fp32_step_close_to_oracle(L, N):
    # the float form of the same transition: float leapfrog trajectories, energies summed in
    # double. Against the double oracle on the same streams, particles whose decisions and
    # ancestors agree match to float rounding; a decision at the threshold may flip
    run = p.Run(gpu_cfg(L=L, N=N, n_mcmc=2, seed=5, kind=p.SMC_HMC, precision=p.FP32))
    ref = SMC(oracle_cfg(L=L, N=N, n_mcmc=2, seed=5, inner="hmc"))
    beta = run.temper_step()
    rec = ref.temper_step()
    # beta comes from the float-rounded initial fields' log-weights (a relative 1.2e-5 off
    # the double oracle's at D = 4096)
    assert beta == pytest.approx(rec["beta"], rel=1e-4)
    phi = run.particles().cpu().numpy().astype(np.float64)
    close = np.abs(phi - ref.phi).max(axis=1) < 1e-3
    assert (~close).sum() <= max(1, 0.01 * N), (~close).sum()
    assert abs(run.observables()["acc_rate"] - rec["acc_rate"]) <= max(0.01, 1.0 / N)
    run.close()


@pytest.mark.slow
@pytest.mark.parametrize("precision", [p.FP64, p.FP32], ids=["fp64", "fp32"])
def test_broken_phase_hmc_16_seeds(precision):
    # L = 8, N = 1024, m2 = -4, lambda = 8: SMC-HMC runs to beta = 1 agree with the oracle's
    # in log Z, <|M|> and chi within three standard errors of the seed-to-seed spread
    g = _gpu_runs(16, kind=p.SMC_HMC, n_mcmc=3, precision=precision)
    o = _oracle_runs(16, inner="hmc", n_mcmc=3)
    _within_3se(g, o)
    if precision == p.FP64:
        assert np.abs(g[:, 0] - o[:, 0]).max() < 1e-6


def test_hmc_configuration_checks():
    with pytest.raises(RuntimeError):
        p.Run(gpu_cfg(L=8, N=64, kind=p.SMC_HMC, precision=p.MIXED_BF16))
    with pytest.raises(RuntimeError):
        p.Run(gpu_cfg(L=72, N=64, kind=p.SMC_HMC))


def test_flags_are_checked():
    with pytest.raises(RuntimeError):
        p.Run(gpu_cfg(L=4, N=64, flags=2))
    with pytest.raises(RuntimeError):
        p.Run(gpu_cfg(L=4, N=64, kind=p.NS_SLICE, ns_n_delete=8, flags=p.FLAG_Z2_FLIP))


@pytest.mark.parametrize("precision", [p.FP64, p.FP32, p.MIXED_BF16], ids=["fp64", "fp32", "bf16"])
def test_observables_match_oracle_summary(precision):
    # a12: every population moment of M, the susceptibility and the mode balance of the
    # device's smc_observables against the oracle's summary of the same device fields (the
    # fields themselves are compared elsewhere; this pins the reduction and its formulas)
    from oracle import observables as oobs
    L, N = 8, 700
    run = p.Run(gpu_cfg(L=L, N=N, n_mcmc=3, seed=8, precision=precision))
    for _ in range(3):
        run.temper_step()
    o = run.observables()
    phi = run.particles().cpu().numpy().astype(np.float64)
    ref = oobs.summary(phi)
    for k in ("mean_M", "mean_absM", "mean_M2", "chi"):
        assert o[k] == pytest.approx(ref[k], rel=1e-10, abs=1e-13), k
    assert o["mode_balance"] == pytest.approx(ref["mode_balance"], rel=1e-12)
    assert 0.0 <= o["acc_rate"] <= 1.0 and o["n_steps"] == 3
    run.close()


def test_run_to_completion_and_done_status():
    run = p.Run(gpu_cfg(L=4, N=512, seed=1))
    obs = run.run()
    assert obs["beta"] == 1.0 and obs["n_steps"] >= 1
    with pytest.raises(p.Phi4Error) as e:
        run.temper_step()
    assert e.value.status == p.PHI4_ERR_DONE
    with pytest.raises(p.Phi4Error) as e:
        run.replace_step()
    assert e.value.status == p.PHI4_ERR_ARG
    run.close()


def test_nonfinite_particles_reported():
    run = p.Run(gpu_cfg(L=4, N=128))
    phi = run.particles()
    phi[5, 3] = float("nan")
    run.load_particles(phi)
    with pytest.raises(p.Phi4Error) as e:
        run.temper_step()
    assert e.value.status == p.PHI4_ERR_NONFINITE
    run.close()


def test_particles_round_trip():
    run = p.Run(gpu_cfg(L=8, N=256, precision=p.FP32))
    phi = run.particles()
    assert phi.dtype == torch.float32 and phi.shape == (256, 64)
    run.load_particles(phi * 0.5)
    assert torch.equal(run.particles(), phi * 0.5)
    run.close()


def _stats(vals):
    v = np.asarray(vals, dtype=np.float64)
    return v.mean(), v.std(ddof=1) / math.sqrt(len(v))


def _gpu_runs(n_seeds, **kw):
    out = []
    for s in range(n_seeds):
        run = p.Run(gpu_cfg(seed=s, **kw))
        o = run.run()
        out.append((o["logz"], o["mean_absM"], o["chi"]))
        run.close()
    return np.array(out)


def _oracle_runs(n_seeds, **kw):
    out = []
    for s in range(n_seeds):
        r = SMC(oracle_cfg(seed=s, **kw)).run()
        out.append((r["logz"], r["mean_absM"], r["chi"]))
    return np.array(out)


def _within_3se(a, b):
    for k in range(a.shape[1]):
        ma, sa = _stats(a[:, k])
        mb, sb = _stats(b[:, k])
        se = math.sqrt(sa * sa + sb * sb)
        assert abs(ma - mb) <= 3.0 * se + 1e-12, (k, ma, mb, se)


@pytest.mark.slow
def test_broken_phase_fp64_32_seeds():
    # L = 8 (D = 64), N = 1024, m2 = -4, lambda = 8, ESS 0.5 N, 10 sweeps per temperature
    g = _gpu_runs(32)
    o = _oracle_runs(32)
    _within_3se(g, o)
    # same streams in double precision: seed-by-seed agreement as well
    assert np.abs(g[:, 0] - o[:, 0]).max() < 1e-6


_ORACLE_RUNS = {}


def _oracle_runs_cached(n_seeds, **kw):
    key = (n_seeds, tuple(sorted(kw.items())))
    if key not in _ORACLE_RUNS:
        _ORACLE_RUNS[key] = _oracle_runs(n_seeds, **kw)
    return _ORACLE_RUNS[key]


@pytest.mark.slow
@pytest.mark.parametrize("precision", [p.FP32, p.MIXED_BF16], ids=["fp32", "bf16"])
def test_broken_phase_single_forms_32_seeds(precision):
    # the float and mixed forms against the oracle with float-precision normals (the same
    # 32 oracle runs serve both forms)
    g = _gpu_runs(32, precision=precision)
    o = _oracle_runs_cached(32, normal_bits=24)
    _within_3se(g, o)


def _logz_plus_half_var(lz):
    # log Zhat is biased low by about Var/2: mean + var/2 estimates log Z; its error combines
    # the mean's standard error and the spread of the variance estimate
    lz = np.asarray(lz, dtype=np.float64)
    n, var = len(lz), lz.var(ddof=1)
    return lz.mean() + 0.5 * var, math.sqrt(var / n + (0.5 * var * math.sqrt(2.0 / (n - 1))) ** 2)


@pytest.mark.parametrize("L,N,keep", [(8, 512, False), (16, 1024, False), (6, 300, True)])
def test_free_kernel_covariance_fp64_steps_match_oracle(L, N, keep):
    # PHI4_FLAG_FREE_KERNEL_COV: the proposal's factor comes from the exact covariance of the
    # tempered Gaussian part (built on the device from the Fourier spectrum; the oracle
    # inverts the precision matrix assembled site by site) and the run follows the oracle
    run = p.Run(gpu_cfg(L=L, N=N, n_mcmc=3, seed=6, m2=1.0, lam=0.0, keep_reference=keep,
                        flags=p.FLAG_FREE_KERNEL_COV))
    ref = SMC(oracle_cfg(L=L, N=N, n_mcmc=3, seed=6, m2=1.0, lam=0.0, keep_reference=keep,
                         kernel_cov="gaussian_part"))
    for _ in range(3):
        beta = run.temper_step()
        rec = ref.temper_step()
        assert beta == pytest.approx(rec["beta"], rel=1e-10, abs=1e-13)
        assert np.abs(run.particles().cpu().numpy() - ref.phi).max() < 1e-8
        assert run.log_evidence()[0] == pytest.approx(rec["logz"], rel=1e-10, abs=1e-9)
    run.close()


@pytest.mark.slow
@pytest.mark.parametrize("precision", [p.FP64, p.FP32, p.MIXED_BF16], ids=["fp64", "fp32", "bf16"])
def test_free_field_closed_form_each_form_with_the_free_kernel_covariance(precision):
    # the precision check against the closed form, in a setting where the sampler mixes:
    # the 8 x 8 free field (m2 = 1), N = 1024, ESS 0.9 N, 20 sweeps, the exact Gaussian-part
    # kernel covariance, 32 seeds; each arithmetic form's mean log Zhat + Var/2 lands on the
    # closed form -11.6228852573 within four of its errors
    lz = _gpu_runs(32, L=8, N=1024, m2=1.0, lam=0.0, ess_target=0.9, n_mcmc=20, precision=precision,
                   flags=p.FLAG_FREE_KERNEL_COV)[:, 0]
    est, err = _logz_plus_half_var(lz)
    exact = cf.free_field_logz(8, 1.0)
    print("free field L=8, %s: log Zhat mean %.4f sd %.4f; mean + var/2 - exact = %+.4f (err %.4f)"
          % (precision, lz.mean(), lz.std(ddof=1), est - exact, err))
    assert abs(est - exact) < 4.0 * err + 0.01


@pytest.mark.slow
def test_free_field_closed_form_mixed_form_at_the_32x32_size():
    # the precision-check lattice itself (32 x 32, m2 = 1, N = 4096) in a setting where the
    # sampler mixes: ESS 0.9 N, 640 sweeps per temperature, the exact Gaussian kernel
    # covariance; the bf16-GEMM form's mean log Zhat + Var/2 over 32 seeds lands on the closed
    # form -185.9853908122 within four of its errors (about 3.5 s per run)
    lz = _gpu_runs(32, L=32, N=4096, m2=1.0, lam=0.0, ess_target=0.9, n_mcmc=640, precision=p.MIXED_BF16,
                   flags=p.FLAG_FREE_KERNEL_COV)[:, 0]
    est, err = _logz_plus_half_var(lz)
    exact = cf.free_field_logz(32, 1.0)
    print("free field L=32, mixed: log Zhat mean %.4f sd %.4f; mean + var/2 - exact = %+.4f (err %.4f)"
          % (lz.mean(), lz.std(ddof=1), est - exact, err))
    assert abs(est - exact) < 4.0 * err + 0.01


@pytest.mark.slow
def test_free_field_precision_forms_32_seeds():
    # the precision-check workload as configured: free field (lambda = 0, m2 = 1), L = 32
    # (D = 1024), N = 4096, ESS 0.5 N, 10 sweeps, the population's covariance. The three
    # arithmetic forms run on the same random streams; the float and bf16 forms' log Z, <|M|>
    # and chi agree with the FP64 form (step-matched to the oracle elsewhere) within three
    # standard errors over 32 seeds. Each form's log Zhat - log Z (closed form
    # -185.9853908122) is printed: with this sampler and 10 sweeps it is hundreds of nats
    # above the closed form for every form alike, the bias of the population-estimated
    # kernel covariance, not an arithmetic error (the free-kernel-covariance test above is
    # the closed-form comparison where the sampler mixes).
    res = {}
    exact = cf.free_field_logz(32, 1.0)
    for prec in (p.FP64, p.FP32, p.MIXED_BF16):
        res[prec] = _gpu_runs(32, L=32, N=4096, m2=1.0, lam=0.0, precision=prec)
        m, se = _stats(res[prec][:, 0])
        print("L=32 free field, precision %d: log Zhat - log Z = %+.3f (SE %.3f); minus the FP64 form's: %+.3f"
              % (prec, m - exact, se, m - res[p.FP64][:, 0].mean()))
        assert np.isfinite(res[prec]).all()
    for prec in (p.FP32, p.MIXED_BF16):
        _within_3se(res[prec], res[p.FP64])


@pytest.mark.parametrize("L,N", [(16, 2048), (20, 300), (10, 2048)],
                         ids=["pipelined_sweeps", "pipelined_ragged", "sequential_sweeps"])
def test_mixed_runs_are_deterministic(L, N):
    # L % 4 == 0: the sweeps' normals, proposal GEMM and accept overlap on three streams
    # with a ring of normals buffers and double-buffered increments; a buffer reused before its reader
    # finished would make two identical runs differ. L = 20, N = 300: D = 400 and an odd
    # number of 128-row tiles (a ragged last tile in the GEMM and the accept). L = 10
    # takes the sequential path.
    cfg = gpu_cfg(L=L, N=N, n_mcmc=6, precision=p.MIXED_BF16, seed=5)
    runs = [p.Run(cfg) for _ in range(2)]
    for _ in range(3):
        b = [r.temper_step() for r in runs]
        assert b[0] == b[1]
    assert torch.equal(runs[0].particles(), runs[1].particles())
    assert runs[0].log_evidence()[0] == runs[1].log_evidence()[0]
    o = [r.observables() for r in runs]
    assert o[0]["acc_rate"] == o[1]["acc_rate"] and 0.0 < o[0]["acc_rate"] < 1.0
    for r in runs:
        r.close()


@pytest.mark.parametrize("rho", [0.9, 0.99])
def test_paper_mode_fp64_steps_match_oracle(rho):
    # the paper's own setting step by step: Eq. (1) with factors 1/2 (c_kin = c_mass = 1/2),
    # m^2 = -4, lambda = 1, the reference kept at beta = 1 (target exp(-U_0 - S)), L = 10,
    # target ESS 0.9 and 0.99 (App. E), FP64 on the same streams as the oracle
    kw = dict(L=10, N=1000, m2=-4.0, lam=1.0, c_kin=0.5, c_mass=0.5, keep_reference=True, n_mcmc=5, seed=12)
    run = p.Run(gpu_cfg(ess_target=rho, **kw))
    ref = SMC(oracle_cfg(rho=rho, **kw))
    for _ in range(4):
        beta = run.temper_step()
        rec = ref.temper_step()
        assert beta == pytest.approx(rec["beta"], rel=1e-10, abs=1e-13)
        assert run.log_evidence()[0] == pytest.approx(rec["logz"], rel=1e-10, abs=1e-9)
        assert np.abs(run.particles().cpu().numpy() - ref.phi).max() < 1e-8
        assert run.observables()["ess"] == pytest.approx(rec["ess"], rel=1e-10)
    run.close()


def test_paper_mode_logz_L10():
    # the paper's setting (Sec. 3, App. A): L = 10, Eq. (1) with factors 1/2, m^2 = -4,
    # lambda = 1, target exp(-U_0 - S), N = 5000, n_MCMC = 3 V, ESS target 0.9. The
    # library's log Z is log E_N(0,I)[exp(-S_E)] (about -36.65 here); the paper prints that
    # value minus (V/4) log(pi) (checked at L = 10, 15, 18): Tables 1 and 3 give -65.26
    # (SMC-RW), -65.20 / -65.4 (NS), -65.64 / -65.7 (SMC-HMC). Loose window +-0.5 around
    # -65.4 (the paper's runs differ in seeds, float32 arithmetic and inner kernels).
    from paper_2511_15196_gb300 import ess_sweep
    row = ess_sweep.sweep([0.9], seeds=2)[0]
    assert -65.9 < row["logz_paper_convention"] < -64.9, row
    assert -37.2 < row["logz_mean"] < -36.1, row
    assert row["logz_sd"] < 0.5, row
    assert 0.5 < row["mode_balance"] < 2.0, row


@pytest.mark.parametrize("precision,kind", [(p.FP64, p.SMC_RW), (p.MIXED_BF16, p.SMC_RW), (p.FP32, p.SMC_HMC)],
                         ids=["fp64_rw", "bf16_rw", "fp32_hmc"])
def test_checkpoint_resume_is_bit_identical(precision, kind):
    # save after two temperatures, continue the original for two more; a fresh run of the
    # same configuration restored from the saved state follows it bit for bit
    cfg = gpu_cfg(L=16, N=512, n_mcmc=3, seed=21, precision=precision, kind=kind)
    a = p.Run(cfg)
    for _ in range(2):
        a.temper_step()
    state = a.save_state()
    ba = [a.temper_step() for _ in range(2)]
    b = p.Run(cfg)
    b.restore_state(state)
    bb = [b.temper_step() for _ in range(2)]
    assert ba == bb
    assert torch.equal(a.particles(), b.particles())
    assert a.log_evidence()[0] == b.log_evidence()[0]
    oa, ob = a.observables(), b.observables()
    assert oa["n_steps"] == ob["n_steps"] == 4 and oa["acc_rate"] == ob["acc_rate"]
    # another configuration is refused
    c = p.Run(gpu_cfg(L=16, N=512, n_mcmc=3, seed=22, precision=precision, kind=kind))
    with pytest.raises(p.Phi4Error) as e:
        c.restore_state(state)
    assert e.value.status == p.PHI4_ERR_ARG
    for r in (a, b, c):
        r.close()
