"""Failure detection on the GPU without a fault: a bounded device wait that gives up.

The library's software waits (the bisection's grid barrier, the flags between the
diagonal-block CTA and the CTAs of its streamed inverse, the hand-offs between the
diagonal block's warps) give up after a limit of SM clock cycles. With the limit
lowered to 1000 cycles the streamed inverse's first wait (for the first eight
columns of a 64 x 64 block, tens of thousands of cycles of FP64 work) runs out: its
kernel sets the timeout bit of the run's status word and returns, and
smc_temper_step returns PHI4_ERR_TIMEOUT. Nothing hangs, and the context stays
usable: with the default limit restored, a new run matches the oracle step for step.
The FP64 form with the SIMT trailing update is used so that no TMA copy or
tensor-core pipeline is involved (their waits keep the default limit).
"""
import numpy as np
import pytest

from oracle.smc import SMC, SMCConfig

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2511_15196_gb300 as p  # noqa: E402


def test_a_wait_that_runs_out_returns_timeout_and_the_context_survives():
    L, N = 16, 1024
    cfg = p.Config(L=L, N=N, m2=-4.0, lam=8.0, precision=p.FP64, chol_mode=1, n_mcmc=2, seed=5)
    p.set_spin_limit(1000)
    try:
        run = p.Run(cfg)
        with pytest.raises(p.Phi4Error) as err:
            run.temper_step()
        assert err.value.status == p.PHI4_ERR_TIMEOUT
        assert "wait gave up" in str(err.value)
        run.close()
    finally:
        p.set_spin_limit(0)
    torch.cuda.synchronize()
    run = p.Run(cfg)
    ref = SMC(SMCConfig(L=L, N=N, m2=-4.0, lam=8.0, n_mcmc=2, rho=0.5, seed=5))
    for _ in range(2):
        beta = run.temper_step()
        rec = ref.temper_step()
        assert beta == pytest.approx(rec["beta"], rel=1e-10, abs=1e-13)
        assert np.abs(run.particles().cpu().numpy() - ref.phi).max() < 1e-8
    run.close()


def test_spin_limit_default_restores():
    # a non-positive limit restores the default, under which a whole run finishes
    p.set_spin_limit(-1)
    run = p.Run(p.Config(L=8, N=256, precision=p.FP64, n_mcmc=2, seed=2))
    beta = 0.0
    for _ in range(200):
        beta = run.temper_step()
        if beta >= 1.0:
            break
    assert beta == 1.0
    run.close()
