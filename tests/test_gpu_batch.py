"""The batched form (smc_init_batch / smc_temper_step_batch): heterogeneous runs
advanced together must follow the same trajectories as the same runs advanced
one by one (the kernels are the same; only the bisection's reduction order differs,
so results agree to rounding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2511_15196_gb300 as p  # noqa: E402


def member_cfgs():
    shapes = [(4, 256, 4.0, p.FP64), (8, 512, 8.0, p.FP32), (12, 1024, 16.0, p.MIXED_BF16), (6, 300, 8.0, p.FP64),
              (8, 1024, 4.0, p.MIXED_BF16), (10, 257, 16.0, p.FP32)]
    return [p.Config(L=L, N=N, m2=-4.0, lam=lam, precision=prec, n_mcmc=6, seed=100 + r)
            for r, (L, N, lam, prec) in enumerate(shapes)]


def test_batch_matches_individual_runs():
    cfgs = member_cfgs()
    batch = p.Batch(cfgs)
    singles = [p.Run(c) for c in cfgs]
    steps = 0
    while True:
        n_active = batch.temper_step()
        steps += 1
        for c, m, s in zip(cfgs, batch.members, singles):
            if s.cfg and not getattr(s, "_done", False):
                b = s.temper_step()
                s._done = b >= 1.0
                lz_b, _ = m.log_evidence()
                lz_s, _ = s.log_evidence()
                assert lz_b == pytest.approx(lz_s, rel=1e-9, abs=1e-9)
        if n_active == 0 or steps > 400:
            break
    assert n_active == 0
    for c, m, s in zip(cfgs, batch.members, singles):
        ob, os_ = m.observables(), s.observables()
        assert ob["beta"] == 1.0 and os_["beta"] == 1.0
        assert ob["n_steps"] == os_["n_steps"]
        assert ob["mean_absM"] == pytest.approx(os_["mean_absM"], rel=1e-6, abs=1e-9)
        pb, ps_ = m.particles().cpu().numpy(), s.particles().cpu().numpy()
        assert np.abs(pb - ps_).max() < 1e-4
    with pytest.raises(p.Phi4Error) as e:
        batch.temper_step()
    assert e.value.status == p.PHI4_ERR_DONE
    # members belong to the batch
    assert p.lib().smc_free(batch.members[0].handle) == p.PHI4_ERR_ARG
    batch.close()
    for s in singles:
        s.close()


def test_batch_rejects_large_members():
    with pytest.raises(p.Phi4Error) as e:
        p.Batch([p.Config(L=4, N=8192)])
    assert e.value.status == p.PHI4_ERR_ARG
