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


def test_batch_fp64_members_match_oracle():
    # FP64 members of a batch follow the oracle step by step: the batched bisection,
    # reweighting, resampling and gather (one launch each over all members) and the
    # members' own refits and sweeps
    from oracle.smc import SMC, SMCConfig
    shapes = [(4, 256, 4.0), (6, 300, 8.0), (8, 512, 16.0), (3, 130, 8.0)]
    cfgs = [p.Config(L=L, N=N, m2=-4.0, lam=lam, precision=p.FP64, n_mcmc=3, seed=40 + r)
            for r, (L, N, lam) in enumerate(shapes)]
    refs = [SMC(SMCConfig(L=L, N=N, m2=-4.0, lam=lam, n_mcmc=3, rho=0.5, seed=40 + r))
            for r, (L, N, lam) in enumerate(shapes)]
    batch = p.Batch(cfgs)
    for _ in range(3):
        batch.temper_step()
        for m, ref in zip(batch.members, refs):
            if ref.done:
                continue
            rec = ref.temper_step()
            assert m.observables()["beta"] == pytest.approx(rec["beta"], rel=1e-10, abs=1e-13)
            assert m.log_evidence()[0] == pytest.approx(rec["logz"], rel=1e-10, abs=1e-9)
            assert np.abs(m.particles().cpu().numpy() - ref.phi).max() < 1e-8
    batch.close()


def test_batch_graph_sweeps_and_tuning_cache(tmp_path, monkeypatch):
    # an all-mixed batch takes the captured-graph sweeps (normals, grouped tcgen05 GEMM and
    # fused accept over all members per sweep); its launch shapes are measured at the first
    # temperature and written to the JSON cache, which a second batch of the same members
    # reads back; both batches follow the same trajectories (no shape changes a result)
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("PHI4_TUNE_CACHE", str(cache))
    monkeypatch.delenv("PHI4_TUNE", raising=False)
    shapes = [(8, 1024), (12, 2048), (16, 4096), (24, 1024), (32, 2048), (8, 300)]
    cfgs = [p.Config(L=L, N=N, m2=-4.0, lam=8.0, precision=p.MIXED_BF16, n_mcmc=5, seed=70 + r)
            for r, (L, N) in enumerate(shapes)]
    a = p.Batch(cfgs)
    assert a.tuning() == {}
    for _ in range(3):
        a.temper_step()
    ta = a.tuning()
    assert ta["graph"] is True and ta["gemm_ctas_source"] == "measured" and cache.exists()
    b = p.Batch(cfgs)
    for _ in range(3):
        b.temper_step()
    tb = b.tuning()
    assert tb["gemm_ctas_source"] == "cache" and tb["gemm_ctas"] == ta["gemm_ctas"]
    for ma, mb in zip(a.members, b.members):
        assert torch.equal(ma.particles(), mb.particles())
        assert ma.log_evidence()[0] == mb.log_evidence()[0]
        o = ma.observables()
        assert o["n_steps"] == 3 and 0.0 < o["acc_rate"] < 1.0
    # the members agree with the same runs advanced alone (the bisection sums in another
    # order, so to rounding)
    singles = [p.Run(c) for c in cfgs]
    for s, m in zip(singles, a.members):
        for _ in range(3):
            s.temper_step()
        assert m.log_evidence()[0] == pytest.approx(s.log_evidence()[0], rel=1e-9, abs=1e-9)
        assert np.abs(m.particles().cpu().numpy() - s.particles().cpu().numpy()).max() < 1e-4
        s.close()
    a.close()
    b.close()


def test_batch_mixed_members_with_and_without_the_batched_sweeps():
    # mixed-form members with L % 4 != 0 (10 x 10, 6 x 6) take their own streams' sweeps while
    # the L % 4 == 0 ones take the batched graph sweeps; a single member and one particle
    # block short of full (N = 1001) are covered; every member follows its single run
    shapes = [(10, 600), (8, 1001), (6, 256), (16, 2048)]
    cfgs = [p.Config(L=L, N=N, m2=-4.0, lam=8.0, precision=p.MIXED_BF16, n_mcmc=4, seed=90 + r)
            for r, (L, N) in enumerate(shapes)]
    for group in (cfgs, cfgs[1:2]):
        batch = p.Batch(group)
        singles = [p.Run(c) for c in group]
        for _ in range(3):
            batch.temper_step()
            for s in singles:
                s.temper_step()
        for m, s in zip(batch.members, singles):
            assert m.log_evidence()[0] == pytest.approx(s.log_evidence()[0], rel=1e-9, abs=1e-9)
            assert np.abs(m.particles().cpu().numpy() - s.particles().cpu().numpy()).max() < 1e-4
            assert m.observables()["n_steps"] == 3
            s.close()
        batch.close()
