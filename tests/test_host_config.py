"""Host-side configuration helpers of the binding (no GPU): the kappa form of App. G
mapped onto the library's action coefficients, checked with the oracle's action against
the kappa form written out bond by bond."""
import numpy as np

import paper_2511_15196_gb300 as p
from oracle import lattice


def test_kappa_config_reproduces_the_kappa_form_and_its_log_z_shift():
    L, kappa, lam = 5, 0.43, 0.8
    cfg = p.kappa_config(kappa, lam, L=L, N=8)
    assert (cfg.L, cfg.N) == (L, 8)
    phi = np.random.default_rng(17).standard_normal((8, L * L))
    f = phi.reshape(8, L, L)
    bonds = sum(((np.roll(f, -1, axis=a) - f) ** 2).sum(axis=(1, 2)) for a in (1, 2))
    s_kappa = 0.5 * kappa * bonds + (f ** 2 + lam * (f ** 2 - 1.0) ** 2).sum(axis=(1, 2))
    s_cfg = lattice.action(phi, L, cfg.m2, cfg.lam, cfg.c_kin, cfg.c_mass)
    # Z_kappa = exp(-lam V) Z_cfg, so S_kappa = S_cfg - kappa_logz_shift
    np.testing.assert_allclose(s_cfg - p.kappa_logz_shift(lam, L * L), s_kappa, rtol=1e-13)


def test_batched_workload_assignment():
    # 64 runs: L round-robin over {8, 12, 16, 24, 32}, N = {1024, 2048, 4096}[seed mod 3],
    # lambda = {4, 8, 16}[(r div 3) mod 3] so that every lambda meets every N, m2 = -4,
    # float fields with bf16 tensor-core GEMMs, seed = run index
    import itertools

    import bench
    cfgs = bench.batch_configs(p, 64, 10)
    assert len(cfgs) == 64
    assert [c.L for c in cfgs[:6]] == [8, 12, 16, 24, 32, 8]
    assert all(c.seed == r and c.N == [1024, 2048, 4096][r % 3] for r, c in enumerate(cfgs))
    assert {(c.lam, c.N) for c in cfgs} == set(itertools.product([4.0, 8.0, 16.0], [1024, 2048, 4096]))
    assert {c.L for c in cfgs} == {8, 12, 16, 24, 32}
    assert all(c.m2 == -4.0 and c.precision == p.MIXED_BF16 and c.n_mcmc == 10 for c in cfgs)
    total = sum(p.workspace_bytes(c) for c in cfgs)
    assert total < 64 * 2 ** 30
