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
