"""The covariance-bias study script's code paths run (tiny sizes, CPU): every variant
returns a finite evidence estimate, and the exact-covariance control restores the
oracle's own covariance routines afterwards."""
import math

import study_covariance_bias as st
from oracle import covariance, tempering


def test_study_variants_run_on_a_tiny_lattice():
    before = (tempering.bisect_dbeta, covariance.sample_covariance)
    for exact in (False, True):
        lz = st.logz_seeds(2, 64, 0.5, 2, 2, exact_covariance=exact)
        assert len(lz) == 2 and all(math.isfinite(x) for x in lz)
    assert (tempering.bisect_dbeta, covariance.sample_covariance) == before
    for mode in ("split", "weighted"):
        assert math.isfinite(st.variant_logz(2, 64, 0, mode, n_mcmc=2))
    assert math.isfinite(st.replica_logz(2, 64, 0, n_mcmc=2))
