"""FP64 CPU oracle for the particle Monte Carlo samplers of arXiv 2511.15196.

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it. The product
(the CUDA library and its Python binding) never imports, links or calls it, and
it shares no code, constants module or helper with the CUDA path.

It is a plain, slow, obviously correct restatement of the method, in float64:

* ``philox``      counter-based Philox4x32-10 generator (Salmon et al., SC'11) and
                  the Box-Muller / uniform conversions of the shared counter layout;
* ``lattice``     the lattice phi^4 action of Eq. (1) (coefficient reading below),
                  the tempering log-weight and the magnetisation (Sec. 2);
* ``tempering``   adaptive tempering: ESS, bisection for the next beta, reweighting
                  and the running log Z (Sec. 2 (i), App. A);
* ``resample``    systematic resampling in exact fixed point (the paper names no
                  scheme; the reading is stated in the module);
* ``covariance``  particle covariance and its Cholesky factor (App. A);
* ``mutation``    covariance-preconditioned random-walk Metropolis (App. A);
* ``irmh``        independent Metropolis-Hastings sweep from the population's Gaussian
                  (Sec. 2 sampler (ii));
* ``hmc``         Hamiltonian Monte Carlo transition, 20 leapfrog steps with a
                  diagonal mass matrix (Sec. 2 sampler (iii), App. A);
* ``smc``         the adaptive tempered SMC driver (Sec. 2 (i), App. A);
* ``ns``          nested sampling with slice-sampling rejuvenation (Sec. 2 (iv), App. A);
* ``observables`` magnetisation moments, susceptibility, mode balance (Sec. 2, App. F).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, brute force or published values. Functions without such a pin say
"parity unpinned" in their docstring.
"""
