"""Pins for ESS, the bisection for the next temperature, reweighting and the
compensated running log Z."""
import math

import numpy as np
import pytest
from scipy import optimize

import inputs
from oracle import tempering


def test_ess_bounds_and_monotone():
    ell = inputs.log_weights(500, seed=1, spread=3.0)
    assert tempering.ess(ell, 0.0) == pytest.approx(500.0, rel=1e-14)
    grid = np.linspace(0.0, 2.0, 201)
    e = np.array([tempering.ess(ell, d) for d in grid])
    assert (e <= 500.0 * (1 + 1e-12)).all() and (e >= 1.0 - 1e-12).all()
    # d/d(dbeta) log ESS = 2 (E_t[ell] - E_2t[ell]) <= 0: non-increasing
    assert (np.diff(e) <= 1e-9 * e[:-1]).all()


def test_ess_equal_weights_is_n_and_single_spike_is_one():
    assert tempering.ess(np.full(64, -3.0), 0.7) == pytest.approx(64.0, rel=1e-14)
    ell = np.full(64, 0.0)
    ell[5] = 1e6
    assert tempering.ess(ell, 1.0) == pytest.approx(1.0, rel=1e-12)


def test_bisection_matches_independent_root_finder():
    for seed in range(5):
        ell = inputs.log_weights(300, seed=seed, spread=20.0)
        beta, rho = 0.2, 0.5
        d, used = tempering.bisect_dbeta(ell, beta, rho, iters=64)
        f = lambda x: tempering.ess(ell, x) - rho * len(ell)
        root = optimize.brentq(f, 0.0, 1.0 - beta, xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
        assert d == pytest.approx(root, rel=1e-12)
        assert tempering.ess(ell, d) >= rho * len(ell)
        assert used <= 64


def test_bisection_steps_to_one_when_possible():
    ell = inputs.log_weights(100, seed=3, spread=1e-3)
    d, used = tempering.bisect_dbeta(ell, 0.75, 0.5)
    assert d == 0.25 and used == 0


def test_bisection_brute_force_grid_tiny():
    ell = np.array([-3.0, 0.0, 1.0, 2.5])
    d, _ = tempering.bisect_dbeta(ell, 0.0, 0.6)
    grid = np.linspace(0, 1, 100001)
    ok = np.array([tempering.ess(ell, x) >= 0.6 * 4 for x in grid])
    last_ok = grid[ok].max()
    assert abs(d - last_ok) <= grid[1]


def test_reweight_closed_forms():
    w, inc = tempering.reweight(np.full(10, -7.5), 0.3)
    assert inc == pytest.approx(0.3 * -7.5, rel=1e-15)
    assert (w == 1.0).all()
    a, b = -2.0, 5.0
    w, inc = tempering.reweight(np.array([a, b]), 0.4)
    assert inc == pytest.approx(math.log((math.exp(0.4 * a) + math.exp(0.4 * b)) / 2), rel=1e-14)
    assert w.max() == 1.0
    # shift covariance: inc(ell + c) = inc(ell) + dbeta c, weights unchanged
    ell = inputs.log_weights(50, seed=4, spread=30.0)
    w1, i1 = tempering.reweight(ell, 0.05)
    w2, i2 = tempering.reweight(ell + 123.0, 0.05)
    assert i2 - i1 == pytest.approx(0.05 * 123.0, abs=1e-10)
    np.testing.assert_allclose(w1, w2, rtol=1e-12)


def test_kahan_matches_exact_rounded_sum():
    g = inputs.rng(7)
    xs = list(1e-3 * g.standard_normal(20000) + 1e3)
    k = tempering.KahanSum()
    for x in xs:
        k.add(x)
    assert k.s == pytest.approx(math.fsum(xs), rel=1e-15)
    # increments below half an ulp of the running value are kept by the compensation
    xs = [2.0 ** 53] + [1.0] * 1000
    k = tempering.KahanSum()
    for x in xs:
        k.add(x)
    assert k.s == math.fsum(xs) == 2.0 ** 53 + 1000
