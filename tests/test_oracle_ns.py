"""Pins for the nested-sampling oracle: the exact prior bracket, evidence on
one site against quadrature and on the 2 x 2 torus against its transfer matrix, the
error bar sqrt(H / N) against the seed-to-seed spread, the information H against
quadrature, the evidence with the live points at any stopping point, and the stopping
rule."""
import math

import numpy as np
import pytest

import closed_forms as cf
import inputs
from oracle import ns


def test_prior_bracket_roots():
    g = inputs.rng(1)
    for _ in range(20):
        x, d = g.standard_normal(6), g.standard_normal(6)
        E = float(g.exponential())
        lo, hi = ns.prior_bracket(x, d, E)
        assert lo < 0 < hi
        for t in (lo, hi):
            assert np.dot(x + t * d, x + t * d) == pytest.approx(np.dot(x, x) + 2 * E, rel=1e-10)


def test_one_site_evidence_and_error_bar():
    ref = cf.one_site_logz(-4.0, 8.0)
    res = [ns.NS(ns.NSConfig(L=1, N=64, m2=-4.0, lam=8.0, n_delete=32, seed=s)).run() for s in range(4)]
    lz = np.array([r["logz"] for r in res])
    err = np.mean([r["logz_err"] for r in res])
    assert abs(lz.mean() - ref) < 4.0 * err / math.sqrt(len(lz)) + 0.02
    assert 0.02 < err < 0.5
    assert all(r["capped"] == 0 for r in res)


def test_volume_bookkeeping_single_deletion():
    s = ns.NS(ns.NSConfig(L=1, N=16, m2=-4.0, lam=8.0, n_delete=1, seed=2))
    for _ in range(10):
        s.replace_step()
    # each single deletion shrinks log X by exactly 1/N
    assert s.logX == pytest.approx(-10.0 / 16, rel=1e-14)
    w = np.exp(np.array(s.dead_logw))
    assert w.sum() == pytest.approx(1.0 - math.exp(s.logX), rel=1e-12)


def test_two_by_two_torus_evidence_and_error_bar():
    # the interacting 2 x 2 torus (the kinetic term a 4-cycle with coupling 2): log Z from
    # the transfer matrix, tr T^4; the error bar sqrt(H / N) matches the spread of 8 seeds
    ref = cf.two_by_two_logz(-4.0, 8.0)
    res = [ns.NS(ns.NSConfig(L=2, N=64, m2=-4.0, lam=8.0, n_delete=32, seed=100 + s)).run() for s in range(8)]
    lz = np.array([r["logz"] for r in res])
    err = np.mean([r["logz_err"] for r in res])
    assert abs(lz.mean() - ref) < 4.0 * err / math.sqrt(len(lz)) + 0.02, (lz.mean(), ref, err)
    assert 0.4 < lz.std(ddof=1) / err < 2.5
    assert all(r["capped"] == 0 for r in res)


def test_evidence_with_the_live_points_at_any_stopping_point():
    # dead points' weights plus X times the mean live likelihood estimate Z after any
    # number of iterations; after 3 deletions of half the points the live points still
    # carry most of the mass, so their weight X / N is what this checks
    ref = cf.one_site_logz(-4.0, 8.0)
    lz = []
    for s in range(6):
        run = ns.NS(ns.NSConfig(L=1, N=64, m2=-4.0, lam=8.0, n_delete=32, seed=20 + s))
        for _ in range(3):
            run.replace_step()
        lz.append(run.final()[0])
    lz = np.array(lz)
    assert abs(lz.mean() - ref) < 4.0 * lz.std(ddof=1) / math.sqrt(len(lz)) + 0.02, (lz.mean(), ref)


def test_information_and_stopping_rule():
    # H = E_post[log L] - log Z against quadrature; the run stops at the first iteration
    # whose remaining evidence X mean(L_live) is below stop_frac of the accumulated Z
    H_ref = cf.one_site_information(-4.0, 8.0)
    Hs = []
    for s in range(4):
        run = ns.NS(ns.NSConfig(L=1, N=64, m2=-4.0, lam=8.0, n_delete=32, seed=s))
        prev = []
        while not run.done:
            prev.append(run.remaining_log_evidence() - run.logZ)
            run.replace_step()
        assert run.remaining_log_evidence() - run.logZ < math.log(1e-3)
        assert all(g >= math.log(1e-3) for g in prev[1:]), prev
        assert run.it >= 2
        Hs.append(run.result()["H"])
    Hs = np.array(Hs)
    assert abs(Hs.mean() - H_ref) < 4.0 * Hs.std(ddof=1) / math.sqrt(len(Hs)) + 0.02, (Hs.mean(), H_ref)
