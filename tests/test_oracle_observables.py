"""Pins for the magnetisation observables and mode balance (App. F)."""
import math

import numpy as np
import pytest

import closed_forms as cf
import inputs
from oracle import observables


def test_mode_balance_edge_cases():
    assert observables.mode_balance([1.0, 2.0, -1.0]) == 2.0
    assert observables.mode_balance([0.0, 1.0, -1.0, 0.0]) == 1.0     # zeros ignored
    assert observables.mode_balance([0.5, 0.1]) == math.inf           # nothing negative
    assert observables.mode_balance([-0.5, -0.1]) == 0.0              # nothing positive
    assert math.isnan(observables.mode_balance([0.0, 0.0]))
    assert observables.mode_balance([1.0, -1.0], weights=[3.0, 1.0]) == 3.0


def test_free_field_moments_from_exact_draws():
    L, m2, N = 8, 1.0, 40000
    phi = cf.free_field_sample(L, m2, 1.0, N, inputs.rng(3))
    o = observables.summary(phi)
    var, absm, chi = cf.free_field_moments(L, m2)
    assert abs(o["mean_M"]) < 4 * math.sqrt(var / N)
    assert abs(o["mean_absM"] - absm) < 4 * math.sqrt(var / N)
    assert abs(o["chi"] - chi) < 4 * chi * math.sqrt(2.0 / N)
    assert 0.9 < o["mode_balance"] < 1.1


def test_weighted_moments_by_hand():
    # four particles on a 2 x 2 lattice whose lattice means are 0.5, -1, 2 and 0, with
    # weights 3 : 2 : 1 : 4; every moment worked out by hand over the normalised weights
    phi = np.array([[0.9, 0.1, 0.7, 0.3],
                    [-1.0, -2.0, 0.0, -1.0],
                    [2.5, 1.5, 2.0, 2.0],
                    [0.4, -0.4, 1.0, -1.0]])
    o = observables.summary(phi, weights=[3.0, 2.0, 1.0, 4.0])
    assert o["mean_M"] == pytest.approx(0.15, rel=1e-14)             # (1.5 - 2 + 2 + 0) / 10
    assert o["mean_absM"] == pytest.approx(0.55, rel=1e-14)          # (1.5 + 2 + 2) / 10
    assert o["mean_M2"] == pytest.approx(0.675, rel=1e-14)           # (0.75 + 2 + 4) / 10
    assert o["chi"] == pytest.approx(4 * (0.675 - 0.15 ** 2), rel=1e-13)
    assert o["mode_balance"] == pytest.approx(2.0, rel=1e-14)        # (3 + 1) / 2, the zero ignored
