"""Pins for the magnetisation observables and mode balance (App. F)."""
import math

import numpy as np

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
