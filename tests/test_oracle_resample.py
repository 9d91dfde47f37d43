"""Pins for the fixed-point systematic resampler: brute force with exact
rationals, the offspring-count property and the textbook float form."""
from fractions import Fraction

import numpy as np
import pytest

import inputs
from oracle import resample


def brute_force(w, U):
    q = resample.quantise(w)
    Q = sum(q)
    n = len(q)
    out = []
    for i in range(n):
        pos = (Fraction(i) + Fraction(U, 2 ** 32)) * Fraction(Q, n)  # position in quantised mass
        acc = 0
        for j, qj in enumerate(q):
            acc += qj
            if acc > pos:
                out.append(j)
                break
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 16])
def test_brute_force_tiny(n):
    for seed in range(6):
        w = inputs.positive_weights(n, seed=seed, zeros=min(seed % 3, n - 1))
        U = inputs.word32(seed + 100)
        assert list(resample.systematic(w, U)) == brute_force(w, U)


def test_offspring_counts_floor_or_ceil():
    for seed in range(10):
        n = 257
        w = inputs.positive_weights(n, seed=seed, heavy=bool(seed % 2))
        U = inputs.word32(seed)
        anc = resample.systematic(w, U)
        assert (np.diff(anc) >= 0).all()
        q = np.array(resample.quantise(w), dtype=object)
        Q = int(sum(q))
        counts = np.bincount(anc, minlength=n)
        for j in range(n):
            lo = (n * int(q[j])) // Q
            hi = lo + (1 if (n * int(q[j])) % Q else 0)
            assert lo <= counts[j] <= hi
        assert counts.sum() == n


def test_equal_and_degenerate_weights():
    n = 40
    assert list(resample.systematic(np.ones(n), 0)) == list(range(n))
    assert list(resample.systematic(np.ones(n), 2 ** 32 - 1)) == list(range(n))
    w = np.zeros(n)
    w[17] = 0.3
    assert set(resample.systematic(w, 12345)) == {17}


def test_agrees_with_textbook_float_form_away_from_ties():
    n = 1000
    w = inputs.positive_weights(n, seed=11)
    U = inputs.word32(5)
    anc = resample.systematic(w, U)
    cdf = np.cumsum(w / w.sum())
    pos = (np.arange(n) + U / 2 ** 32) / n
    tb = np.searchsorted(cdf, pos, side="right")
    gap = np.min(np.abs(cdf[:, None] - pos[None, :]), axis=0)
    far = gap > 1e-9
    assert far.sum() > 990
    np.testing.assert_array_equal(anc[far], tb[far])
