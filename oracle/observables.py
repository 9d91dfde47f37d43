"""Observables of a weighted particle population (Sec. 2 magnetisation; App. F
mode balance).

Test infrastructure (see ``oracle/__init__``).

Readings: the paper does not define a susceptibility; chi = D (<M^2> - <M>^2)
(connected, M the lattice-mean field) is used. Mode balance follows App. F:
the (weighted) count of M > 0 over the count of M < 0, zeros ignored, +inf when
nothing is negative, 0 when nothing is positive (and NaN when both are empty).
"""
import math

import numpy as np

from . import lattice


def mode_balance(M, weights=None):
    M = np.asarray(M, dtype=np.float64)
    w = np.ones_like(M) if weights is None else np.asarray(weights, dtype=np.float64)
    pos = float(w[M > 0].sum())
    neg = float(w[M < 0].sum())
    if neg == 0.0:
        return math.inf if pos > 0.0 else math.nan
    return pos / neg


def summary(phi, weights=None):
    """Weighted moments of M over the particles (weights default to uniform)."""
    M = lattice.magnetisation(phi)
    D = np.asarray(phi).shape[-1]
    w = np.ones_like(M) if weights is None else np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    mean_M = float((w * M).sum())
    mean_absM = float((w * np.abs(M)).sum())
    mean_M2 = float((w * M * M).sum())
    return {
        "mean_M": mean_M,
        "mean_absM": mean_absM,
        "mean_M2": mean_M2,
        "chi": D * (mean_M2 - mean_M ** 2),
        "mode_balance": mode_balance(M, w),
    }
