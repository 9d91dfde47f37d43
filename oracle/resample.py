"""Systematic resampling in exact fixed point.

Test infrastructure (see ``oracle/__init__``).

The paper resamples inside blackjax's tempered SMC (Sec. 2 (i); Table 3 notes
that a higher target ESS resamples more often) without naming a scheme. The
reading used here is systematic resampling with integer arithmetic so that
every implementation returns the same ancestors for the same weights:

    q_i = floor(ldexp(w_i / w_max, 46))            (unsigned 64-bit)
    Q   = sum_i q_i,  C_j = sum_{k <= j} q_k        (exact for N <= 2^17)
    p_i = floor(((i * 2^32 + U) * Q) / (N * 2^32))  (exact integer arithmetic)
    a_i = min { j : C_j > p_i }

with U a 32-bit random word. Since C_j is an integer, C_j > p_i exactly when
C_j exceeds the real position (i + U 2^-32) Q / N, so this is textbook
systematic resampling on the quantised weights q.
"""
import bisect
import math

import numpy as np

FIXED_POINT_BITS = 46


def quantise(w):
    w = np.asarray(w, dtype=np.float64)
    wmax = w.max()
    return [int(math.floor(math.ldexp(float(x) / float(wmax), FIXED_POINT_BITS))) for x in w]


def systematic(w, U):
    """Ancestor indices (nondecreasing, int64) for weights w and offset word U."""
    q = quantise(w)
    n = len(q)
    Q = sum(q)
    C = []
    acc = 0
    for x in q:
        acc += x
        C.append(acc)
    out = np.empty(n, dtype=np.int64)
    for i in range(n):
        p = (((i << 32) + int(U)) * Q) // (n << 32)
        out[i] = bisect.bisect_right(C, p)
    return out
