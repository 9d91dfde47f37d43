"""Pins for the oracle's Philox4x32-10 and its uniform / normal conversions."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_rows():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        yield v[:4], v[4:6], v[6:]


def test_known_answer_vectors():
    rows = list(kat_rows())
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = [int(x) for x in philox.philox4x32_10(*ctr, *key)]
        assert got == out


def test_counter_sensitivity_and_vectorisation():
    # vectorised evaluation equals element-wise evaluation
    c2 = np.arange(5)
    vec = philox.philox4x32_10(7, 3, c2, 11, 0x1234, 0x5678)
    for i in range(5):
        one = philox.philox4x32_10(7, 3, i, 11, 0x1234, 0x5678)
        assert [int(v[i]) for v in vec] == [int(o) for o in one]
    assert len({int(vec[0][i]) for i in range(5)}) == 5


def test_box_muller_special_points():
    # u1 = 1 (word 2^32 - 1 -> (w + 1) 2^-32 = 1) gives radius 0
    z0, z1 = philox.box_muller_fp64(np.array([2 ** 32 - 1], np.uint64), np.array([12345], np.uint64))
    assert z0[0] == 0.0 and z1[0] == 0.0
    # u2 = 1/4 -> angle pi/2: cos = 0, sin = r; u1 = 2^-32 * (w+1) with w = 2^31 - 1 -> u1 = 1/2
    z0, z1 = philox.box_muller_fp64(np.array([2 ** 31 - 1], np.uint64), np.array([2 ** 30], np.uint64))
    r = np.sqrt(-2.0 * np.log(0.5))
    assert abs(z0[0]) < 1e-15 and abs(z1[0] - r) < 1e-15


def test_normals_moments():
    z = philox.normals(42, 0, philox.KIND_PROPOSE, 3, 1, 2000, 256)
    assert z.shape == (2000, 256)
    n = z.size
    assert abs(z.mean()) < 4.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 4.0 * np.sqrt(2.0 / n)
    # fourth moment 3, odd moments 0
    assert abs((z ** 4).mean() - 3.0) < 4.0 * np.sqrt(96.0 / n)
    # neighbouring columns (same and different Box-Muller pairs) uncorrelated
    for a, b in ((0, 1), (1, 2), (3, 4)):
        assert abs(np.corrcoef(z[:, a], z[:, b])[0, 1]) < 4.0 / np.sqrt(2000)
    z24 = philox.normals(42, 0, philox.KIND_PROPOSE, 3, 1, 2000, 256, bits=24)
    assert np.abs(z24 - z).max() < 2e-3  # same words, 24-bit truncation of the uniforms
    assert np.median(np.abs(z24 - z)) < 1e-6


def test_uniform53_range_and_streams():
    u = philox.uniform53(1, 0, philox.KIND_ACCEPT, 1, 0, np.arange(100000))
    assert (u > 0).all() and (u <= 1).all()
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
    # a different stream id changes the key and hence the draws
    v = philox.uniform53(1, 1, philox.KIND_ACCEPT, 1, 0, np.arange(100000))
    assert not np.array_equal(u, v)
