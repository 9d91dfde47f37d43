"""Philox4x32-10 counter-based generator and the random-number layout of the samplers.

Test infrastructure (see ``oracle/__init__``). Written from the published
definition of Philox4x32 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11): a 4x32-bit counter is mixed with a 2x32-bit key by
ten rounds; each round multiplies counter words 0 and 2 by the two Philox
constants, exchanges high and low product halves with the other two words and
xors in the key; the key is advanced by the two Weyl constants between rounds.

The paper draws its random numbers from JAX keys (Sec. 2, samplers run through
blackjax) and fixes no generator, so both the oracle and the CUDA path use this
counter layout (a reading of the paper, listed in the design notes):

* key     = (seed mod 2^32, (seed >> 32) xor stream)          (both 32-bit)
* counter = (kind << 24 | step, sub, particle, block)

with ``step`` the temperature (or nested-sampling iteration) index, ``sub`` the
MCMC sweep (or slice step), ``particle`` the particle (or slot) index and
``block`` the group of four consecutive outputs.
"""
import numpy as np

MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85

# Stream kinds (bits 24..31 of counter word 0).
KIND_INIT = 1
KIND_RESAMPLE = 2
KIND_PROPOSE = 3
KIND_ACCEPT = 4
KIND_NS_START = 5
KIND_NS_DIRECTION = 6
KIND_NS_SLICE = 7
KIND_FLIP = 8


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds. Arguments are integers or uint arrays (broadcast).

    Returns four uint64 arrays holding 32-bit words.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (c.copy() for c in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & MASK32)
    k1 = np.uint64(int(k1) & MASK32)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    mask = np.uint64(MASK32)
    s32 = np.uint64(32)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint64((int(k0) + PHILOX_W0) & MASK32)
            k1 = np.uint64((int(k1) + PHILOX_W1) & MASK32)
        p0 = m0 * c0          # < 2^64, exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def key_of(seed, stream=0):
    seed = int(seed)
    return seed & MASK32, ((seed >> 32) ^ int(stream)) & MASK32


def counter_word0(kind, step):
    return ((int(kind) & 0xFF) << 24) | (int(step) & 0xFFFFFF)


def words(seed, stream, kind, step, sub, particles, blocks):
    """Philox output for every (particle, block) pair: uint64 array [P, B, 4]."""
    k0, k1 = key_of(seed, stream)
    p = np.asarray(particles, dtype=np.uint64)[:, None]
    b = np.asarray(blocks, dtype=np.uint64)[None, :]
    w = philox4x32_10(counter_word0(kind, step), sub, p, b, k0, k1)
    return np.stack(w, axis=-1)


def box_muller_fp64(wa, wb):
    """Two normals from two 32-bit words, in float64.

    u1 = (wa + 1) 2^-32 in (0, 1], u2 = wb 2^-32 in [0, 1);
    r = sqrt(-2 ln u1); returns (r cos 2 pi u2, r sin 2 pi u2).
    """
    u1 = (wa.astype(np.float64) + 1.0) * 2.0 ** -32
    u2 = wb.astype(np.float64) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return r * np.cos(ang), r * np.sin(ang)


def box_muller_24(wa, wb):
    """Two normals from the top 24 bits of two words (the single-precision draw),
    evaluated here in float64: u1 = ((wa >> 8) + 1) 2^-24, u2 = (wb >> 8) 2^-24."""
    u1 = ((wa >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (wb >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return r * np.cos(ang), r * np.sin(ang)


def normals(seed, stream, kind, step, sub, n_rows, n_cols, bits=32, row0=0):
    """Standard normals [n_rows, n_cols]: row r uses particle counter row0 + r,
    column j is output j % 4 of block j // 4 (pairs (0,1) and (2,3) of each
    block feed one Box-Muller transform each). ``bits`` = 32 (double-precision
    draw) or 24 (single-precision draw)."""
    n_blocks = (n_cols + 3) // 4
    w = words(seed, stream, kind, step, sub, np.arange(row0, row0 + n_rows), np.arange(n_blocks))
    bm = box_muller_fp64 if bits == 32 else box_muller_24
    z0, z1 = bm(w[..., 0], w[..., 1])
    z2, z3 = bm(w[..., 2], w[..., 3])
    z = np.stack([z0, z1, z2, z3], axis=-1).reshape(n_rows, n_blocks * 4)
    return z[:, :n_cols]


def uniform53(seed, stream, kind, step, sub, particles):
    """One uniform in (0, 1] per particle from words 0 and 1 of block 0:
    x = (w0 << 21) | (w1 >> 11) (53 bits), u = (x + 1) 2^-53."""
    w = words(seed, stream, kind, step, sub, particles, [0])[:, 0, :]
    x = (w[:, 0] << np.uint64(21)) | (w[:, 1] >> np.uint64(11))
    return (x.astype(np.float64) + 1.0) * 2.0 ** -53


def uniform53_words(w0, w1):
    x = (np.asarray(w0, np.uint64) << np.uint64(21)) | (np.asarray(w1, np.uint64) >> np.uint64(11))
    return (x.astype(np.float64) + 1.0) * 2.0 ** -53


def word32(seed, stream, kind, step, sub=0, particle=0, block=0, index=0):
    """A single 32-bit word (e.g. the systematic-resampling offset)."""
    w = words(seed, stream, kind, step, sub, [particle], [block])
    return int(w[0, 0, index])
