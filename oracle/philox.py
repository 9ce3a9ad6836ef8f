"""Philox4x32-10 counter-based generator (oracle side).

Written from the published definition: J. Salmon, M. Moraes, R. Dror,
D. Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11, Sec. 3
(the Philox S-box built from two 32x32->64 multiplies, the key schedule
adding the Weyl constants, 10 rounds for the 4x32 variant).

The paper on triangle counting leaves its random source unspecified (Step 1
``randInt``, Sec. 4.2; Step 2 coin and phi, Sec. 4.3), so a counter-based
generator is used to make every draw reproducible from
(seed, stream, estimator, batch, slot).

Pins: the published known-answer vectors of the Random123 distribution for
philox4x32 with 10 rounds (tests/test_oracle_philox.py), agreement of the
scalar and numpy forms, and -- on a GPU -- agreement with the toolkit's own
Philox4x32-10 device function.
"""
from __future__ import annotations

import numpy as np

# Multipliers and Weyl key increments of Philox4x32 (Salmon et al., Table 2).
M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF
ROUNDS = 10


def _round(c, k):
    """One Philox S-box round on four 32-bit words with a two-word key."""
    p0 = M0 * c[0]
    p1 = M1 * c[2]
    hi0, lo0 = p0 >> 32, p0 & MASK32
    hi1, lo1 = p1 >> 32, p1 & MASK32
    return (hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0)


def philox4x32(counter, key, rounds: int = ROUNDS):
    """Scalar Philox4x32-R: counter = 4 ints, key = 2 ints -> 4 ints.

    Round j (0-based) uses the key advanced j times by the Weyl increments.
    """
    c = tuple(int(x) & MASK32 for x in counter)
    k = [int(key[0]) & MASK32, int(key[1]) & MASK32]
    for j in range(rounds):
        if j:
            k = [(k[0] + W0) & MASK32, (k[1] + W1) & MASK32]
        c = _round(c, k)
    return c


def philox4x32_np(c0, c1, c2, c3, k0: int, k1: int, rounds: int = ROUNDS):
    """Vectorised Philox4x32-R over numpy arrays of 32-bit counter words.

    All counter arguments broadcast; the key is a pair of Python ints.
    Returns four uint64 arrays holding 32-bit values.
    """
    m = np.uint64(MASK32)
    x0 = np.asarray(c0, dtype=np.uint64) & m
    x1 = np.asarray(c1, dtype=np.uint64) & m
    x2 = np.asarray(c2, dtype=np.uint64) & m
    x3 = np.asarray(c3, dtype=np.uint64) & m
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    ka, kb = int(k0) & MASK32, int(k1) & MASK32
    s32 = np.uint64(32)
    for j in range(rounds):
        if j:
            ka, kb = (ka + W0) & MASK32, (kb + W1) & MASK32
        p0 = np.uint64(M0) * x0
        p1 = np.uint64(M1) * x2
        hi0, lo0 = p0 >> s32, p0 & m
        hi1, lo1 = p1 >> s32, p1 & m
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(ka), lo1,
                          hi0 ^ x3 ^ np.uint64(kb), lo0)
    return x0, x1, x2, x3
