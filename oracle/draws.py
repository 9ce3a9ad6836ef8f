"""Bounded integer draws and the fixed draw conventions (oracle side).

The paper's Step 1 draws ``randInt(|W|+|E|)`` (Sec. 4.2) and Step 2 flips a
coin with probability chi-/(chi-+chi+) and draws phi in [0, chi+) (Sec. 4.3);
it fixes neither the generator nor how words become bounded integers.  The
readings used here (identical on the CUDA side, written independently):

* Words.  One Philox4x32-10 call with counter (i, b, stream, slot) and key
  (seed_lo32, seed_hi32) gives two 64-bit words, (x0 | x1<<32) then
  (x2 | x3<<32).  i = estimator index, b = batch index of the stream.
* Purposes.  Step 1 consumes words from slots 0, 2, 4, ...; Step 2 from slots
  1, 3, 5, ....  Word j of purpose P is half (j mod 2) of slot P + 2*(j div 2).
* Bounded draw U(n), n >= 1: Lemire's nearly-divisionless method
  (D. Lemire, "Fast Random Integer Generation in an Interval", ACM TOMACS
  29(1), 2019): multiply the word by n in double width; if the low half is
  below the threshold (2^k - n) mod n the word is rejected and the next word
  of the same purpose is used; the result is the high half.
* Step 2 makes a single draw y = U(chi- + chi+); y < chi- keeps f2, otherwise
  phi = y - chi- names the new level-2 edge.  This has exactly the two-stage
  distribution of Sec. 4.3.  No draw is made when chi+ = 0.

Pins: exhaustive uniformity of ``bounded`` on 8- and 12-bit words for every
n (tests/test_oracle_draws.py); slot/half layout checked against direct
Philox calls.
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32, philox4x32_np

STEP1 = 0  # purpose of the level-1 reservoir draw (Sec. 4.2)
STEP2 = 1  # purpose of the level-2 coin / phi draw (Sec. 4.3)


def bounded(words, n: int, bits: int = 64) -> int:
    """Lemire's bounded draw of an integer in [0, n) from an iterator of words.

    ``bits`` is the word width (64 in production; small widths let the tests
    enumerate every word).
    """
    if n < 1:
        raise ValueError("bounded draw needs n >= 1")
    full = 1 << bits
    x = next(words)
    prod = x * n
    low = prod % full
    if low < n:
        threshold = (full - n) % n
        while low < threshold:
            x = next(words)
            prod = x * n
            low = prod % full
    return prod >> bits


def word(seed: int, stream: int, i: int, b: int, purpose: int, j: int) -> int:
    """64-bit word j of the given purpose for estimator i in batch b."""
    slot = purpose + 2 * (j // 2)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    x0, x1, x2, x3 = philox4x32((i, b, stream, slot), key)
    if j % 2 == 0:
        return x0 | (x1 << 32)
    return x2 | (x3 << 32)


def word_stream(seed: int, stream: int, i: int, b: int, purpose: int):
    """Infinite iterator over the words of one purpose."""
    j = 0
    while True:
        yield word(seed, stream, i, b, purpose, j)
        j += 1


class PhiloxDraws:
    """Draw source for the scalar oracle: U(n) for (estimator, purpose).

    ``begin_batch(b)`` selects the batch counter; each estimator makes at
    most one draw per purpose per batch, restarting at word 0.
    """

    def __init__(self, seed: int, stream: int = 0):
        self.seed = int(seed)
        self.stream = int(stream)
        self.b = 0

    def begin_batch(self, b: int) -> None:
        self.b = int(b)

    def U(self, i: int, purpose: int, n: int) -> int:
        return bounded(word_stream(self.seed, self.stream, i, self.b, purpose), n)


# ---------------------------------------------------------------------------
# numpy form, one draw per selected estimator
# ---------------------------------------------------------------------------

def _words_np(seed, stream, idx, b, purpose, j):
    slot = purpose + 2 * (j // 2)
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    x0, x1, x2, x3 = philox4x32_np(idx, np.uint64(b), np.uint64(stream),
                                   np.uint64(slot), k0, k1)
    if j % 2 == 0:
        return x0 | (x1 << np.uint64(32))
    return x2 | (x3 << np.uint64(32))


def _mul64(x, n):
    """Full 128-bit product of uint64 arrays as (high, low) uint64 arrays."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    xl, xh = x & m32, x >> s32
    nl, nh = n & m32, n >> s32
    ll = xl * nl
    lh = xl * nh
    hl = xh * nl
    hh = xh * nh
    mid = (ll >> s32) + (lh & m32) + (hl & m32)
    low = (ll & m32) | ((mid & m32) << s32)
    high = hh + (lh >> s32) + (hl >> s32) + (mid >> s32)
    return high, low


def bounded_np(seed: int, stream: int, idx, b: int, purpose: int, n):
    """U(n) for each estimator index in ``idx`` (uint64 arrays, n >= 1)."""
    idx = np.asarray(idx, dtype=np.uint64)
    n = np.asarray(n, dtype=np.uint64)
    if idx.size == 0:
        return np.zeros(0, dtype=np.uint64)
    if np.any(n == 0):
        raise ValueError("bounded draw needs n >= 1")
    out = np.empty(idx.shape, dtype=np.uint64)
    pending = np.arange(idx.size)
    # threshold (2^64 - n) mod n, computed in uint64 arithmetic
    thresh = (np.uint64(0) - n) % n
    j = 0
    while pending.size:
        x = _words_np(seed, stream, idx[pending], b, purpose, j)
        high, low = _mul64(x, n[pending])
        ok = low >= thresh[pending]
        out[pending[ok]] = high[ok]
        pending = pending[~ok]
        j += 1
    return out
