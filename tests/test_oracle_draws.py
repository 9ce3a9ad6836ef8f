"""Oracle pins for the bounded draw and the draw conventions.

Lemire's method accepts exactly 2^k - (2^k mod n) of the 2^k words and maps
floor(2^k / n) of them to each value in [0, n); checked exhaustively on 8-
and 12-bit words, where every word can be enumerated.
"""
import numpy as np
import pytest

from oracle import draws
from oracle.philox import philox4x32


@pytest.mark.parametrize("bits", [8, 12])
def test_bounded_exhaustively_uniform(bits):
    full = 1 << bits
    for n in list(range(1, 80)) + [full // 3, full // 2 + 1, full - 1, full]:
        hits = [0] * n
        rejected = 0
        for x in range(full):
            it = iter([x, None])
            try:
                v = draws.bounded(it, n, bits=bits)
            except TypeError:
                rejected += 1   # the method asked for another word
                continue
            hits[v] += 1
        assert rejected == full % n
        assert all(h == full // n for h in hits), n


def test_power_of_two_is_a_shift():
    for k in (1, 5, 17, 63):
        for x in (0, 1, 12345, (1 << 64) - 1, 0xDEADBEEFCAFEF00D):
            assert draws.bounded(iter([x]), 1 << k) == x >> (64 - k)


def test_word_layout():
    seed, stream, i, b = 0x1122334455667788, 7, 99, 3
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for purpose in (draws.STEP1, draws.STEP2):
        for j in range(6):
            slot = purpose + 2 * (j // 2)
            x = philox4x32((i, b, stream, slot), key)
            expect = x[0] | (x[1] << 32) if j % 2 == 0 else x[2] | (x[3] << 32)
            assert draws.word(seed, stream, i, b, purpose, j) == expect


def test_numpy_form_matches_scalar_including_rejections():
    seed, stream, b = 42, 3, 5
    idx = np.arange(400, dtype=np.uint64)
    # huge n forces frequent rejection (threshold near 2^63)
    for n in (1, 2, 7, 10**9 + 7, (1 << 63) + 12345, (1 << 64) - 3):
        got = draws.bounded_np(seed, stream, idx, b, draws.STEP2,
                               np.full(idx.size, n, dtype=np.uint64))
        for i in range(0, 400, 7):
            ref = draws.bounded(draws.word_stream(seed, stream, i, b, draws.STEP2), n)
            assert int(got[i]) == ref
