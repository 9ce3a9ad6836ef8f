"""Oracle pins for Philox4x32-10 (Salmon et al., SC'11).

Known-answer vectors are the ones published with the Random123 library for
philox4x32 with 10 rounds (counter, key -> output).
"""
import numpy as np

from oracle.philox import philox4x32, philox4x32_np

KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


def test_known_answers_scalar():
    for ctr, key, out in KAT:
        assert philox4x32(ctr, key) == out


def test_known_answers_numpy():
    for ctr, key, out in KAT:
        got = philox4x32_np(*[np.array([c], dtype=np.uint64) for c in ctr], *key)
        assert tuple(int(g[0]) for g in got) == out


def test_scalar_and_numpy_agree():
    rng = np.random.default_rng(5)
    c = rng.integers(0, 2**32, size=(4, 200), dtype=np.uint64)
    k0, k1 = 0x12345678, 0x9ABCDEF0
    got = philox4x32_np(c[0], c[1], c[2], c[3], k0, k1)
    for j in range(200):
        ref = philox4x32(tuple(int(x) for x in c[:, j]), (k0, k1))
        assert tuple(int(g[j]) for g in got) == ref
