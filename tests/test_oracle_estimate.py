"""Pins for the exact aggregate of Lemma 3.1 and median-of-means.

Every expected value here is written out by hand: the integer arithmetic of
the cases is small enough to check on paper, and each case is chosen so that
one plausible slip (N not multiplied by |E|, the rem / r term dropped, a
group boundary off by one, the upper median taken for even g) changes it.
"""
from fractions import Fraction

import pytest

from oracle import estimate


def test_mean_estimate_hand_values():
    # Lemma 3.1: X_i = |E| * chi_i for a closed estimator, tau_hat = mean X_i.
    # |E| = 10, closed chis 3 and 4, r = 4: S = 7, N = 70, 70 / 4 = 17.5.
    assert estimate.mean_estimate(10, [3, 4], 4) == (7, 70, 17.5)
    # rem / r matters: |E| = 5, S = 1, r = 3 -> N = 5 = 1 * 3 + 2, so
    # tau_hat = 1 + fl(2/3).  fl(2/3) = 0x1.5555555555555p-1; adding 1 gives
    # 0x1.aaaaaaaaaaaaa8p+0, a tie at 53 bits that rounds to the even
    # 0x1.aaaaaaaaaaaaap+0 -- one ulp below the correctly rounded 5/3, which
    # is what the defined q + rem / r form (two roundings) must give.
    S, N, tau = estimate.mean_estimate(5, [1], 3)
    assert (S, N) == (1, 5)
    assert tau == float.fromhex("0x1.aaaaaaaaaaaaap+0") and tau != 5 / 3
    # nothing closed
    assert estimate.mean_estimate(123, [], 7) == (0, 0, 0.0)


def test_mean_estimate_beyond_64_bits():
    # |E| = 2^32, closed chis 2^33 and 2^33: S = 2^34, N = 2^66 (three words
    # wide); r = 3: 2^66 = 3 q + 1 with q = (2^66 - 1) / 3 =
    # 24595658764946068821 (the 0x5555...5 pattern: 2^66 - 1 = 3 * 0x1555...5).
    S, N, tau = estimate.mean_estimate(1 << 32, [1 << 33, 1 << 33], 3)
    assert S == 1 << 34 and N == 1 << 66
    assert 3 * 24595658764946068821 + 1 == 1 << 66
    # q's nearest double is 0x4395555555555555 (q = 0x15555555555555555, 65
    # bits: the 53 kept bits are 1 0101...01, the 12 dropped ones 0101 0101
    # 0101 are below half an ulp); rem / r = 1/3 is far below an ulp of q.
    assert tau == float.fromhex("0x1.5555555555555p+64")
    # r = 2^64 + 1 does not divide 2^66: q = 3, rem = 2^66 - 3 (2^64 + 1)
    # = 2^64 - 3, so tau = 3 + (2^64 - 3) / (2^64 + 1) ~= 4 - 4/2^64, which
    # rounds to exactly 4.0; r = 2^66 + 1 leaves q = 0 and tau = fl(2^66 /
    # (2^66 + 1)) = fl(1 - 1/(2^66 + 1)) = 1.0 (the gap to 1 is far below
    # half an ulp, 2^-54): the whole value comes from the rem / r term.
    assert estimate.mean_estimate(1 << 32, [1 << 33, 1 << 33], (1 << 64) + 1)[2] == 4.0
    assert estimate.mean_estimate(1 << 32, [1 << 33, 1 << 33], (1 << 66) + 1)[2] == 1.0


def test_group_bounds_hand_values():
    # group k holds estimators [k r / g, (k+1) r / g), floors
    assert estimate.group_bounds(5, 1) == [(0, 5)]
    assert estimate.group_bounds(5, 2) == [(0, 2), (2, 5)]
    assert estimate.group_bounds(5, 3) == [(0, 1), (1, 3), (3, 5)]
    assert estimate.group_bounds(7, 3) == [(0, 2), (2, 4), (4, 7)]
    assert estimate.group_bounds(4, 4) == [(0, 1), (1, 2), (2, 3), (3, 4)]


def test_median_of_means_hand_values():
    m = 6
    chis = [1, 2, 3, 4, 5]
    closed = [True, False, True, True, False]
    # g = 2, r = 5: groups {0,1} and {2,3,4}; closed sums 1 and 3+4 = 7;
    # means 6*1/2 = 3 and 6*7/3 = 14; lower median of two = 3.
    assert estimate.median_of_means(m, chis, closed, 2) == Fraction(3)
    # g = 3: groups {0}, {1,2}, {3,4}; sums 1, 3, 4; means 6, 9, 12 -> 9.
    assert estimate.median_of_means(m, chis, closed, 3) == Fraction(9)
    # g = 5: each estimator alone: 6, 0, 18, 24, 0 -> sorted 0 0 6 18 24 -> 6.
    assert estimate.median_of_means(m, chis, closed, 5) == Fraction(6)
    # g = 4, r = 5: groups {0}, {1}, {2}, {3,4}: 6, 0, 18, 6*4/2 = 12;
    # sorted 0 6 12 18, lower median 6.
    assert estimate.median_of_means(m, chis, closed, 4) == Fraction(6)
    # g = 1 is the plain mean: 6 * (1+3+4) / 5 = 48/5
    assert estimate.median_of_means(m, chis, closed, 1) == Fraction(48, 5)
    # one group is the plain mean (exact fraction)
    assert estimate.median_of_means(7, [3, 4], [True, True], 1) == Fraction(49, 2)


def test_median_of_means_rejects_bad_g():
    with pytest.raises(ValueError):
        estimate.median_of_means(1, [1, 2], [True, True], 0)
    with pytest.raises(ValueError):
        estimate.median_of_means(1, [1, 2], [True, True], 3)
