"""Pins for the exact aggregate of Lemma 3.1 and median-of-means."""
import random
import statistics
from fractions import Fraction

from oracle import estimate


def test_mean_estimate_exact():
    rnd = random.Random(1)
    for _ in range(50):
        r = rnd.randint(1, 1000)
        m = rnd.randint(1, 10**12)
        chis = [rnd.randint(0, 10**7) for _ in range(r)]
        closed = [rnd.random() < 0.3 for _ in range(r)]
        S, N, tau = estimate.mean_estimate(m, [c for c, k in zip(chis, closed) if k], r)
        assert N == m * S
        assert Fraction(N, r) == Fraction(sum(m * c for c, k in zip(chis, closed) if k), r)
        assert abs(tau - N / r) <= 1e-9 * max(1.0, N / r)


def test_median_of_means():
    rnd = random.Random(2)
    for _ in range(30):
        r = rnd.randint(5, 200)
        g = rnd.randint(1, r)
        m = rnd.randint(1, 1000)
        chis = [rnd.randint(0, 50) for _ in range(r)]
        closed = [rnd.random() < 0.5 for _ in range(r)]
        bounds = estimate.group_bounds(r, g)
        assert bounds[0][0] == 0 and bounds[-1][1] == r
        assert all(b[1] == c[0] for b, c in zip(bounds, bounds[1:]))
        means = [Fraction(m * sum(chis[i] for i in range(lo, hi) if closed[i]), hi - lo)
                 for lo, hi in bounds]
        assert estimate.median_of_means(m, chis, closed, g) == statistics.median_low(means)
    # one group is the plain mean
    assert estimate.median_of_means(7, [3, 4], [True, True], 1) == Fraction(49, 2)
