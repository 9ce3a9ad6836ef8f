"""The estimate of Lemma 3.1 aggregated over r estimators (oracle).

Lemma 3.1: X_i = chi_i * |E| if the estimator's wedge is closed, else 0, and
E[X_i] = tau.  The plain mean tau_hat = (1/r) * sum_i X_i is computed exactly:
S = sum of chi over closed estimators, N = |E| * S, both as unbounded Python
integers (the CUDA side holds them in 128 bits); tau_hat as a double is
q + rem/r with q = N div r.  Median-of-means (Sec. 3.1, used by the paper's
implementation, Sec. 5) splits the estimators into g contiguous groups of
near-equal size, takes each group's exact mean and the median of those.

Pins: tests/test_oracle_estimate.py (Python big-integer arithmetic and
Fractions on random values).
"""
from __future__ import annotations

from fractions import Fraction


def mean_estimate(m: int, closed_chis, r: int):
    """(S, N, tau_hat) for the plain mean."""
    S = sum(int(c) for c in closed_chis)
    N = m * S
    q, rem = divmod(N, r)
    return S, N, float(q) + rem / r


def group_bounds(r: int, g: int):
    """Contiguous groups [lo, hi): group k holds estimators k*r//g .. (k+1)*r//g."""
    return [(k * r // g, (k + 1) * r // g) for k in range(g)]


def median_of_means(m: int, chis, closed, g: int) -> Fraction:
    """Median (lower median for even g) of the g exact group means."""
    r = len(chis)
    if not 1 <= g <= r:
        raise ValueError("1 <= g <= r")
    means = []
    for lo, hi in group_bounds(r, g):
        s = sum(int(chis[i]) for i in range(lo, hi) if closed[i])
        means.append(Fraction(m * s, hi - lo))
    means.sort()
    return means[(g - 1) // 2]
