"""Statistical pin: the oracle's estimate is unbiased (Lemma 3.1).

10^4 seeds (1..10^4), each a stream of a small Chung-Lu graph in batches,
r estimators per seed.  The exact variance of one estimator follows from the
Claim of Sec. 3.1: Var[X] = m * sum_t C(t) - tau^2.  The mean of the
10^4 * r estimates must lie within 4.5 standard errors of tau.
"""
import math

import numpy as np

import synth
from oracle import exact, nbsi_bulk


def test_unbiased_over_ten_thousand_seeds():
    n, m, r, w = 40, 120, 4, 40
    keys = synth.finish(synth.chung_lu(n, 2.3, 6.0, m, seed=21), n, seed=22)
    edges = [(int(k) >> 32, int(k) & 0xFFFFFFFF) for k in keys]
    tau = len(exact.triangles(edges))
    assert tau > 0
    var = m * sum(exact.C_values(edges)) - tau * tau
    total = 0
    seeds = 10_000
    for seed in range(1, seeds + 1):
        s = nbsi_bulk.BulkStream(r, seed=seed)
        for W in synth.batches(keys, w):
            s.process_batch(W)
        total += m * s.closed_sum()
    mean = total / (seeds * r)
    se = math.sqrt(var / (seeds * r))
    assert abs(mean - tau) <= 4.5 * se, (mean, tau, se)
