"""Pins for the exact triangle counters (closed forms and cross-checks)."""
import itertools
import math
import random

import numpy as np

import synth
from oracle import exact


def _keys(edges):
    return np.array([(min(a, b) << 32) | max(a, b) for a, b in edges], dtype=np.uint64)


def test_closed_forms():
    for n in range(3, 12):
        kn = list(itertools.combinations(range(n), 2))
        assert exact.count(_keys(kn)) == math.comb(n, 3)
        assert len(exact.triangles(kn)) == math.comb(n, 3)
    # complete bipartite graphs have no triangle
    kab = [(a, 10 + b) for a in range(6) for b in range(7)]
    assert exact.count(_keys(kab)) == 0
    # wheel: hub 0 joined to a k-cycle has k triangles (k >= 4)
    for k in range(4, 15):
        cyc = [(1 + i, 1 + (i + 1) % k) for i in range(k)]
        assert exact.count(_keys(cyc + [(0, 1 + i) for i in range(k)])) == k


def test_counters_agree_on_random_graphs():
    for seed in range(6):
        rnd = random.Random(seed)
        n = rnd.randint(8, 30)
        pairs = [p for p in itertools.combinations(range(n), 2) if rnd.random() < 0.3]
        k = _keys(pairs)
        t = len(exact.triangles(pairs))
        assert exact.count(k, n) == t
        assert exact.count_dense(k, n) == t


def test_forward_matches_dense_on_chung_lu():
    keys = synth.finish(synth.chung_lu(2000, 2.3, 12.0, None, seed=4), 2000, seed=5)
    assert exact.count(keys, 2000) == exact.count_dense(keys, 2000)
