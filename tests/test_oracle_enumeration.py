"""Oracle pins by exhaustive enumeration with exact rational probabilities.

* Claim of Sec. 3.1 / NBSI (Invariant 3.1): after the stream, f1 is uniform
  on E, chi = |Gamma(f1)|, f2 is uniform on Gamma(f1) (or empty when that is
  empty), and the wedge is closed iff its closing edge arrives after f2.
* Lemma 3.1: E[X] = tau with X = chi * |E| when closed, else 0.
* Second moment from the Claim: E[X^2] = sum_t (m C(t))^2 / (m C(t))
  = m * sum_t C(t), so Var[X] = m * sum_t C(t) - tau^2.
* Any split of the stream into batches gives exactly the distribution of the
  edge-at-a-time estimator (an independent formulation, oracle.sequential).
"""
import itertools
import random
from fractions import Fraction

import pytest

from oracle import enumerate as en
from oracle import exact, sequential

TRI_PENDANT = [(0, 1), (1, 2), (0, 2), (2, 3)]
K4 = [(0, 1), (2, 3), (0, 2), (1, 3), (0, 3), (1, 2)]
BOWTIE = [(0, 1), (1, 2), (3, 4), (0, 2), (2, 3), (2, 4), (1, 3)]


def _random_graph(seed, n=6, m=9):
    rnd = random.Random(seed)
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    rnd.shuffle(pairs)
    return pairs[:m]


def _compositions(m):
    for cuts in itertools.product([0, 1], repeat=m - 1):
        sizes, run = [], 1
        for c in cuts:
            if c:
                sizes.append(run)
                run = 1
            else:
                run += 1
        sizes.append(run)
        yield sizes


def _split(edges, sizes):
    out, i = [], 0
    for s in sizes:
        out.append(edges[i:i + s])
        i += s
    return out


def _check_claim(edges, dist):
    m = len(edges)
    pos = {e: i for i, e in enumerate(edges)}
    assert sum(dist.values()) == 1
    for e in edges:
        gam = exact.gamma(edges, e)
        states = {s: p for s, p in dist.items() if s[0] == e}
        assert sum(states.values()) == Fraction(1, m)
        for (f1, f2, c, closed), p in states.items():
            assert c == len(gam)
            if not gam:
                assert f2 is None and not closed
                continue
            assert f2 in gam
            assert p == Fraction(1, m * len(gam))
            s_shared = set(f1) & set(f2)
            g = tuple(sorted((set(f1) | set(f2)) - s_shared))
            expect = g in pos and pos[g] > pos[f2]
            assert closed == expect


def _moments(edges, dist):
    m = len(edges)
    ex = sum(p * (c * m if closed else 0) for (f1, f2, c, closed), p in dist.items())
    ex2 = sum(p * (c * m if closed else 0) ** 2 for (f1, f2, c, closed), p in dist.items())
    return ex, ex2 - ex * ex


@pytest.mark.parametrize("edges", [TRI_PENDANT, K4, BOWTIE, _random_graph(3), _random_graph(8)])
def test_claim_and_lemma_one_batch_and_singletons(edges):
    tau = len(exact.triangles(edges))
    Cs = exact.C_values(edges)
    var_closed = len(edges) * sum(Cs) - tau * tau
    seq = sequential.distribution(edges)
    for sizes in ([len(edges)], [1] * len(edges), [2] * (len(edges) // 2) + [len(edges) % 2]):
        sizes = [s for s in sizes if s]
        dist = en.distribution(_split(edges, sizes))
        _check_claim(edges, dist)
        ex, var = _moments(edges, dist)
        assert ex == tau
        assert var == var_closed
        assert dist == seq


def test_every_batch_split_matches_sequential():
    edges = _random_graph(11, n=5, m=7)
    seq = sequential.distribution(edges)
    _check_claim(edges, seq)
    for sizes in _compositions(len(edges)):
        assert en.distribution(_split(edges, sizes)) == seq, sizes


def test_sequential_estimator_obeys_claim():
    for seed in range(4):
        edges = _random_graph(100 + seed, n=6, m=10)
        dist = sequential.distribution(edges)
        _check_claim(edges, dist)
        ex, _ = _moments(edges, dist)
        assert ex == len(exact.triangles(edges))
