"""Exact state distributions of the batched update by exhaustive enumeration.

Drives ``oracle.nbsi.Stream`` (one estimator) with every possible outcome of
every bounded draw, each outcome of U(n) weighted 1/n, batch by batch, and
merges equal states.  The result is the exact distribution of
(f1, f2, chi, closed) after the stream, as rational numbers, which the tests
compare with the Claim of Sec. 3.1 (Pr[(f1,f2) = (e,g)] = 1/(|E| |Gamma(e)|)),
Lemma 3.1 (E[X] = tau) and the edge-at-a-time estimator.
"""
from __future__ import annotations

from fractions import Fraction

from .nbsi import Estimator, Stream


class _Need(Exception):
    def __init__(self, n: int):
        super().__init__(n)
        self.n = n


class _ScriptDraws:
    """Replays a fixed list of draw outcomes; asks for a branch when empty."""

    def __init__(self, script):
        self.script = script
        self.k = 0

    def begin_batch(self, b: int) -> None:
        pass

    def U(self, i: int, purpose: int, n: int) -> int:
        if self.k < len(self.script):
            v, nn = self.script[self.k]
            assert nn == n, "replay diverged"
            self.k += 1
            return v
        raise _Need(n)


def _run_batch(state, m: int, b: int, W):
    """All (final_state, probability) outcomes of one batch from ``state``."""
    results = []
    stack = [([], Fraction(1))]
    while stack:
        script, p = stack.pop()
        s = Stream(1, draws=_ScriptDraws(script))
        s.m, s.b = m, b
        f1, f2, c, closed = state
        s.est[0] = Estimator(f1, f2, c, closed)
        try:
            s.process_batch(W)
        except _Need as need:
            for v in range(need.n):
                stack.append((script + [(v, need.n)], p / need.n))
            continue
        results.append((s.est[0].as_tuple(), p))
    return results


def distribution(batches) -> dict:
    """Exact distribution of one estimator's state after the given batches.

    ``batches`` is a list of lists of (u, v) edges with u < v.
    """
    dist = {(None, None, 0, False): Fraction(1)}
    m = 0
    b = 0
    for W in batches:
        W = [tuple(e) for e in W]
        if not W:
            continue
        nxt: dict = {}
        for state, p in dist.items():
            for st, q in _run_batch(state, m, b, W):
                nxt[st] = nxt.get(st, 0) + p * q
        dist = nxt
        m += len(W)
        b += 1
    return dist
