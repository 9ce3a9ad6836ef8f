"""Edge-at-a-time neighborhood sampling (batch size one), exact distribution.

Sec. 4.2 notes that with |W| = 1 Step 1 is plain reservoir sampling; Sec. 3.1
(Invariant 3.1) describes the state the sequential estimator of Pavan et al.
maintains.  This module restates that estimator as its own per-edge rule,
independently of ``oracle.nbsi`` (no shared code), and propagates its exact
state distribution with rational probabilities:

on the t-th edge e (t = 1, 2, ...):
  * with probability 1/t: f1 <- e, chi <- 0, f2 <- none, f3 <- none;
  * otherwise, if e shares a vertex with f1: chi <- chi + 1, and with
    probability 1/chi f2 <- e, f3 <- none; if f2 was not replaced and e is
    the edge closing the wedge (f1, f2), f3 <- e.

Used as a pin: the batched update must produce exactly this distribution of
(f1, f2, chi, closed) for every split of the stream into batches.
"""
from __future__ import annotations

from fractions import Fraction


def _closes(f1, f2, e) -> bool:
    a = set(f1) ^ set(f2)          # the two endpoints not shared
    return len(a) == 2 and set(e) == a


def step(dist: dict, e, t: int) -> dict:
    """Advance a distribution {(f1, f2, chi, closed): prob} by edge e (t-th)."""
    out: dict = {}

    def add(s, p):
        out[s] = out.get(s, 0) + p

    p_new = Fraction(1, t)
    for (f1, f2, chi, closed), p in dist.items():
        add((e, None, 0, False), p * p_new)
        q = p * (1 - p_new)
        if q == 0:
            continue
        if f1 is not None and len(set(f1) & set(e)) == 1:
            chi2 = chi + 1
            add((f1, e, chi2, False), q * Fraction(1, chi2))
            keep = q * (1 - Fraction(1, chi2))
            if keep:
                cl = closed or (f2 is not None and _closes(f1, f2, e))
                add((f1, f2, chi2, cl), keep)
        else:
            add((f1, f2, chi, closed), q)
    return out


def distribution(edges) -> dict:
    """Exact state distribution after the whole edge sequence."""
    dist = {(None, None, 0, False): Fraction(1)}
    for t, e in enumerate(edges, start=1):
        dist = step(dist, tuple(e), t)
    return dist
