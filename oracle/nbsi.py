"""Batched neighborhood-sampling update, one estimator at a time (oracle).

Follows Sec. 4 of the paper ("bulkUpdateAll"): each estimator holds the tuple
(f1, f2, f3, chi) of Invariant 3.1 (NBSI); a batch W = <w_0 .. w_{s-1}> is
folded in by

* Step 1 (Sec. 4.2): reservoir choice of the level-1 edge -- with probability
  |W|/(|W|+|E|) replace f1 by a uniform edge of W, and reset chi to 0;
* Step 2 (Sec. 4.3): chi- = chi, chi+ = rank(u->v) + rank(v->u) computed
  from rankAll(W) (Lemma 4.3, Def. 4.2); keep f2 with probability
  chi-/(chi- + chi+), else take the level-2 edge named by phi in [0, chi+)
  under the naming system (Observation and Fig. 3); chi <- chi- + chi+;
* Step 3 (Sec. 4.4): look the closing edge up in ``edges`` (W sorted by
  (src, dst)) and keep it if it arrives after f2.

The paper leaves some points open; the readings taken here (and on the CUDA
side) are:

1. x = randInt(|W|+|E|) replaces iff x >= |E|, taking W[x - |E|].
2. Step 2 uses one draw y = U(chi- + chi+): keep iff y < chi-, else
   phi = y - chi-; no draw when chi+ = 0.
3. In the naming system u is the smaller vertex id of f1.
4. An old f1 gets rank(u->v) = deg_W(u) (Def. 4.2 for pairs not in W; the
   footnote to Sec. 4.3 calls this "the largest rank", but the definition
   gives the largest rank plus one, and the definition is what makes chi+
   the size of the W-neighbourhood).
5. Replacing f1 also clears f2 and f3 (NBSI item 3 forces it: the new f2
   must come after the new f1).
6. Replacing f2 clears f3; Step 3 then re-checks within the same batch.
7. Positions are 0-based indices into the batch; batches are totally
   ordered by arrival.

Draws come from an injectable source with ``begin_batch(b)`` and
``U(i, purpose, n)``; ``draws.PhiloxDraws`` is the production one and
``enumerate`` drives the same code with every possible outcome.

Pins: the worked example of Figs. 1-3 (tests/golden/), exact distributions
against the Claim of Sec. 3.1 and Lemma 3.1 by exhaustive enumeration,
distributional equality with the edge-at-a-time estimator, the NBSI
invariants checked by brute force, and an unbiasedness test over 10^4 seeds.
"""
from __future__ import annotations

from dataclasses import dataclass

from .draws import STEP1, STEP2, PhiloxDraws

EMPTY_KEY = (1 << 64) - 1
MASK32 = 0xFFFFFFFF


class BatchError(ValueError):
    """The batch violates the stream model (self-loop, id range, duplicate)."""


def pack(u: int, v: int) -> int:
    """Packed edge key (min << 32) | max."""
    a, b = (u, v) if u < v else (v, u)
    return (a << 32) | b


def unpack(key: int):
    return key >> 32, key & MASK32


@dataclass
class Estimator:
    f1: tuple | None = None   # level-1 edge (u, v), u < v
    f2: tuple | None = None   # level-2 edge
    c: int = 0                # chi = |Gamma(f1)|
    closed: bool = False      # f3 present (closing edge seen after f2)

    def as_tuple(self):
        return (self.f1, self.f2, self.c, self.closed)


def validate_batch(W, vertex_bits: int = 32):
    """Check the stream model of Sec. 2: simple graph, each edge once.

    Returns the batch as a list of (u, v) with u < v.  Raises BatchError on a
    self-loop, an id outside [0, 2^vertex_bits) or an edge repeated inside
    the batch.  (Repeats across batches are the caller's contract.)
    """
    out = []
    seen = set()
    lim = 1 << vertex_bits
    for e in W:
        if isinstance(e, tuple):
            u, v = e
        else:
            u, v = unpack(int(e))
        if u == v:
            raise BatchError("self-loop")
        if not (u < v):
            raise BatchError("edge key not in (min, max) form")
        if v >= lim:
            raise BatchError("vertex id out of range")
        if (u, v) in seen:
            raise BatchError("duplicate edge in batch")
        seen.add((u, v))
        out.append((u, v))
    return out


def rank_all(W):
    """rankAll(W) of Lemma 4.3.

    Forms the 2|W| arcs (src, dst, pos), one per orientation of each batch
    edge, sorts them by src ascending and pos descending, and assigns each
    arc its rank: 0 for the first arc of a src, else one more than the arc
    before it (the scan with resets of App. B).  Returns a list of dicts
    with keys src, dst, pos, rank in the sorted order.
    """
    arcs = []
    for pos, (u, v) in enumerate(W):
        arcs.append((u, v, pos))
        arcs.append((v, u, pos))
    arcs.sort(key=lambda a: (a[0], -a[2]))
    out = []
    prev_src = None
    run = 0
    for src, dst, pos in arcs:
        run = run + 1 if src == prev_src else 0
        prev_src = src
        out.append({"src": src, "dst": dst, "pos": pos, "rank": run})
    return out


class RankTable:
    """Lookups over rankAll(W): Def. 4.2 ranks, Q1 and Q2 of Sec. 4.3."""

    def __init__(self, W):
        self.W = W
        self.F = rank_all(W)
        self.by_src_pos = {}
        self.by_src_rank = {}
        self.deg = {}
        for a in self.F:
            self.by_src_pos[(a["src"], a["pos"])] = a
            self.by_src_rank[(a["src"], a["rank"])] = a
            self.deg[a["src"]] = self.deg.get(a["src"], 0) + 1

    def rank(self, x: int, y: int) -> int:
        """rank(x -> y), Def. 4.2."""
        e = (min(x, y), max(x, y))
        try:
            i = self.W.index(e)
        except ValueError:
            return self.deg.get(x, 0)
        return self.by_src_pos[(x, i)]["rank"]

    def rank_at(self, x: int, pos: int) -> int:
        """rank of the arc from x of the batch edge at ``pos`` (Q1)."""
        return self.by_src_pos[(x, pos)]["rank"]

    def arc_of(self, src: int, rank: int):
        """The arc with the given src and rank (Q2)."""
        return self.by_src_rank[(src, rank)]

    def name(self, u: int, v: int, phi: int):
        """Naming system of Sec. 4.3: phi -> arc of Gamma_W(f1), f1 = {u, v}.

        phi < rank(u->v) names (src=u, rank=phi); otherwise
        (src=v, rank=phi-rank(u->v)).
        """
        ld = self.rank(u, v)
        if phi < ld:
            return self.arc_of(u, phi)
        return self.arc_of(v, phi - ld)


def closing_edge(f1, f2):
    """The edge that closes the wedge (f1, f2), packed as (min, max)."""
    s = set(f1) & set(f2)
    if len(s) != 1:
        raise AssertionError("level-2 edge not adjacent to level-1 edge")
    (x,) = set(f1) - s
    (y,) = set(f2) - s
    return (min(x, y), max(x, y))


class Stream:
    """One stream of r estimators under bulk updates (scalar oracle)."""

    def __init__(self, r: int, seed: int = 1, stream: int = 0, draws=None,
                 vertex_bits: int = 32):
        if r < 1:
            raise ValueError("r >= 1")
        self.r = r
        self.seed = seed
        self.stream = stream
        self.vertex_bits = vertex_bits
        self.m = 0          # |E|: edges before the next batch
        self.b = 0          # batches processed
        self.est = [Estimator() for _ in range(r)]
        self.draws = draws if draws is not None else PhiloxDraws(seed, stream)

    def process_batch(self, W) -> None:
        W = validate_batch(W, self.vertex_bits)
        w = len(W)
        if w == 0:
            return
        self.draws.begin_batch(self.b)
        m = self.m
        ranks = RankTable(W)
        # Step 3's sorted edge list: (src < dst, pos) sorted by (src, dst).
        edges = sorted((u, v, pos) for pos, (u, v) in enumerate(W))
        edge_pos = {(u, v): pos for u, v, pos in edges}
        for i, e in enumerate(self.est):
            # -- Step 1: level-1 reservoir over E u W (Sec. 4.2)
            x = self.draws.U(i, STEP1, m + w)
            p1 = None
            if x >= m:
                p1 = x - m
                e.f1 = W[p1]
                e.c = 0
                e.f2 = None
                e.closed = False
            # -- Step 2: chi+, coin and level-2 rank-select (Sec. 4.3)
            u, v = e.f1
            if p1 is None:
                ld, rd = ranks.deg.get(u, 0), ranks.deg.get(v, 0)
            else:
                ld, rd = ranks.rank_at(u, p1), ranks.rank_at(v, p1)
            chi_minus = e.c
            chi_plus = ld + rd
            p2 = None
            if chi_plus > 0:
                y = self.draws.U(i, STEP2, chi_minus + chi_plus)
                if y >= chi_minus:
                    phi = y - chi_minus
                    if phi < ld:
                        arc = ranks.arc_of(u, phi)
                    else:
                        arc = ranks.arc_of(v, phi - ld)
                    p2 = arc["pos"]
                    e.f2 = W[p2]
                    e.closed = False
            e.c = chi_minus + chi_plus
            # -- Step 3: closing edge after f2 (Sec. 4.4)
            if e.f2 is not None and not e.closed:
                g = closing_edge(e.f1, e.f2)
                q = edge_pos.get(g)
                if q is not None and (p2 is None or q > p2):
                    e.closed = True
        self.m += w
        self.b += 1

    # -- views ---------------------------------------------------------------
    def state_arrays(self):
        """(f1, f2, c, flags) as lists in the C-ABI layout.

        f1/f2 packed (min<<32)|max or 2^64-1 for the empty edge; flags bit 0
        is the closed bit.
        """
        f1 = [pack(*e.f1) if e.f1 else EMPTY_KEY for e in self.est]
        f2 = [pack(*e.f2) if e.f2 else EMPTY_KEY for e in self.est]
        c = [e.c for e in self.est]
        fl = [1 if e.closed else 0 for e in self.est]
        return f1, f2, c, fl

    def closed_sum(self) -> int:
        """S = sum of chi over estimators whose wedge is closed."""
        return sum(e.c for e in self.est if e.closed)
