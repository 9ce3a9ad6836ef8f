"""Batched neighborhood-sampling update over whole arrays (oracle).

The same ``bulkUpdateAll`` as ``oracle.nbsi`` (Sec. 4), written the way the
paper describes its parallel algorithm: as a sequence of bulk primitives
(Sec. 3.2) over length-r and length-|W| arrays.  numpy's stable argsort
serves as ``sort`` and ``searchsorted`` as the multisearch of Lemma 3.3;
nothing is blocked, fused or reordered beyond the paper's own steps:

* Step 1 (Sec. 4.2): ``map`` randInt(|W|+|E|) -> idx, ``extract`` W[idx],
  ``combine`` into f1; chi <- 0 (and f2, f3 cleared) where replaced.
* Step 2 (Sec. 4.3): rankAll (Lemma 4.3: concat the two orientations, sort by
  src asc / pos desc, scan with resets for the rank); Q1 lookups for
  ld = rank(u->v), rd = rank(v->u); chi+ = ld + rd; one draw per estimator
  for the coin and phi; Q2 lookups (src, rank) -> arc; chi <- chi- + chi+.
* Step 3 (Sec. 4.4): ``edges`` = W as (src<dst, pos) sorted by (src, dst);
  exact multisearch of the candidate closing edge; closed iff present and
  after f2.

The readings of the paper's open points are those listed in ``oracle.nbsi``;
draws follow ``oracle.draws``.  The state layout matches the C ABI: f1/f2 as
packed uint64 (min<<32)|max with 2^64-1 for the empty edge, chi as uint64,
closed as a bool.

Pins: bit-identical to ``oracle.nbsi`` on random batches (whose own pins are
listed there), the worked example of Figs. 1-3, the NBSI invariants by brute
force.
"""
from __future__ import annotations

import numpy as np

from .draws import STEP1, STEP2, bounded_np

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
M32 = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)
NONE = np.int64(-1)


class BatchError(ValueError):
    """The batch violates the stream model (self-loop, id range, duplicate)."""


def validate(W: np.ndarray, vertex_bits: int = 32) -> None:
    u, v = W >> S32, W & M32
    if np.any(u == v):
        raise BatchError("self-loop")
    if np.any(u > v):
        raise BatchError("edge key not in (min, max) form")
    if vertex_bits < 32 and np.any(v >= np.uint64(1 << vertex_bits)):
        raise BatchError("vertex id out of range")
    if np.unique(W).size != W.size:
        raise BatchError("duplicate edge in batch")


def rank_all(W: np.ndarray):
    """rankAll(W), Lemma 4.3: arrays (src, dst, pos, rank) in sorted order.

    Sorted by src ascending, then pos descending; rank = position within the
    run of equal src (the scan with resets of App. B).
    """
    w = W.size
    u, v = W >> S32, W & M32
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    pos = np.concatenate([np.arange(w, dtype=np.int64)] * 2)
    order = np.lexsort((-pos, src))        # last key is the primary key
    src, dst, pos = src[order], dst[order], pos[order]
    n = src.size
    idx = np.arange(n, dtype=np.int64)
    head = np.ones(n, dtype=bool)
    head[1:] = src[1:] != src[:-1]
    seg_start = np.maximum.accumulate(np.where(head, idx, 0))
    rank = idx - seg_start
    return src, dst, pos, rank


class BulkStream:
    """r estimators of one stream, updated batch by batch (bulk oracle)."""

    def __init__(self, r: int, seed: int = 1, stream: int = 0,
                 vertex_bits: int = 32):
        if r < 1:
            raise ValueError("r >= 1")
        self.r = int(r)
        self.seed = int(seed)
        self.stream = int(stream)
        self.vertex_bits = vertex_bits
        self.m = 0
        self.b = 0
        self.f1 = np.full(r, EMPTY, dtype=np.uint64)
        self.f2 = np.full(r, EMPTY, dtype=np.uint64)
        self.c = np.zeros(r, dtype=np.uint64)
        self.closed = np.zeros(r, dtype=bool)

    def process_batch(self, W) -> None:
        W = np.ascontiguousarray(W, dtype=np.uint64)
        validate(W, self.vertex_bits)
        w = W.size
        if w == 0:
            return
        r, m, b = self.r, self.m, self.b
        est = np.arange(r, dtype=np.uint64)

        # ---- Step 1 (Sec. 4.2): map randInt(|W|+|E|), extract, combine
        x = bounded_np(self.seed, self.stream, est, b, STEP1,
                       np.full(r, m + w, dtype=np.uint64))
        rep = x >= np.uint64(m)
        p1 = np.where(rep, x.astype(np.int64) - m, NONE)
        self.f1[rep] = W[p1[rep]]
        self.c[rep] = 0
        self.f2[rep] = EMPTY
        self.closed[rep] = False

        # ---- Step 2 (Sec. 4.3): rankAll, Q1 for ld/rd, coin + phi, Q2
        src, dst, pos, rank = rank_all(W)
        # rank of each batch edge's two arcs, indexed by pos ("extract")
        u_w = W >> S32
        from_u = src == u_w[pos]
        rank_u = np.empty(w, dtype=np.int64)
        rank_v = np.empty(w, dtype=np.int64)
        rank_u[pos[from_u]] = rank[from_u]
        rank_v[pos[~from_u]] = rank[~from_u]

        fu, fv = self.f1 >> S32, self.f1 & M32
        lo_u = np.searchsorted(src, fu, side="left")
        hi_u = np.searchsorted(src, fu, side="right")
        lo_v = np.searchsorted(src, fv, side="left")
        hi_v = np.searchsorted(src, fv, side="right")
        ld = np.where(rep, 0, hi_u - lo_u).astype(np.int64)
        rd = np.where(rep, 0, hi_v - lo_v).astype(np.int64)
        ld[rep] = rank_u[p1[rep]]
        rd[rep] = rank_v[p1[rep]]
        chi_minus = self.c.copy()
        chi_plus = (ld + rd).astype(np.uint64)

        drawn = chi_plus > 0
        y = np.zeros(r, dtype=np.uint64)
        y[drawn] = bounded_np(self.seed, self.stream, est[drawn], b, STEP2,
                              chi_minus[drawn] + chi_plus[drawn])
        take = drawn & (y >= chi_minus)
        phi = (y - chi_minus).astype(np.int64)      # meaningful where take
        on_u = take & (phi < ld)
        on_v = take & ~(phi < ld)
        arc = np.full(r, -1, dtype=np.int64)
        arc[on_u] = lo_u[on_u] + phi[on_u]
        arc[on_v] = lo_v[on_v] + (phi[on_v] - ld[on_v])
        p2 = np.full(r, NONE, dtype=np.int64)
        p2[take] = pos[arc[take]]
        self.f2[take] = W[p2[take]]
        self.closed[take] = False
        self.c = chi_minus + chi_plus

        # ---- Step 3 (Sec. 4.4): multisearch of the closing edge in `edges`
        order = np.argsort(W, kind="stable")      # (src, dst) order of keys
        ekeys = W[order]
        epos = order.astype(np.int64)
        chk = (self.f2 != EMPTY) & ~self.closed
        a1, b1 = self.f1 >> S32, self.f1 & M32
        a2, b2 = self.f2 >> S32, self.f2 & M32
        # shared vertex s; g = {f1 \ s, f2 \ s}
        x1 = np.where((a1 == a2) | (a1 == b2), b1, a1)
        x2 = np.where((a2 == a1) | (a2 == b1), b2, a2)
        g = (np.minimum(x1, x2) << S32) | np.maximum(x1, x2)
        at = np.searchsorted(ekeys, g)
        at_c = np.minimum(at, w - 1)
        found = chk & (at < w) & (ekeys[at_c] == g)
        q = np.where(found, epos[at_c], NONE)
        after = (p2 == NONE) | (q > p2)
        self.closed |= found & after

        self.m += w
        self.b += 1

    def state_arrays(self):
        fl = self.closed.astype(np.uint32)
        return self.f1.copy(), self.f2.copy(), self.c.copy(), fl

    def closed_sum(self) -> int:
        return int(sum(int(x) for x in self.c[self.closed]))
