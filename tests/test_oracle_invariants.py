"""Oracle pins on Philox-driven runs.

* The two oracle forms (per-estimator ``nbsi`` and bulk-primitive
  ``nbsi_bulk``) give bit-identical states after every batch.
* NBSI (Invariant 3.1) holds for every estimator after every batch, checked
  by brute force against global arrival positions: f2 shares exactly one
  vertex with f1 and arrives after it; chi equals the brute-force count of
  later edges adjacent to f1; f2 is empty iff chi = 0; closed iff the closing
  edge exists and arrives after f2.
* Invalid batches raise and leave the state unchanged.
"""
import numpy as np
import pytest

import synth
from oracle import nbsi, nbsi_bulk


def _stream(n, m, seed):
    keys = synth.chung_lu(n, 2.3, 2.0 * m / n, m, seed=seed)
    return synth.finish(keys, n, seed=seed + 1)


def _check_nbsi(all_edges, state):
    pos = {int(k): i for i, k in enumerate(all_edges)}
    inc = {}
    for i, k in enumerate(all_edges):
        u, v = int(k) >> 32, int(k) & 0xFFFFFFFF
        inc.setdefault(u, []).append(i)
        inc.setdefault(v, []).append(i)
    f1s, f2s, cs, fls = state
    for f1, f2, c, fl in zip(f1s, f2s, cs, fls):
        f1, f2, c, fl = int(f1), int(f2), int(c), int(fl)
        assert f1 in pos
        u, v = f1 >> 32, f1 & 0xFFFFFFFF
        p1 = pos[f1]
        later = {j for j in inc[u] + inc[v] if j > p1}
        assert c == len(later)
        if f2 == nbsi.EMPTY_KEY:
            assert c == 0 and fl == 0
            continue
        assert f2 in pos and pos[f2] in later
        a, b = f2 >> 32, f2 & 0xFFFFFFFF
        shared = {u, v} & {a, b}
        assert len(shared) == 1
        x, y = sorted(({u, v} | {a, b}) - shared)
        g = (x << 32) | y
        assert bool(fl & 1) == (g in pos and pos[g] > pos[f2])


@pytest.mark.parametrize("n,m,w,r,seed", [(64, 300, 37, 50, 1), (200, 1500, 256, 64, 2),
                                          (50, 400, 1, 8, 3), (300, 2000, 2000, 33, 4)])
def test_scalar_equals_bulk_and_invariants(n, m, w, r, seed):
    E = _stream(n, m, seed)
    a = nbsi.Stream(r, seed=seed * 7 + 1, stream=seed)
    b = nbsi_bulk.BulkStream(r, seed=seed * 7 + 1, stream=seed)
    done = 0
    for W in synth.batches(E, w):
        a.process_batch(W)
        b.process_batch(W)
        done += W.size
        sa, sb = a.state_arrays(), b.state_arrays()
        for x, y in zip(sa, sb):
            assert [int(t) for t in x] == [int(t) for t in y]
        _check_nbsi(E[:done], sb)
        assert a.closed_sum() == b.closed_sum()
    assert a.m == b.m == m


def test_invalid_batches_rejected_without_state_change():
    E = _stream(64, 300, 9)
    for cls in (nbsi.Stream, nbsi_bulk.BulkStream):
        s = cls(16, seed=3)
        s.process_batch(E[:100])
        before = [list(map(int, x)) for x in s.state_arrays()]
        bad = [np.concatenate([E[100:110], E[105:106]]),            # repeat
               np.array([(5 << 32) | 5], dtype=np.uint64),          # self-loop
               np.array([(9 << 32) | 4], dtype=np.uint64)]          # not (min, max)
        for W in bad:
            with pytest.raises(ValueError):
                s.process_batch(W)
            assert [list(map(int, x)) for x in s.state_arrays()] == before
            assert s.m == 100 and s.b == 1
        s2 = cls(4, seed=3, vertex_bits=4)
        with pytest.raises(ValueError):
            s2.process_batch(np.array([(1 << 32) | 16], dtype=np.uint64))


def test_empty_batch_is_a_noop():
    s = nbsi_bulk.BulkStream(8, seed=1)
    s.process_batch(np.zeros(0, dtype=np.uint64))
    assert s.m == 0 and s.b == 0
