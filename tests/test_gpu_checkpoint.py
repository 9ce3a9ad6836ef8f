"""Checkpoint / resume: a stream saved after some batches and loaded into a
new context continues bit for bit as if it had never stopped (the draws are
a function of seed, stream id, estimator, batch and slot), and a damaged
blob is refused."""
import numpy as np
import pytest

import paper_1308_2166_gb300 as tc
import synth
from gpu_util import assert_state_equal, to_device
from oracle import nbsi_bulk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_2166_gb300 import build
    build.build()
    tc.load()


@pytest.mark.parametrize("vertex_bits", [12, 32])
def test_resume_is_bit_exact(vertex_bits):
    keys = synth.tiny_chung_lu()
    parts = synth.batches(keys, 4096)
    r, seed, sid = 777, 2**40 + 3, 5
    whole = tc.tc_create_ex(r, seed, sid, 4096, vertex_bits)
    first = tc.tc_create_ex(r, seed, sid, 4096, vertex_bits)
    ref = nbsi_bulk.BulkStream(r, seed=seed, stream=sid, vertex_bits=vertex_bits)
    resumed = None
    try:
        for b in parts[:3]:
            tc.tc_process_batch(first, to_device(b))
        blob = tc.tc_save(first)
        assert len(blob) == 128 + 28 * r
        tc.tc_destroy(first)
        first = None
        resumed = tc.tc_load(blob, 4096)
        assert tc.tc_get_counters(resumed)[1:] == (3 * 4096, 3)
        for b in parts[3:]:
            tc.tc_process_batch(resumed, to_device(b))
        for b in parts:
            tc.tc_process_batch(whole, to_device(b))
            ref.process_batch(b)
        assert_state_equal(tc.tc_get_state(resumed), tc.tc_get_state(whole), "resumed vs whole")
        assert_state_equal(tc.tc_get_state(resumed), ref.state_arrays(), "resumed vs oracle")
        e1, e2 = tc.tc_estimate(resumed), tc.tc_estimate(whole)
        assert (e1["S"], e1["m"], e1["n_closed"], e1["batches"]) == \
               (e2["S"], e2["m"], e2["n_closed"], e2["batches"])
    finally:
        for c in (whole, first, resumed):
            if c:
                tc.tc_destroy(c)


def test_damaged_blob_is_refused():
    ctx = tc.tc_create_ex(64, 1, 0, 4096, 12)
    try:
        tc.tc_process_batch(ctx, to_device(synth.tiny_chung_lu()[:4096]))
        blob = bytearray(tc.tc_save(ctx))
    finally:
        tc.tc_destroy(ctx)
    for cut in (bytes(blob[:100]), bytes(blob[:-1])):
        with pytest.raises(tc.TcError) as e:
            tc.tc_load(cut, 4096)
        assert e.value.code == tc.TC_ERR_INVAL
    bad = bytearray(blob)
    bad[0] ^= 1                                     # magic
    with pytest.raises(tc.TcError):
        tc.tc_load(bytes(bad), 4096)
    bad = bytearray(blob)
    chi0 = 128 + 16 * 64
    bad[chi0:chi0 + 8] = (np.uint64(1 << 40)).tobytes()   # chi no longer sums to S
    flags = np.frombuffer(bytes(blob[128 + 24 * 64:]), dtype=np.uint32)
    if flags[0] & 1:
        with pytest.raises(tc.TcError):
            tc.tc_load(bytes(bad), 4096)
    bad = bytearray(blob)
    bad[128 + 24 * 64] |= 2                         # a flag bit that does not exist
    with pytest.raises(tc.TcError):
        tc.tc_load(bytes(bad), 4096)


def test_unreachable_tuples_are_refused():
    """A blob whose tuples the update cannot reach is refused before any of
    its vertex ids could index a directory."""
    r, B = 64, 12
    ctx = tc.tc_create_ex(r, 1, 0, 4096, B)
    try:
        tc.tc_process_batch(ctx, to_device(synth.tiny_chung_lu()[:4096]))
        blob = bytes(tc.tc_save(ctx))
    finally:
        tc.tc_destroy(ctx)
    f1 = np.frombuffer(blob[128:128 + 8 * r], dtype=np.uint64)
    f2 = np.frombuffer(blob[128 + 8 * r:128 + 16 * r], dtype=np.uint64)
    chi = np.frombuffer(blob[128 + 16 * r:128 + 24 * r], dtype=np.uint64)
    fl = np.frombuffer(blob[128 + 24 * r:], dtype=np.uint32)
    with_f2 = int(np.flatnonzero((f2 != tc.TC_EMPTY_EDGE) & (fl == 0))[0])
    without_f2 = np.flatnonzero(f2 == tc.TC_EMPTY_EDGE)

    def patched(i, f1v=None, f2v=None, chiv=None, flv=None):
        b = bytearray(blob)
        for off, arr, val, size in ((128, f1, f1v, 8), (128 + 8 * r, f2, f2v, 8),
                                    (128 + 16 * r, chi, chiv, 8), (128 + 24 * r, fl, flv, 4)):
            if val is not None:
                b[off + size * i:off + size * (i + 1)] = \
                    np.array([val], dtype=np.uint64 if size == 8 else np.uint32).tobytes()
        return bytes(b)

    u, v = int(f1[with_f2]) >> 32, int(f1[with_f2]) & 0xFFFFFFFF
    a, b = [x for x in range(4) if x not in (u, v)][:2]
    cases = [
        patched(with_f2, f1v=(u << 32) | (1 << B)),             # id beyond 2^B
        patched(with_f2, f1v=tc.TC_EMPTY_EDGE),                 # empty f1 once |E| > 0
        patched(with_f2, f1v=(5 << 32) | 3),                    # u > v
        patched(with_f2, f2v=int(f1[with_f2])),                 # f2 = f1
        patched(with_f2, f2v=(a << 32) | b),                    # f2 not adjacent to f1
        patched(with_f2, chiv=0),                               # f2 drawn from no neighbour
    ]
    if without_f2.size:
        i = int(without_f2[0])
        cases += [patched(i, chiv=3), patched(i, flv=1)]       # chi or closed without f2
    for bad in cases:
        with pytest.raises(tc.TcError) as e:
            tc.tc_load(bad, 4096)
        assert e.value.code == tc.TC_ERR_INVAL
    ok = tc.tc_load(blob, 4096)
    tc.tc_destroy(ok)
