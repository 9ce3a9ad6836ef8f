"""Step 4 (Lemma 3.1) through the C ABI: the exact N = |E| * S and the
double tau_hat = q + rem / r (q = N div r) of every estimate record -- the
synchronous tc_estimate, the device record of tc_estimate_async, and the
multi-stream forms -- equal the oracle's ``estimate.mean_estimate`` on the
same closed chis, bit for bit, including N beyond 64 bits.

Large N needs streams far longer than a test can run, so those cases load
a checkpoint blob (tc_load) whose state is written here: the loader checks
only that the stored S and closed count agree with the state, and the
estimate is then formed by the library from that state as after any batch.
"""
import random
import struct

import numpy as np
import pytest

import paper_1308_2166_gb300 as tc
import synth
from gpu_util import to_device
from oracle import estimate, nbsi_bulk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_2166_gb300 import build
    build.build()
    tc.load()


def _async_record(ctx):
    import torch
    d = torch.zeros(tc.ESTIMATE_BYTES // 8, dtype=torch.int64, device="cuda")
    tc.tc_estimate_async(ctx, d)
    torch.cuda.synchronize()
    (rec,) = tc.estimate_records(d.cpu())
    return rec


def _expected(m, chis, closed, r):
    S, N, tau = estimate.mean_estimate(m, [int(c) for c, k in zip(chis, closed) if k], r)
    return S, N, tau


def _blob(r, m, batches, chis, closed, seed=1, sid=0, vb=32):
    S = sum(int(c) for c, k in zip(chis, closed) if k)
    head = struct.pack("<16Q", 0x3145544154534354, 1, r, seed, sid, vb, m, batches,
                       S & (2**64 - 1), S >> 64, int(sum(closed)), 0, 0, 0, 0, 0)
    # a tuple the update can reach: f2 (adjacent to f1) exactly where chi > 0
    f1 = np.full(r, (1 << 32) | 2, dtype="<u8")
    ch = np.asarray(chis, dtype="<u8")
    f2 = np.where(ch > 0, np.uint64((1 << 32) | 3), np.uint64(2**64 - 1)).astype("<u8")
    fl = np.asarray(closed, dtype="<u4")
    return head + f1.tobytes() + f2.tobytes() + ch.tobytes() + fl.tobytes()


def test_estimate_matches_oracle_on_a_stream():
    keys = synth.tiny_chung_lu()
    r, seed = 1000, 9
    ctx = tc.tc_create_ex(r, seed, 0, 4096, 12)
    ref = nbsi_bulk.BulkStream(r, seed=seed, vertex_bits=12)
    try:
        for b in synth.batches(keys, 4096):
            tc.tc_process_batch(ctx, to_device(b))
            ref.process_batch(b)
            e = tc.tc_estimate(ctx)
            S, N, tau = _expected(ref.m, ref.c, ref.closed, r)
            assert (e["S"], e["N"], e["r"], e["m"]) == (S, N, r, ref.m)
            assert e["n_closed"] == int(ref.closed.sum()) and e["batches"] == ref.b
            assert e["tau_hat"] == tau            # the same double, bit for bit
            assert _async_record(ctx) == e
    finally:
        tc.tc_destroy(ctx)


def test_estimate_beyond_64_bits_from_a_loaded_state():
    rnd = random.Random(5)
    cases = [
        # N = 2^66, r = 3: q = (2^66 - 1) / 3, rem = 1
        (3, 1 << 32, [1 << 33, 1 << 33, 7], [1, 1, 0]),
        # |E| = 5, S = 1, r = 3: the 1 + fl(2/3) tie of the q + rem / r form
        (3, 5, [1, 0, 0], [1, 0, 0]),
        # S itself above 2^64 (three chis near 2^63)
        (5, 3, [2**63 + 11, 2**63 - 1, 2**63 + 5, 4, 9], [1, 1, 1, 0, 1]),
    ]
    for _ in range(40):
        r = rnd.choice([1, 2, 3, 7, 10, 97, 1000, 65537])
        m = rnd.choice([rnd.randint(1, 1000), rnd.randint(1, 2**40), rnd.randint(2**40, 2**50)])
        # chi <= 2 |E| as in any stream (|Gamma(f1)| counts later edges), which
        # keeps N = |E| * S below 2^128 here
        chis = [rnd.randint(0, min(2 * m, 2**rnd.choice([8, 30, 50]))) for _ in range(r)]
        # closed only with an f2, which needs chi >= 1
        closed = [c > 0 and rnd.random() < 0.6 for c in chis]
        cases.append((r, m, chis, closed))
    beyond = 0
    for r, m, chis, closed in cases:
        ctx = tc.tc_load(_blob(r, m, 3, chis, closed), 16)
        try:
            e = tc.tc_estimate(ctx)
            S, N, tau = _expected(m, chis, closed, r)
            beyond += N >= 2**64
            assert (e["S"], e["N"], e["m"], e["r"], e["batches"]) == (S, N, m, r, 3)
            assert e["tau_hat"] == tau, (r, m, N)
            assert _async_record(ctx) == e
        finally:
            tc.tc_destroy(ctx)
    assert beyond >= 10


def test_multi_estimate_records_match_oracle():
    import torch
    S = 5
    keys = synth.tiny_chung_lu()
    r = np.array([100, 1, 333, 64, 2000], dtype=np.uint64)
    seeds = np.arange(11, 11 + S, dtype=np.uint64)
    sids = np.arange(S, dtype=np.uint32)
    M = tc.MultiStream(r, seeds, sids, w_max_round=S * 1500, vertex_bits=12)
    refs = [nbsi_bulk.BulkStream(int(r[s]), seed=int(seeds[s]), stream=int(sids[s]),
                                 vertex_bits=12) for s in range(S)]
    try:
        for rnd in range(3):
            parts = [keys[(s * 3 + rnd) * 1500:(s * 3 + rnd + 1) * 1500] for s in range(S)]
            offs = np.concatenate([[0], np.cumsum([p.size for p in parts])]).astype(np.uint64)
            M.process_async(to_device(np.concatenate(parts)), offs)
            for s in range(S):
                refs[s].process_batch(parts[s])
        assert not M.sync().any()
        d = torch.zeros(S * tc.ESTIMATE_BYTES // 8, dtype=torch.int64, device="cuda")
        M.estimates_async(d)
        torch.cuda.synchronize()
        recs = tc.estimate_records(d.cpu())
        for s in range(S):
            ref = refs[s]
            Sx, N, tau = _expected(ref.m, ref.c, ref.closed, int(r[s]))
            e = M.estimate(s)
            assert (e["S"], e["N"], e["m"], e["tau_hat"]) == (Sx, N, ref.m, tau)
            assert recs[s] == e
    finally:
        M.close()
