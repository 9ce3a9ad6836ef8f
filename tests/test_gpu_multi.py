"""Many streams in one round vs each stream alone (oracle and single-stream ABI).

Each stream's estimator state after every round must be bit-identical to the
CPU oracle run on that stream alone with the same seed, stream id and batch
boundaries, and to the single-stream library path; a rejected batch must
affect only its own stream.
"""
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


def _streams(S, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for s in range(S):
        n = int(rng.integers(64, 3000))
        m = int(min(n * rng.integers(2, 12), n * (n - 1) // 2))
        keys = synth.finish(synth.chung_lu(n, float(rng.uniform(2.1, 2.5)), 2.0 * m / n, m,
                                           seed=seed * 1000 + s), n, seed=seed * 1000 + s + 7)
        out.append(keys)
    return out


def _round(streams, cursors, sizes):
    parts, offs = [], [0]
    for s, keys in enumerate(streams):
        b = keys[cursors[s]:cursors[s] + sizes[s]]
        cursors[s] += b.size
        parts.append(b)
        offs.append(offs[-1] + b.size)
    cat = np.concatenate(parts) if offs[-1] else np.zeros(0, dtype=np.uint64)
    return cat, np.array(offs, dtype=np.uint64), parts


@pytest.mark.parametrize("S,vertex_bits", [(1, 12), (7, 12), (33, 20)])
def test_rounds_match_oracle_and_single_stream(S, vertex_bits):
    streams = _streams(S, seed=S)
    rng = np.random.default_rng(S + 100)
    r = rng.integers(1, 700, size=S)
    seeds = rng.integers(0, 2**63, size=S, dtype=np.uint64)
    sids = rng.integers(0, 2**32, size=S, dtype=np.uint64).astype(np.uint32)
    M = tc.MultiStream(r, seeds, sids, w_max_round=40000, vertex_bits=vertex_bits)
    refs = [nbsi_bulk.BulkStream(int(r[s]), seed=int(seeds[s]), stream=int(sids[s]),
                                 vertex_bits=vertex_bits) for s in range(S)]
    singles = [tc.tc_create_ex(int(r[s]), int(seeds[s]), int(sids[s]), 4096, vertex_bits)
               for s in range(S)]
    try:
        cur = [0] * S
        for rnd in range(6):
            sizes = [0 if rng.random() < 0.2 else int(rng.integers(1, 900)) for _ in range(S)]
            cat, offs, parts = _round(streams, cur, sizes)
            if offs[-1] == 0:
                continue
            if rnd % 3 == 1:
                M.process_ptrs_async([to_device(b) if b.size else None for b in parts])
            elif rnd % 3 == 2:
                dcat = to_device(cat)
                import torch
                torch.cuda.synchronize()          # in place before the pipelined call
                M.process_ready_async(dcat, offs)
            else:
                M.process_async(to_device(cat), offs)
            for s in range(S):
                if parts[s].size:
                    refs[s].process_batch(parts[s])
                    tc.tc_process_batch(singles[s], to_device(parts[s]))
            assert not M.sync().any()
            for s in range(S):
                exp = refs[s].state_arrays()
                assert_state_equal(M.state(s), exp, f"round {rnd} stream {s}")
                assert_state_equal(tc.tc_get_state(singles[s]), exp, f"single {s}")
                est = M.estimate(s)
                assert est["S"] == refs[s].closed_sum() and est["m"] == refs[s].m
                assert est["batches"] == refs[s].b
    finally:
        M.close()
        for c in singles:
            tc.tc_destroy(c)


def test_rejected_batch_affects_only_its_stream():
    streams = _streams(4, seed=9)
    r = [50, 60, 70, 80]
    M = tc.MultiStream(r, [1, 2, 3, 4], [0, 1, 2, 3], w_max_round=10000, vertex_bits=12)
    refs = [nbsi_bulk.BulkStream(r[s], seed=s + 1, stream=s, vertex_bits=12) for s in range(4)]
    try:
        cur = [0] * 4
        cat, offs, parts = _round(streams, cur, [100, 100, 100, 100])
        M.process_async(to_device(cat), offs)
        for s in range(4):
            refs[s].process_batch(parts[s])
        assert not M.sync().any()
        cat, offs, parts = _round(streams, cur, [50, 50, 50, 50])
        bad = parts[2].copy()
        bad[-1] = bad[0]                       # repeated edge inside stream 2's batch
        parts2 = [parts[0], parts[1], bad, parts[3]]
        M.process_async(to_device(np.concatenate(parts2)), offs)
        for s in (0, 1, 3):
            refs[s].process_batch(parts2[s])
        errs = M.sync()
        assert list(errs) == [0, 0, tc.TC_ERR_INPUT, 0]
        for s in range(4):
            assert_state_equal(M.state(s), refs[s].state_arrays(), f"stream {s}")
        assert M.counters(2)[2] == 1 and M.counters(0)[2] == 2
    finally:
        M.close()


def test_captured_round_replays_match_oracle():
    """One round captured as a CUDA graph, replayed with fresh batches."""
    import torch
    streams = _streams(5, seed=41)
    r = [300, 10, 1000, 77, 512]
    M = tc.MultiStream(r, [5, 6, 7, 8, 9], [9, 8, 7, 6, 5], w_max_round=5000, vertex_bits=12)
    refs = [nbsi_bulk.BulkStream(r[s], seed=5 + s, stream=9 - s, vertex_bits=12)
            for s in range(5)]
    sizes = [200, 50, 0, 120, 300]
    s_torch = torch.cuda.Stream()
    try:
        cur = [0] * 5
        cat, offs, parts = _round(streams, cur, sizes)
        buf = to_device(cat)
        M.capture(buf, offs, s_torch.cuda_stream)
        for rep in range(3):
            if rep:
                cat, offs2, parts = _round(streams, cur, sizes)
                assert list(offs2) == list(offs)
                with torch.cuda.stream(s_torch):
                    buf.copy_(to_device(cat))
            M.replay(s_torch.cuda_stream)
            s_torch.synchronize()
            for s in range(5):
                if parts[s].size:
                    refs[s].process_batch(parts[s])
            assert not M.sync().any()
            for s in range(5):
                assert_state_equal(M.state(s), refs[s].state_arrays(), f"replay {rep} stream {s}")
    finally:
        M.close()


def test_512_streams_sampled_against_oracle():
    """The batching configuration's scale: 512 streams of uneven length and
    estimator count (Chung-Lu, m log-uniform [1e3, 3e4], r log-uniform
    [2^6, 2^12], 21-bit ids as in the 512-stream bench), each cut into 8
    rounds of m_s // 8 edges, folded as CUDA-graph replays of one captured
    round.  A sample of 24 streams (the longest, the shortest, the most and
    fewest estimators, and random ones) must equal the oracle bit for bit
    after the last round, and every stream must equal its single-stream run
    and the engine's estimate records."""
    import torch
    S, T, VB = 512, 8, 21
    rng = np.random.default_rng(512)
    m = np.exp(rng.uniform(np.log(1e3), np.log(3e4), size=S)).astype(np.int64)
    r = np.exp(rng.uniform(np.log(2 ** 6), np.log(2 ** 12), size=S)).astype(np.uint64)
    seeds = rng.integers(1, 2**63, size=S, dtype=np.uint64)
    sids = np.arange(S, dtype=np.uint32)
    streams = []
    for s in range(S):
        n = max(64, int(m[s] // 8))
        g = float(rng.uniform(2.1, 2.5))
        streams.append(synth.finish(synth.chung_lu(n, g, 2.0 * m[s] / n, int(m[s]), seed=9000 + s),
                                    n, seed=19000 + s))
    ws = m // T
    offs = np.concatenate([[0], np.cumsum(ws)]).astype(np.uint64)
    rounds = [np.concatenate([streams[s][k * ws[s]:(k + 1) * ws[s]] for s in range(S)])
              for k in range(T)]
    M = tc.MultiStream(r, seeds, sids, w_max_round=int(offs[-1]), vertex_bits=VB)
    st = torch.cuda.Stream()
    try:
        buf = torch.empty(int(offs[-1]), dtype=torch.int64, device="cuda")
        M.capture(buf, offs, st.cuda_stream)
        for k in range(T):
            with torch.cuda.stream(st):
                buf.copy_(to_device(rounds[k]), non_blocking=True)
                M.replay(st.cuda_stream)
            st.synchronize()
        assert not M.sync().any()
        sample = {int(np.argmax(m)), int(np.argmin(m)), int(np.argmax(r)), int(np.argmin(r))}
        sample |= set(rng.choice(S, size=24 - len(sample), replace=False).tolist())
        for s in sorted(sample):
            ref = nbsi_bulk.BulkStream(int(r[s]), seed=int(seeds[s]), stream=int(sids[s]),
                                       vertex_bits=VB)
            for k in range(T):
                ref.process_batch(streams[s][k * ws[s]:(k + 1) * ws[s]])
            assert_state_equal(M.state(s), ref.state_arrays(), f"stream {s} vs oracle")
            e = M.estimate(s)
            assert e["S"] == ref.closed_sum() and e["m"] == ref.m == T * ws[s]
        d = torch.zeros(S * tc.ESTIMATE_BYTES // 8, dtype=torch.int64, device="cuda")
        M.estimates_async(d)
        torch.cuda.synchronize()
        recs = tc.estimate_records(d.cpu())
        for s in range(S):
            ctx = tc.tc_create_ex(int(r[s]), int(seeds[s]), int(sids[s]), int(ws[s]), VB)
            try:
                for k in range(T):
                    tc.tc_process_batch(ctx, to_device(streams[s][k * ws[s]:(k + 1) * ws[s]]))
                assert_state_equal(M.state(s), tc.tc_get_state(ctx), f"stream {s} vs alone")
                assert recs[s] == tc.tc_estimate(ctx)
            finally:
                tc.tc_destroy(ctx)
    finally:
        M.close()
