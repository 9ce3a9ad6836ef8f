"""The request server: every result the same alone and in the mix.

Streams are opened, fed batches and queried through tc_server in a random
interleaving, with fewer stream slots than streams (opens wait for closes)
and, in one test, a memory budget that holds only a few streams' state.
Every batch and query completion must carry exactly the estimate of the same
stream run alone through the single-stream path (same seed, stream id and
batch boundaries), and a sample of streams is checked against the oracle.
"""
import numpy as np
import pytest

import paper_1308_2166_gb300 as tc
import synth
from gpu_util import to_device
from oracle import nbsi_bulk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_2166_gb300 import build
    build.build()
    tc.load()


def _graph(seed, n_lo=64, n_hi=3000):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(n_lo, n_hi))
    m = int(min(n * rng.integers(2, 12), n * (n - 1) // 2))
    return synth.finish(synth.chung_lu(n, float(rng.uniform(2.1, 2.5)), 2.0 * m / n, m,
                                       seed=seed), n, seed=seed + 7)


def _plan(rng, keys, n_ops, q_frac=0.1, max_w=900):
    """A stream's requests after its open: ('b', edges) or ('q',), then close."""
    ops, cur = [], 0
    for _ in range(n_ops):
        if rng.random() < q_frac or cur >= keys.size:
            ops.append(("q",))
        else:
            w = int(rng.integers(1, max_w))
            ops.append(("b", keys[cur:cur + w].copy()))
            cur += w
    ops.append(("c",))
    return ops


def _run_mix(srv, specs, plans, rng):
    """Submit every stream's open + plan in a random interleaving; return
    {ticket: (stream, op index)} and all completions keyed by ticket."""
    left = {s: 0 for s in range(len(specs))}
    handles, where = {}, {}
    order = []
    for s, (r, seed, sid) in enumerate(specs):
        order += [s] * (len(plans[s]) + 1)
    rng.shuffle(order)
    done = {}
    for s in order:
        k = left[s]
        left[s] += 1
        if k == 0:
            h, t = srv.open(*specs[s])
            handles[s] = h
            where[t] = (s, -1)
        else:
            op = plans[s][k - 1]
            if op[0] == "b":
                t = srv.submit(handles[s], op[1])
            elif op[0] == "q":
                t = srv.query(handles[s])
            else:
                t = srv.close(handles[s])
            where[t] = (s, k - 1)
        for c in srv.poll():
            done[int(c["ticket"])] = c
    srv.drain(120000)
    for c in srv.poll():
        done[int(c["ticket"])] = c
    while True:
        more = srv.poll(wait_us=1000)
        if more.size == 0:
            break
        for c in more:
            done[int(c["ticket"])] = c
    return where, done


def _run_mix_many(srv, specs, plans, rng, chunk=7):
    """As _run_mix, but batches and queries go in chunks through
    tc_server_submit_many (opens and closes flush the chunk first)."""
    left = {s: 0 for s in range(len(specs))}
    handles, where = {}, {}
    order = []
    for s, (r, seed, sid) in enumerate(specs):
        order += [s] * (len(plans[s]) + 1)
    rng.shuffle(order)
    done = {}
    pend = []   # (stream, op index, kind, handle, ptr, w)

    def flush():
        if not pend:
            return
        t = srv.submit_many([p[2] for p in pend], [p[3] for p in pend],
                            [p[4] for p in pend], [p[5] for p in pend])
        for (s, i, *_), tk in zip(pend, t):
            where[int(tk)] = (s, i)
        pend.clear()

    for s in order:
        k = left[s]
        left[s] += 1
        if k == 0:
            flush()
            h, t = srv.open(*specs[s])
            handles[s] = h
            where[t] = (s, -1)
            continue
        op = plans[s][k - 1]
        if op[0] == "b":
            pend.append((s, k - 1, tc.TC_REQ_BATCH, handles[s], op[1].ctypes.data, op[1].size))
        elif op[0] == "q":
            pend.append((s, k - 1, tc.TC_REQ_QUERY, handles[s], 0, 0))
        else:
            flush()
            where[srv.close(handles[s])] = (s, k - 1)
        if len(pend) >= chunk:
            flush()
        for c in srv.poll():
            done[int(c["ticket"])] = c
    flush()
    srv.drain(120000)
    while True:
        more = srv.poll(wait_us=1000)
        if more.size == 0:
            break
        for c in more:
            done[int(c["ticket"])] = c
    return where, done


def _alone(spec, plan, vertex_bits, bad=()):
    """Expected (batches, S, closed, m, N, tau_hat) after each op of the plan,
    alone."""
    r, seed, sid = spec
    ctx = tc.tc_create_ex(r, seed, sid, 4096, vertex_bits)
    out = []
    try:
        for i, op in enumerate(plan):
            if op[0] == "b" and i not in bad:
                tc.tc_process_batch(ctx, to_device(op[1]))
            e = tc.tc_estimate(ctx)
            out.append((e["batches"], e["S"], e["n_closed"], e["m"], e["N"], e["tau_hat"]))
    finally:
        tc.tc_destroy(ctx)
    return out


def _check(where, done, specs, plans, vertex_bits, bad=None):
    bad = bad or {}
    assert len(done) == len(where), "every request completes exactly once"
    expect = {s: _alone(specs[s], plans[s], vertex_bits, bad.get(s, ())) for s in range(len(specs))}
    for t, (s, i) in where.items():
        c = done[t]
        assert c["t_submit_ns"] <= c["t_admit_ns"] <= c["t_done_ns"]
        if i < 0:
            assert c["kind"] == tc.TC_REQ_OPEN and c["status"] == tc.TC_OK
            continue
        op = plans[s][i]
        if op[0] == "c":
            assert c["kind"] == tc.TC_REQ_CLOSE and c["status"] == tc.TC_OK
            continue
        if i in bad.get(s, ()):
            assert c["status"] == tc.TC_ERR_INPUT, (s, i)
        else:
            assert c["status"] == tc.TC_OK, (s, i, c["status"])
        got = (int(c["batches"]), int(c["sum_lo"]) | (int(c["sum_hi"]) << 64),
               int(c["n_closed"]), int(c["m"]), int(c["num_lo"]) | (int(c["num_hi"]) << 64),
               float(c["tau_hat"]))
        # (a rejected batch reports the unchanged stream: the alone run skips it)
        assert got == expect[s][i], (s, i, got, expect[s][i])


@pytest.mark.parametrize("depth", [1, 0], ids=["depth1", "default_depth2"])
def test_mix_equals_alone_with_slot_waits(depth):
    rng = np.random.default_rng(5)
    n_streams = 24
    specs, plans = [], []
    for s in range(n_streams):
        keys = _graph(1000 + s)
        specs.append((int(rng.integers(1, 700)), int(rng.integers(0, 2**63)),
                      int(rng.integers(0, 2**32))))
        plans.append(_plan(rng, keys, int(rng.integers(3, 14))))
    srv = tc.Server(max_streams=8, vertex_bits=12, budget_bytes=2 << 30, w_max_round=4096,
                    depth=depth)
    try:
        where, done = _run_mix(srv, specs, plans, rng)
        st = srv.stats()
    finally:
        srv.destroy()
    _check(where, done, specs, plans, 12)
    assert st["opens"] == n_streams and st["closes"] == n_streams
    assert st["streams_open"] == 0 and st["max_round_streams"] <= 8
    assert st["queries"] == sum(op[0] == "q" for p in plans for op in p)
    # the oracle agrees with the alone runs on a sample of streams
    for s in (0, 7, 19):
        r, seed, sid = specs[s]
        ref = nbsi_bulk.BulkStream(r, seed=seed, stream=sid, vertex_bits=12)
        exp = _alone(specs[s], plans[s], 12)
        for i, op in enumerate(plans[s]):
            if op[0] == "b":
                ref.process_batch(op[1])
            if op[0] != "c":
                assert exp[i][1] == ref.closed_sum() and exp[i][3] == ref.m


def test_submit_many_equals_alone():
    """The same kind of mix with batches and queries submitted in chunks."""
    rng = np.random.default_rng(15)
    specs, plans = [], []
    for s in range(16):
        keys = _graph(2000 + s)
        specs.append((int(rng.integers(1, 700)), int(rng.integers(0, 2**63)),
                      int(rng.integers(0, 2**32))))
        plans.append(_plan(rng, keys, int(rng.integers(3, 14))))
    srv = tc.Server(max_streams=6, vertex_bits=12, budget_bytes=2 << 30, w_max_round=4096,
                    depth=2)
    try:
        where, done = _run_mix_many(srv, specs, plans, rng)
        # an unknown handle or another kind fails the whole call
        with pytest.raises(tc.TcError):
            srv.submit_many([tc.TC_REQ_QUERY, tc.TC_REQ_QUERY], [0, 0xFFFFFF], [0, 0], [0, 0])
        with pytest.raises(tc.TcError):
            srv.submit_many([tc.TC_REQ_OPEN], [0], [0], [0])
        st = srv.stats()
    finally:
        srv.destroy()
    _check(where, done, specs, plans, 12)
    assert st["opens"] == 16 and st["closes"] == 16


def test_memory_budget_limits_admission():
    """Budget for the fixed scratch plus about three streams' state: opens
    and batches wait, the reserved bytes never pass the budget, and every
    result is still the stream's alone result."""
    rng = np.random.default_rng(11)
    probe = tc.Server(max_streams=16, vertex_bits=12, budget_bytes=2 << 30, w_max_round=2048)
    fixed = probe.stats()["bytes_fixed"]
    probe.destroy()
    r = 3000
    state = (28 * r + 255) // 256 * 256
    budget = fixed + 3 * state + 2 * 8 * 2048
    n_streams = 10
    specs = [(r, 100 + s, s) for s in range(n_streams)]
    plans = [_plan(rng, _graph(2000 + s), 6, max_w=2000) for s in range(n_streams)]
    srv = tc.Server(max_streams=16, vertex_bits=12, budget_bytes=budget, w_max_round=2048)
    try:
        where, done = _run_mix(srv, specs, plans, rng)
        st = srv.stats()
    finally:
        srv.destroy()
    _check(where, done, specs, plans, 12)
    assert st["bytes_peak"] <= budget
    assert st["admission_waits"] > 0
    assert st["opens"] == n_streams and st["streams_open"] == 0


def test_rejected_batch_and_errors():
    rng = np.random.default_rng(3)
    specs = [(200, 1, 0), (300, 2, 1), (400, 3, 2)]
    plans = [_plan(rng, _graph(3000 + s), 8) for s in range(3)]
    # stream 1: one batch repeats an edge and must be rejected alone
    i_bad = next(i for i, op in enumerate(plans[1]) if op[0] == "b" and op[1].size > 2 and i > 0)
    b = plans[1][i_bad][1].copy()
    b[-1] = b[0]
    plans[1][i_bad] = ("b", b)
    srv = tc.Server(max_streams=4, vertex_bits=12, budget_bytes=1 << 30, w_max_round=4096)
    try:
        with pytest.raises(tc.TcError) as e:
            srv.query(12345)
        assert e.value.code == tc.TC_ERR_INVAL
        h, _ = srv.open(10, 1, 1)
        with pytest.raises(tc.TcError) as e:
            srv.submit(h, np.zeros(5000, dtype=np.uint64))
        assert e.value.code == tc.TC_ERR_RANGE
        srv.close(h)
        with pytest.raises(tc.TcError) as e:
            srv.query(h)
        assert e.value.code == tc.TC_ERR_INVAL
        srv.drain(60000)
        srv.poll()
        where, done = _run_mix(srv, specs, plans, rng)
    finally:
        srv.destroy()
    _check(where, done, specs, plans, 12, bad={1: (i_bad,)})


def _alone_w(spec, plan, vertex_bits, w_max):
    """_alone for batches of up to w_max edges."""
    r, seed, sid = spec
    ctx = tc.tc_create_ex(r, seed, sid, w_max, vertex_bits)
    out = []
    try:
        for op in plan:
            if op[0] == "b":
                tc.tc_process_batch(ctx, to_device(op[1]))
            e = tc.tc_estimate(ctx)
            out.append((e["batches"], e["S"], e["n_closed"], e["m"], e["N"], e["tau_hat"]))
    finally:
        tc.tc_destroy(ctx)
    return out


def test_many_streams_through_fewer_slots():
    """512 streams through 128 slots at the default depth, batches of up to
    20,000 edges submitted in chunks: every request completes once and OK,
    each stream's counters advance batch by batch, and 32 sampled streams
    equal their runs alone bit for bit."""
    rng = np.random.default_rng(23)
    base = [_graph(5000 + g, n_lo=3000, n_hi=40000) for g in range(32)]
    n_streams, w_max = 512, 20000
    specs, plans = [], []
    for s in range(n_streams):
        keys = base[int(rng.integers(0, len(base)))]
        start = int(rng.integers(0, max(1, keys.size // 2)))
        window = keys[start:]
        specs.append((int(round(2 ** rng.uniform(4, 12))), int(rng.integers(0, 2**63)),
                      int(rng.integers(0, 2**32))))
        plan, cur = [], 0
        for _ in range(int(rng.integers(4, 12))):
            if rng.random() < 0.1 or cur >= window.size:
                plan.append(("q",))
            else:
                w = int(min(round(10 ** rng.uniform(0, np.log10(w_max))), window.size - cur))
                plan.append(("b", window[cur:cur + w].copy()))
                cur += w
        plan.append(("c",))
        plans.append(plan)
    srv = tc.Server(max_streams=128, vertex_bits=16, budget_bytes=4 << 30, w_max_round=1 << 20)
    try:
        where, done = _run_mix_many(srv, specs, plans, rng, chunk=64)
        st = srv.stats()
    finally:
        srv.destroy()
    assert len(done) == len(where), "every request completes exactly once"
    assert st["opens"] == n_streams and st["closes"] == n_streams
    assert st["max_round_streams"] <= 128 and st["rejected"] == 0
    per = {s: [] for s in range(n_streams)}
    for t, (s, i) in where.items():
        c = done[t]
        assert c["status"] == tc.TC_OK, (s, i, c["status"])
        if i >= 0 and plans[s][i][0] != "c":
            per[s].append((i, int(c["batches"]), int(c["m"])))
    for s, rows in per.items():
        rows.sort()
        nb = m = 0
        for i, b, mm in rows:
            if plans[s][i][0] == "b":
                nb += 1
                m += plans[s][i][1].size
            assert (b, mm) == (nb, m), (s, i)
    for s in rng.choice(n_streams, size=32, replace=False):
        exp = _alone_w(specs[s], plans[s], 16, w_max)
        for t, (s2, i) in where.items():
            if s2 != s or i < 0 or plans[s][i][0] == "c":
                continue
            c = done[t]
            got = (int(c["batches"]), int(c["sum_lo"]) | (int(c["sum_hi"]) << 64),
                   int(c["n_closed"]), int(c["m"]), int(c["num_lo"]) | (int(c["num_hi"]) << 64),
                   float(c["tau_hat"]))
            assert got == exp[i], (s, i, got, exp[i])
