"""Step-3 lookups and repeat checks inside long runs of equal sorted hash bits.

The Step-3 keys sort on the top bits of a 32-bit edge mix only, so keys whose
top bits agree keep their batch order inside one run, and a lookup or a
repeat check scans that run.  Random batches almost never form runs longer
than one or two keys; here every edge of a dense core (many triangles) gets
six filler edges whose mix agrees with it in the top 16 bits, which is at
least every bit the library sorts on for these batch sizes (whole 8-bit
digits covering about bits(w) - 2 bucket bits, or bw + 1 bits next to the
participant index in a round of two).  Closing edges then sit at every place
of runs of seven, and the GPU state must still match the oracle bit for bit.

The mix is keyed (each context draws a random key, so that no batch can be
crafted against it); these tests fix the key with tc_set_hash_key to build
the runs, and one test checks that under a context's own random key the
crafted batches no longer form long runs and the state still matches.
"""
import numpy as np
import pytest

import paper_1308_2166_gb300 as tc
from gpu_util import assert_state_equal, to_device
from oracle import nbsi_bulk

pytestmark = pytest.mark.gpu

VB = 20
PREFIX_BITS = 16
KEY = 0x243F6A8885A308D3   # the key the runs are built for


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_2166_gb300 import build
    build.build()
    tc.load()


def _mix_high(x, key=KEY):
    """The library's keyed Step-3 edge mix: SplitMix64's finaliser (Steele,
    Lea, Flood, OOPSLA 2014), high 32 bits, on packed edges (u << 32) | v
    xor the key."""
    x = np.asarray(x, dtype=np.uint64) ^ np.uint64(key)
    x ^= x >> np.uint64(30)
    x *= np.uint64(0xBF58476D1CE4E5B9)
    x ^= x >> np.uint64(27)
    x *= np.uint64(0x94D049BB133111EB)
    x ^= x >> np.uint64(31)
    return x >> np.uint64(32)


def _collision_batches(seed, core_n=48, fillers=6):
    """Two batches: each half of K_core plus, per core edge, `fillers` edges
    on other vertices whose mix shares its top PREFIX_BITS bits."""
    rng = np.random.default_rng(seed)
    iu, iv = np.triu_indices(core_n, 1)
    core = (iu.astype(np.uint64) << np.uint64(32)) | iv.astype(np.uint64)
    rng.shuffle(core)
    # candidate fillers: random pairs of vertices in [core_n, 2^VB)
    a = rng.integers(core_n, 1 << VB, size=1 << 22, dtype=np.uint64)
    b = rng.integers(core_n, 1 << VB, size=1 << 22, dtype=np.uint64)
    keep = a != b
    u, v = np.minimum(a, b)[keep], np.maximum(a, b)[keep]
    cand = np.unique((u << np.uint64(32)) | v)
    cpre = _mix_high(cand) >> np.uint64(32 - PREFIX_BITS)
    order = np.argsort(cpre, kind="stable")
    cand, cpre = cand[order], cpre[order]
    used = np.zeros(cand.size, dtype=bool)
    halves = []
    for part in (core[: core.size // 2], core[core.size // 2:]):
        out = [part]
        for e in part:
            p = _mix_high(np.array([e]))[0] >> np.uint64(32 - PREFIX_BITS)
            lo, hi = np.searchsorted(cpre, p), np.searchsorted(cpre, p, side="right")
            idx = [i for i in range(lo, hi) if not used[i]][:fillers]
            assert len(idx) == fillers, "too few candidates for a prefix"
            used[idx] = True
            out.append(cand[idx])
        W = np.concatenate(out)
        rng.shuffle(W)
        halves.append(W)
    return halves


def test_runs_of_equal_sorted_bits_single_stream():
    batches = _collision_batches(1)
    for W in batches:
        pre = _mix_high(W) >> np.uint64(32 - PREFIX_BITS)
        _, counts = np.unique(pre, return_counts=True)
        assert counts.min() >= 7 and not (counts % 7).any()   # runs of seven or more
    r, seed = 4096, 11
    ctx = tc.tc_create_ex(r, seed, 3, max(W.size for W in batches), VB)
    tc.tc_set_hash_key(ctx, KEY)
    ref = nbsi_bulk.BulkStream(r, seed=seed, stream=3, vertex_bits=VB)
    try:
        for k, W in enumerate(batches):
            tc.tc_process_batch(ctx, to_device(W))
            ref.process_batch(W)
            assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), f"batch {k}")
        assert int(ref.closed.sum()) > 100       # many lookups found their closing edge
        est = tc.tc_estimate(ctx)
        assert est["S"] == ref.closed_sum()
    finally:
        tc.tc_destroy(ctx)


def test_repeat_inside_a_run_is_rejected():
    W = _collision_batches(2)[0]
    pre = _mix_high(W) >> np.uint64(32 - PREFIX_BITS)
    # repeat the FIRST member of some run at the end of the batch: in the
    # sorted order the rest of the run lies between the two copies
    members = np.flatnonzero(pre == pre[0])
    bad = np.concatenate([W, W[members[0]:members[0] + 1]])
    ctx = tc.tc_create_ex(256, 5, 0, bad.size, VB)
    tc.tc_set_hash_key(ctx, KEY)
    ref = nbsi_bulk.BulkStream(256, seed=5, vertex_bits=VB)
    try:
        with pytest.raises(tc.TcError) as e:
            tc.tc_process_batch(ctx, to_device(bad))
        assert e.value.code == tc.TC_ERR_INPUT
        tc.tc_process_batch(ctx, to_device(W))
        ref.process_batch(W)
        assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), "after reject")
    finally:
        tc.tc_destroy(ctx)


def test_runs_of_equal_sorted_bits_in_a_round():
    """Round of two: the collision batches in participant 1, and participant
    0's repeat inside a run is rejected without touching participant 1."""
    A = _collision_batches(3)
    B = _collision_batches(4)
    r = [300, 4096]
    seeds, sids = [21, 22], [0, 1]
    M = tc.MultiStream(r, seeds, sids, w_max_round=2 * max(x.size for x in A + B) + 8,
                       vertex_bits=VB)
    M.set_hash_key(KEY)
    refs = [nbsi_bulk.BulkStream(r[s], seed=seeds[s], stream=sids[s], vertex_bits=VB)
            for s in range(2)]
    try:
        for k in range(2):
            W0 = A[k]
            if k == 1:
                pre = _mix_high(W0) >> np.uint64(32 - PREFIX_BITS)
                members = np.flatnonzero(pre == pre[3])
                W0 = np.concatenate([W0, W0[members[0]:members[0] + 1]])
            W1 = B[k]
            offs = np.array([0, W0.size, W0.size + W1.size], dtype=np.uint64)
            M.process_async(to_device(np.concatenate([W0, W1])), offs)
            if k == 0:
                refs[0].process_batch(W0)
            refs[1].process_batch(W1)
            errs = M.sync()
            assert list(errs) == ([0, 0] if k == 0 else [tc.TC_ERR_INPUT, 0])
            for s in range(2):
                assert_state_equal(M.state(s), refs[s].state_arrays(), f"round {k} stream {s}")
        assert int(refs[1].closed.sum()) > 100
    finally:
        M.close()


def test_random_key_defeats_the_crafted_runs():
    """Under a key the batch was not built for, the crafted edges spread over
    the buckets (no run of seven is left), and a context with its own random
    key -- the default -- still matches the oracle bit for bit."""
    batches = _collision_batches(1)
    other = 0x13198A2E03707344
    for W in batches:
        pre = _mix_high(W, other) >> np.uint64(32 - PREFIX_BITS)
        _, counts = np.unique(pre, return_counts=True)
        assert counts.max() < 7
    r, seed = 4096, 11
    ctx = tc.tc_create_ex(r, seed, 3, max(W.size for W in batches), VB)
    ref = nbsi_bulk.BulkStream(r, seed=seed, stream=3, vertex_bits=VB)
    try:
        for k, W in enumerate(batches):
            tc.tc_process_batch(ctx, to_device(W))
            ref.process_batch(W)
            assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), f"batch {k}")
    finally:
        tc.tc_destroy(ctx)
