"""GPU path vs the CPU oracle: bit-identical estimator states and estimates.

Every call goes through the C ABI (ctypes binding).  Integer work throughout,
so the bar is bit equality of (f1, f2, chi, flags) after every batch and of
the 128-bit sum S.
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


def _run_pair(keys, r, w_list, seed, vertex_bits, stream_id=0, host_input=False,
              check_every=True):
    ctx = tc.tc_create_ex(r, seed, stream_id, max(w_list) if w_list else 1, vertex_bits)
    ref = nbsi_bulk.BulkStream(r, seed=seed, stream=stream_id, vertex_bits=vertex_bits)
    try:
        i = 0
        for k, w in enumerate(w_list):
            W = keys[i:i + w]
            i += w
            tc.tc_process_batch(ctx, W if host_input else to_device(W))
            ref.process_batch(W)
            if check_every or k == len(w_list) - 1:
                assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), f"batch {k}")
        est = tc.tc_estimate(ctx)
        assert est["S"] == ref.closed_sum()
        assert est["m"] == ref.m and est["batches"] == ref.b
        assert est["N"] == ref.m * ref.closed_sum()
        assert est["n_closed"] == int(ref.closed.sum())
        return est
    finally:
        tc.tc_destroy(ctx)


@pytest.mark.parametrize("vertex_bits", [12, 32])
def test_tiny_chung_lu_every_batch(vertex_bits):
    """Chung-Lu n=4096, m=32768, r=1024, w=4096: 8 batches; keys-only
    (12-bit ids) and key+value (32-bit ids) edge sorts."""
    keys = synth.tiny_chung_lu()
    _run_pair(keys, 1024, [4096] * 8, seed=1, vertex_bits=vertex_bits)


def test_ragged_sizes_and_host_input():
    """r and w not multiples of any tile; batch sizes vary; host pointers."""
    keys = synth.tiny_chung_lu(gen_seed=3)
    ws = [1, 2, 3, 4097, 5000, 777, 12345, 1, 9000]
    _run_pair(keys, 1001, ws, seed=77, vertex_bits=12, stream_id=5, host_input=True)


def test_singleton_batches_are_the_sequential_estimator():
    keys = synth.tiny_chung_lu(gen_seed=4)[:300]
    _run_pair(keys, 257, [1] * 300, seed=9, vertex_bits=12, check_every=False)


def test_one_estimator_and_whole_stream_in_one_batch():
    keys = synth.tiny_chung_lu(gen_seed=5)
    _run_pair(keys, 1, [keys.size], seed=2, vertex_bits=12)
    _run_pair(keys, 3, [keys.size], seed=2, vertex_bits=32)


def test_large_seed_and_stream_ids():
    keys = synth.tiny_chung_lu(gen_seed=6)[:20000]
    _run_pair(keys, 4000, [7000, 7000, 6000], seed=(1 << 63) + 12345, vertex_bits=13,
              stream_id=0xFFFFFFFF)


def test_rmat20_full_size():
    """R-MAT scale 20 (about 15.7M edges), r = 2^20, w = 2^22: all batches."""
    keys = synth.rmat20_single()
    w = 1 << 22
    ws = [min(w, keys.size - i) for i in range(0, keys.size, w)]
    est = _run_pair(keys, 1 << 20, ws, seed=1, vertex_bits=20, check_every=False)
    assert est["m"] == keys.size


@pytest.mark.parametrize("vertex_bits", [12, 20, 32])
def test_every_sort_tuning_gives_identical_states(vertex_bits):
    """Digit widths 8/10/11 and both warp rankings: same states as the oracle."""
    from paper_1308_2166_gb300 import autotune
    keys = synth.tiny_chung_lu(gen_seed=21)
    r, w = 777, 5000
    ref = nbsi_bulk.BulkStream(r, seed=3, vertex_bits=vertex_bits)
    for W in synth.batches(keys, w):
        ref.process_batch(W)
    exp = ref.state_arrays()
    dev = [to_device(W) for W in synth.batches(keys, w)]
    for cand in autotune.candidates(vertex_bits) + [(0, 0, 0)]:
        ctx = tc.tc_create_ex(r, 3, 0, w, vertex_bits)
        try:
            tc.tc_tune(ctx, *cand)
            for d in dev:
                tc.tc_process_batch(ctx, d)
            assert_state_equal(tc.tc_get_state(ctx), exp, f"tuning {cand}")
        finally:
            tc.tc_destroy(ctx)


def _packed_directory_stream(seed=0):
    """Batch 0 puts 300 arcs into the group of vertices 60..71 (a hub), exactly
    255 into 84..95 and 256 into 96..107 (the packed offsets keep up to 255
    arcs per group of 12 ids), and arcs on every id of the last, partial group
    4092..4095 of the 2^12 ids; later batches are random edges over all ids."""
    rng = np.random.default_rng(seed)
    n, w = 1 << 12, 4096
    designed = set()

    def others(k, avoid):
        pool = np.setdiff1d(np.arange(120, 4092), avoid)
        return rng.choice(pool, size=k, replace=False)

    for x in others(300, []):
        designed.add((63, int(x)))
    for x in others(200, []):
        designed.add((84, int(x)))
    for x in others(55, []):
        designed.add((95, int(x)))
    for x in others(256, []):
        designed.add((96, int(x)))
    for a in range(4092, 4096):
        for x in others(5, []):
            designed.add((int(x), a))
    designed.add((4092, 4095))
    special = set(range(60, 72)) | set(range(84, 108)) | set(range(4092, 4096))
    edges = set(designed)
    batch0 = list(designed)
    while len(batch0) < w:
        u, v = sorted(int(t) for t in rng.integers(0, n, 2))
        if u == v or (u, v) in edges or u in special or v in special:
            continue
        edges.add((u, v))
        batch0.append((u, v))
    rest = []
    # triangles through the hubs: (hub, x) in batch 0, then (x, y) and (hub, y)
    for hub in (63, 84, 96):
        nb = np.array(sorted(b for a, b in designed if a == hub))
        made = 0
        while made < 100:
            x, y = int(rng.choice(nb)), int(rng.integers(120, 4092))
            e1, e2 = (min(x, y), max(x, y)), (hub, y)
            if x == y or e1 in edges or e2 in edges:
                continue
            edges.update((e1, e2))
            rest += [e1, e2]
            made += 1
    while len(rest) < 3 * w:
        u, v = sorted(int(t) for t in rng.integers(0, n, 2))
        if u == v or (u, v) in edges:
            continue
        edges.add((u, v))
        rest.append((u, v))
    rng.shuffle(batch0)
    rng.shuffle(rest)
    pairs = np.array(batch0 + rest, dtype=np.uint64)
    keys = (pairs[:, 0] << np.uint64(32)) | pairs[:, 1]
    # the groups the test is about have the arc counts it claims
    ids = np.concatenate([pairs[:w, 0], pairs[:w, 1]]).astype(np.int64)
    per_group = np.bincount(ids // 12, minlength=(n + 11) // 12)
    assert per_group[5] == 300 and per_group[7] == 255 and per_group[8] == 256
    assert np.all(np.bincount(ids, minlength=n)[4092:4096] > 0)
    return keys, w


def test_packed_arc_offsets_wide_and_boundary_groups():
    """Dense arc offsets (2^12 ids <= 8w): the packed entries, the groups too
    wide to pack and the partial last group all give the oracle's states."""
    keys, w = _packed_directory_stream()
    _run_pair(keys, 4096, [w] * 4, seed=31, vertex_bits=12)
    _run_pair(keys, 999, [w // 2] * 8, seed=32, vertex_bits=12)
