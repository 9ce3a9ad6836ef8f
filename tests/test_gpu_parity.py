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
