"""C-ABI behaviour on the GPU: errors, rejected batches, async path, rankAll,
median-of-means, and the toolkit's Philox against the oracle's."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import paper_1308_2166_gb300 as tc
import synth
from golden_io import worked_example
from gpu_util import assert_state_equal, to_device
from oracle import estimate, nbsi_bulk
from oracle.philox import philox4x32

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_2166_gb300 import build
    build.build()
    tc.load()


def test_invalid_arguments():
    with pytest.raises(tc.TcError) as e:
        tc.tc_create(0, 1)
    assert e.value.code == tc.TC_ERR_INVAL
    with pytest.raises(tc.TcError):
        tc.tc_create_ex(10, 1, 0, 16, 33)
    ctx = tc.tc_create_ex(10, 1, 0, 16, 16)
    try:
        d = to_device(np.arange(1, 40, dtype=np.uint64))
        with pytest.raises(tc.TcError) as e:
            tc.tc_process_batch_async(ctx, d)      # w above scratch capacity
        assert e.value.code == tc.TC_ERR_INVAL
    finally:
        tc.tc_destroy(ctx)


@pytest.mark.parametrize("vertex_bits", [12, 32])
def test_rejected_batches_leave_state_unchanged(vertex_bits):
    keys = synth.tiny_chung_lu(gen_seed=8)
    ctx = tc.tc_create_ex(500, 3, 0, 4096, vertex_bits)
    ref = nbsi_bulk.BulkStream(500, seed=3, vertex_bits=vertex_bits)
    try:
        tc.tc_process_batch(ctx, to_device(keys[:3000]))
        ref.process_batch(keys[:3000])
        good = keys[3000:4000]
        bads = [np.concatenate([good, good[10:11]]),                       # repeat
                np.concatenate([good, np.array([(7 << 32) | 7], np.uint64)]),   # self-loop
                np.concatenate([good, np.array([(9 << 32) | 4], np.uint64)])]   # not (min,max)
        if vertex_bits < 32:
            bads.append(np.concatenate([good, np.array([(1 << 32) | (1 << vertex_bits)],
                                                       np.uint64)]))
        for W in bads:
            with pytest.raises(tc.TcError) as e:
                tc.tc_process_batch(ctx, to_device(W))
            assert e.value.code == tc.TC_ERR_INPUT
            assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), "after reject")
            assert tc.tc_get_counters(ctx) == (500, 3000, 1)
        tc.tc_process_batch(ctx, to_device(good))
        ref.process_batch(good)
        assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), "after good")
    finally:
        tc.tc_destroy(ctx)


def test_async_on_torch_stream_and_sticky_error():
    import torch
    keys = synth.tiny_chung_lu(gen_seed=9)
    ctx = tc.tc_create_ex(700, 5, 2, 4096, 12)
    ref = nbsi_bulk.BulkStream(700, seed=5, stream=2, vertex_bits=12)
    s = torch.cuda.Stream()
    try:
        dev = [to_device(W) for W in synth.batches(keys, 4096)]
        bad = to_device(np.concatenate([keys[:10], keys[:1]]))
        with torch.cuda.stream(s):
            for k, d in enumerate(dev):
                tc.tc_process_batch_async(ctx, d, stream=s.cuda_stream)
                if k == 3:
                    tc.tc_process_batch_async(ctx, bad, stream=s.cuda_stream)
        for W in synth.batches(keys, 4096):
            ref.process_batch(W)
        with pytest.raises(tc.TcError) as e:
            tc.tc_sync(ctx)
        assert e.value.code == tc.TC_ERR_INPUT
        tc.tc_sync(ctx)  # cleared
        assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), "async")
        assert tc.tc_get_counters(ctx) == (700, keys.size, 8)
    finally:
        tc.tc_destroy(ctx)


def test_empty_batch_is_noop():
    ctx = tc.tc_create_ex(8, 1, 0, 16, 8)
    try:
        tc.tc_process_batch(ctx, np.zeros(0, dtype=np.uint64))
        assert tc.tc_get_counters(ctx) == (8, 0, 0)
        f1, f2, chi, fl = tc.tc_get_state(ctx)
        assert (f1 == np.uint64(tc.TC_EMPTY_EDGE)).all() and (chi == 0).all()
        assert tc.tc_estimate(ctx)["tau_hat"] == 0.0
    finally:
        tc.tc_destroy(ctx)


def test_pipelined_host_input_matches_oracle():
    """tc_process_batch_host_async: pinned host batches, copies overlapping
    the previous batch's update through two staging buffers."""
    import torch
    keys = synth.tiny_chung_lu()
    parts = synth.batches(keys, 3000)
    pinned = []
    for b in parts:
        t = torch.empty(b.size, dtype=torch.int64, pin_memory=True)
        t.numpy()[:] = b.view(np.int64)
        pinned.append(t)
    ctx = tc.tc_create_ex(300, 9, 4, 3000, 12)
    ref = nbsi_bulk.BulkStream(300, seed=9, stream=4, vertex_bits=12)
    s = torch.cuda.Stream()
    try:
        for t in pinned:
            tc.tc_process_batch_host_async(ctx, t, stream=s.cuda_stream)
        s.synchronize()
        tc.tc_sync(ctx)
        for b in parts:
            ref.process_batch(b)
        assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), "pipelined host input")
        with pytest.raises(tc.TcError):          # above the scratch capacity
            tc.tc_process_batch_host_async(ctx, np.zeros(3001, dtype=np.uint64))
    finally:
        tc.tc_destroy(ctx)


def test_pipelined_batches_match_oracle_and_isolate_errors():
    """tc_process_batch_ready_async overlaps each batch's sorts with the
    previous sweep through two scratch sets: mixed with the stream-ordered
    and synchronous calls, states equal the oracle, and a rejected batch in
    the pipeline leaves its neighbours alone."""
    import torch
    keys = synth.tiny_chung_lu()
    parts = synth.batches(keys, 2500)
    bad = parts[5].copy()
    bad[7] = bad[3]                                  # repeated edge
    devs = [to_device(b) for b in parts]
    dbad = to_device(bad)
    torch.cuda.synchronize()
    ctx = tc.tc_create_ex(400, 21, 2, 2500, 12)
    ref = nbsi_bulk.BulkStream(400, seed=21, stream=2, vertex_bits=12)
    s = torch.cuda.Stream()
    try:
        modes = ["ready", "ready", "async", "ready", "ready", "bad", "ready", "sync", "ready",
                 "async", "ready", "ready", "ready", "ready"]
        for j, mode in enumerate(modes[:len(parts)]):
            if mode == "bad":
                tc.tc_process_batch_ready_async(ctx, dbad, stream=s.cuda_stream)
                continue
            if mode == "ready":
                tc.tc_process_batch_ready_async(ctx, devs[j], stream=s.cuda_stream)
            elif mode == "async":
                tc.tc_process_batch_async(ctx, devs[j], stream=s.cuda_stream)
            else:
                s.synchronize()
                with pytest.raises(tc.TcError) as e:   # reports the earlier rejected batch
                    tc.tc_process_batch(ctx, parts[j])
                assert e.value.code == tc.TC_ERR_INPUT
                ref.process_batch(parts[j])
                continue
            ref.process_batch(parts[j])
        s.synchronize()
        tc.tc_sync(ctx)
        assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), "pipelined mix")
        e = tc.tc_estimate(ctx)
        assert e["S"] == ref.closed_sum() and e["m"] == ref.m and e["batches"] == ref.b
    finally:
        tc.tc_destroy(ctx)


def test_bounded_wait_gives_up_and_device_stays_usable():
    """A look-back wait whose predecessor never publishes runs out (about a
    second) and reports TC_ERR_TIMEOUT; afterwards a batch still matches the
    oracle."""
    import time
    t0 = time.perf_counter()
    assert tc.tc_selftest_wait_timeout() == tc.TC_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    keys = synth.tiny_chung_lu()[:3000]
    ctx = tc.tc_create_ex(64, 5, 0, 4096, 12)
    ref = nbsi_bulk.BulkStream(64, seed=5, stream=0, vertex_bits=12)
    try:
        tc.tc_process_batch(ctx, to_device(keys))
        ref.process_batch(keys)
        assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), "after the timeout")
    finally:
        tc.tc_destroy(ctx)


def _rank_all_gpu(W, vertex_bits):
    import torch
    n = 2 * W.size
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4)]
    tc.tc_rank_all(to_device(W), W.size, vertex_bits, *outs)
    return [o.cpu().numpy().view(np.uint32).astype(np.int64) for o in outs]


def test_rank_all_worked_example_fig2():
    ex = worked_example()
    rows = sorted(ex["batch"], key=lambda t: t[2])
    W = np.array([(min(a, b) << 32) | max(a, b) for a, b, _ in rows], dtype=np.uint64)
    src, dst, pos, rank = _rank_all_gpu(W, 3)
    got = list(zip(src.tolist(), dst.tolist(), (pos + 1).tolist(), rank.tolist()))
    assert got == ex["rankall"]


@pytest.mark.parametrize("w,vertex_bits", [(1, 12), (2, 13), (4095, 12), (50000, 12), (70001, 32)])
def test_rank_all_matches_oracle(w, vertex_bits):
    keys = synth.tiny_chung_lu(gen_seed=11) if w <= 32768 else \
        synth.finish(synth.chung_lu(1 << 12, 2.3, 40.0, w, seed=12), 1 << 12, seed=13)
    W = keys[:w]
    got = _rank_all_gpu(W, vertex_bits)
    exp = nbsi_bulk.rank_all(W)
    for g, e in zip(got, exp):
        assert np.array_equal(g, np.asarray(e, dtype=np.int64))


@pytest.mark.parametrize("g", [1, 2, 5, 64, 1000])
def test_median_of_means_matches_oracle(g):
    keys = synth.tiny_chung_lu(gen_seed=14)
    ctx = tc.tc_create_ex(1000, 4, 0, 8192, 12)
    ref = nbsi_bulk.BulkStream(1000, seed=4, vertex_bits=12)
    try:
        for W in synth.batches(keys, 8192):
            tc.tc_process_batch(ctx, to_device(W))
            ref.process_batch(W)
        got = tc.tc_estimate_mom(ctx, g)
        exp = estimate.median_of_means(ref.m, ref.c.tolist(), ref.closed.tolist(), g)
        from fractions import Fraction
        assert Fraction(got["num"], got["den"]) == exp
    finally:
        tc.tc_destroy(ctx)


def test_toolkit_philox_matches_oracle_philox():
    so = os.path.join(HERE, "cuda", "_probe.so")
    src = os.path.join(HERE, "cuda", "curand_philox_probe.cu")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                           "-Xcompiler", "-fPIC", "-shared", "-o", so, src])
    lib = ctypes.CDLL(so)
    rng = np.random.default_rng(3)
    n = 512
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0], key[0] = 0, 0
    out = np.zeros((n, 4), dtype=np.uint32)
    assert lib.probe_curand_philox(ctr.ctypes.data_as(ctypes.c_void_p),
                                   key.ctypes.data_as(ctypes.c_void_p),
                                   out.ctypes.data_as(ctypes.c_void_p), n) == 0
    for i in range(n):
        assert tuple(int(x) for x in out[i]) == philox4x32(tuple(ctr[i]), tuple(key[i]))
