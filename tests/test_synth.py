"""The synthetic stream generators: every stream is simple (no self-loops,
no repeats, keys packed (min << 32) | max), ids stay in range, and the
generators are deterministic in their seed."""
import numpy as np
import pytest

import synth


def _check_simple(keys, n):
    keys = np.asarray(keys, dtype=np.uint64)
    u, v = synth.unpack(keys)
    assert (u < v).all(), "packed (min, max) without self-loops"
    assert int(v.max()) < n
    assert np.unique(keys).size == keys.size, "no repeated edge"


def test_chung_lu_and_finish():
    k = synth.chung_lu(2000, 2.2, 12.0, 9000, seed=3, max_degree=200.0)
    assert k.size == 9000
    _check_simple(k, 2000)
    f = synth.finish(k, 2000, seed=4)
    _check_simple(f, 2000)
    # relabelling keeps the degree sequence up to a permutation
    du = np.bincount(np.concatenate(synth.unpack(k)).astype(np.int64), minlength=2000)
    df = np.bincount(np.concatenate(synth.unpack(f)).astype(np.int64), minlength=2000)
    assert np.array_equal(np.sort(du), np.sort(df))
    assert np.array_equal(f, synth.finish(k, 2000, seed=4)), "deterministic in the seed"


def test_rmat_and_workloads():
    k = synth.rmat(10, 8, 0.57, 0.19, 0.19, seed=5)
    _check_simple(k, 1 << 10)
    tiny = synth.tiny_chung_lu()
    assert tiny.size == 32768
    _check_simple(tiny, 4096)
    parts = synth.batches(tiny, 4096)
    assert len(parts) == 8 and all(p.size == 4096 for p in parts)


def test_multi_streams_shapes():
    streams, r, n = synth.multi_streams(6, per_stream_edges=500, seed=2)
    assert len(streams) == 6 and r.size == 6 and n.size == 6
    for s, keys in enumerate(streams):
        _check_simple(keys, int(n[s]))
        assert keys.size <= 500
    assert (r >= 2 ** 10).all() and (r <= 2 ** 16).all()


def test_device_rmat_on_cpu():
    torch = pytest.importorskip("torch")
    from synth.device import rmat_device
    k = rmat_device(11, 8, 0.57, 0.19, 0.19, seed=7, device="cpu").numpy().view(np.uint64)
    _check_simple(k, 1 << 11)
    k2 = rmat_device(11, 8, 0.57, 0.19, 0.19, seed=7, device="cpu").numpy().view(np.uint64)
    assert np.array_equal(k, k2)
