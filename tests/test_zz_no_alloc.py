"""tc_rank_all_noalloc against tc_rank_all, through the C ABI.

The allocation-free entry point serves callers that cannot allocate device
memory when they need rankAll (HBM owned by another allocator, latency-
critical loops where cudaMalloc/cudaFree would synchronise or fail).  It
must give exactly the output of the allocating tc_rank_all -- integer
arrays, so the tolerance is equality -- on two calls in a row (the second
call finds the first call's leftovers in the shared fixed scratch).  This
file is collected last and also runs on its own in a fresh process.
"""
import numpy as np
import pytest

import paper_1308_2166_gb300 as tc
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_2166_gb300 import build
    build.build()
    tc.load()


def _dev(keys):
    import torch
    return torch.from_numpy(np.ascontiguousarray(keys, dtype=np.uint64).view(np.int64)).cuda()


def _outs(n):
    import torch
    return [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4)]


def _host(outs):
    return [o.cpu().numpy().view(np.uint32).copy() for o in outs]


def test_noalloc_matches_allocating_rank_all_twice():
    keys = synth.finish(synth.chung_lu(1 << 14, 2.3, 30.0, 200000, seed=31), 1 << 14, seed=32)
    big = synth.finish(synth.chung_lu(1 << 17, 2.3, 8.0, tc.TC_NOALLOC_MAX_EDGES, seed=33),
                       1 << 17, seed=34)
    # two calls in a row (the second finds the first's leftovers), then the
    # largest accepted batch at 32-bit ids: both arc buffers full and the
    # most look-back words (four 8-bit digit passes)
    calls = [(keys[:150001], 14), (keys[7:7 + tc.TC_NOALLOC_MAX_EDGES // 2], 32),
             (big, 32)]
    assert big.size == tc.TC_NOALLOC_MAX_EDGES
    for W, vb in calls:
        d = _dev(W)
        ref = _outs(2 * W.size)
        tc.tc_rank_all(d, W.size, vb, *ref)
        got = _outs(2 * W.size)
        tc.tc_rank_all_noalloc(d, W.size, vb, *got)
        for g, e, name in zip(_host(got), _host(ref), ("src", "dst", "pos", "rank")):
            assert np.array_equal(g, e), name


def test_noalloc_rejects_oversized_batch():
    w = tc.TC_NOALLOC_MAX_EDGES + 1
    d = _dev(np.arange(1, w + 1, dtype=np.uint64))
    outs = _outs(2)
    with pytest.raises(tc.TcError) as e:
        tc.tc_rank_all_noalloc(d, w, 32, *outs)
    assert e.value.code == tc.TC_ERR_RANGE
