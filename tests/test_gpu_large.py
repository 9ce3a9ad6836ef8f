"""Config 3 at full size: r = 2^24 estimators, batches of w = 2^24 edges,
vertex ids of 25 bits (the Step-3 keys no longer fit 64 bits with the
position, so the edge sort carries it as a value).

The first two batches of the large Chung-Lu stream (exponent 2.1, n = 2^25,
degrees capped at 3e5) go through the library exactly as the benchmark
drives it, and the whole estimator state after each batch must equal the
CPU oracle's bit for bit.  Batch 1 replaces every level-1 edge; batch 2
exercises the old-f1 path.  Slow: the oracle takes minutes at this size.
"""
import numpy as np
import pytest

import paper_1308_2166_gb300 as tc
import synth
from gpu_util import assert_state_equal, to_device
from oracle import nbsi_bulk

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_2166_gb300 import build
    build.build()
    tc.load()


def test_large_config_first_two_batches():
    cfg = synth.WORKLOADS["large"]
    r, w, vb, seed = cfg["r"], cfg["w"], cfg["vertex_bits"], cfg["seed"]
    keys = synth.large_prefix(2)
    assert keys.size == 2 * w
    ctx = tc.tc_create_ex(r, seed, 0, w, vb)
    ref = nbsi_bulk.BulkStream(r, seed=seed, stream=0, vertex_bits=vb)
    try:
        for b in range(2):
            W = keys[b * w:(b + 1) * w]
            tc.tc_process_batch(ctx, to_device(W))
            ref.process_batch(W)
            assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), f"batch {b}")
            est = tc.tc_estimate(ctx)
            assert est["S"] == ref.closed_sum()
            assert est["m"] == ref.m == (b + 1) * w
            assert est["n_closed"] == int(ref.closed.sum())
    finally:
        tc.tc_destroy(ctx)
