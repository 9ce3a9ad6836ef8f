"""Config 3 at full size: r = 2^24 estimators, batches of w = 2^24 edges,
vertex ids of 25 bits, on the first 8 batches of the 1.2e9-edge stream the
benchmark times (the large Chung-Lu graph, exponent 2.1, n = 2^25, degrees
capped at 3e5, drawn on the GPU by synth).

The batches go through the library in the benchmark's launch configuration
(the pipelined tc_process_batch_ready_async: two scratch sets, each batch's
sort phase on the library's own streams), and after every batch the whole
estimator state, S, N and tau_hat must equal the CPU oracle's bit for bit.
Batch 1 replaces every level-1 edge; from batch 2 on most estimators keep an
old level-1 edge (replacement probability 1/(b+1) at batch b), whose
degrees come from the vertex directory, and the Step-3 lookups of old
wedges dominate.  Slow: the oracle takes about a minute per batch here.
"""
import numpy as np
import pytest

import paper_1308_2166_gb300 as tc
import synth
from gpu_util import assert_state_equal
from oracle import estimate, nbsi_bulk

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_BATCHES = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1308_2166_gb300 import build
    build.build()
    tc.load()


def test_large_config_first_eight_batches():
    import torch
    cfg = synth.WORKLOADS["large"]
    r, w, vb, seed = cfg["r"], cfg["w"], cfg["vertex_bits"], cfg["seed"]
    stream = synth.large_stream_device()
    assert stream.numel() == synth.LARGE_EDGES
    dev = [stream[b * w:(b + 1) * w].clone() for b in range(N_BATCHES)]
    del stream
    torch.cuda.empty_cache()
    host = [d.cpu().numpy().view(np.uint64) for d in dev]
    ctx = tc.tc_create_ex(r, seed, 0, w, vb)
    ref = nbsi_bulk.BulkStream(r, seed=seed, stream=0, vertex_bits=vb)
    s = torch.cuda.Stream()
    try:
        replaced_last = None
        for b in range(N_BATCHES):
            torch.cuda.synchronize()
            tc.tc_process_batch_ready_async(ctx, dev[b], stream=s.cuda_stream)
            s.synchronize()
            tc.tc_sync(ctx)
            f1_before = ref.f1.copy()
            ref.process_batch(host[b])
            replaced_last = int((ref.f1 != f1_before).sum())
            assert_state_equal(tc.tc_get_state(ctx), ref.state_arrays(), f"batch {b}")
            e = tc.tc_estimate(ctx)
            S, N, tau = estimate.mean_estimate(ref.m, ref.c[ref.closed].tolist(), r)
            assert (e["S"], e["N"], e["m"]) == (S, N, (b + 1) * w)
            assert e["n_closed"] == int(ref.closed.sum()) and e["batches"] == b + 1
            assert e["tau_hat"] == tau
        # the old-f1 regime was reached: about 1/8 of the estimators replaced
        # their level-1 edge in the last batch
        assert replaced_last < r // 4
    finally:
        tc.tc_destroy(ctx)
