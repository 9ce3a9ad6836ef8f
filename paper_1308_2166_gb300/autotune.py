"""Autotuner for the radix-sort launch parameters of the estimator update.

For a given stream shape (r, w, vertex bits) it replays a few batches of the
caller's data under every candidate tuning -- arc and edge digit widths
(8, 10, 11 bits) and the warp ranking method (match.any vs one ballot per
digit bit) -- times the sort stages with the library's stage events, and
returns the fastest.  Every tuning gives bit-identical results, so tuning
runs on a scratch context and never touches the caller's estimators.
"""
from __future__ import annotations

import itertools

from . import (tc_create_ex, tc_destroy, tc_process_batch_async, tc_profile_begin,
               tc_profile_end, tc_sync, tc_tune)

DIGITS = (8, 10, 11)
RANKINGS = {1: "match", 2: "ballot", 3: "atomic-or"}


def candidates(vertex_bits: int):
    """Tunings worth timing: digit widths that change the pass count or width."""
    out = []
    for ba, be, rk in itertools.product(DIGITS, DIGITS, RANKINGS):
        if vertex_bits <= 8 and ba > 8:
            continue
        out.append((ba, be, rk))
    return out


def tune(dev_batches, r: int, vertex_bits: int, seed: int = 1, reps: int = 2,
         stream: int = 0, candidates_list=None):
    """Time each tuning on the given device batches; return (best, table).

    ``dev_batches``: list of device arrays (torch tensors) of packed edges.
    ``table`` maps (arc_bits, edge_bits, ranking) to milliseconds per batch
    of the two sorts' digit passes (wall time; they run side by side).
    """
    w_max = max(int(b.numel()) for b in dev_batches)
    table = {}
    for cand in candidates_list or candidates(vertex_bits):
        ctx = tc_create_ex(r, seed, 0, w_max, vertex_bits)
        try:
            tc_tune(ctx, *cand)
            for b in dev_batches[:1]:            # warm-up
                tc_process_batch_async(ctx, b, stream=stream)
            tc_sync(ctx)
            tc_profile_begin(ctx)
            n = 0
            for _ in range(reps):
                for b in dev_batches:
                    tc_process_batch_async(ctx, b, stream=stream)
                    n += 1
            prof = tc_profile_end(ctx)
            tc_sync(ctx)
        finally:
            tc_destroy(ctx)
        table[cand] = prof["ms_sort_wall"] / n
    best = min(table, key=table.get)
    return best, table
