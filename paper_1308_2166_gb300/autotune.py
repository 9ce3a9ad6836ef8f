"""Autotuner for the launch parameters of the estimator update.

For a given stream shape (r, w, vertex bits) it replays a few batches of the
caller's data under every candidate tuning and returns the fastest:
``tune`` -- arc and edge digit widths (8 to 11 bits, the widths that save a
pass) and the warp ranking method (one ballot per digit bit, match.any or an
atomic OR per lane), timed on the sorts' stage events; ``tune_sweep`` -- the
estimator sweep's blocks per SM, timed on whole pipelined batches (the sweep
of one batch runs beside the sorts of the next).  Every tuning gives
bit-identical results, so tuning runs on scratch contexts and never touches
the caller's estimators.
"""
from __future__ import annotations

import itertools

from . import (tc_create_ex, tc_destroy, tc_process_batch_async,
               tc_process_batch_ready_async, tc_profile_begin, tc_profile_end, tc_sync, tc_tune,
               tc_tune_sweep)

DIGITS = (8, 9, 10, 11)
RANKINGS = {1: "match", 2: "ballot", 3: "atomic-or"}


def _passes(bits: int, width: int) -> int:
    return max(1, -(-bits // width))


def _widths(bits: int):
    """Digit widths worth timing over `bits` key bits: 8, and each wider
    width that needs fewer passes than every narrower one (a wider digit
    only pays for itself by saving a pass)."""
    out = [8]
    for d in DIGITS[1:]:
        if _passes(bits, d) < _passes(bits, out[-1]):
            out.append(d)
    return out


def step3_bits(w: int) -> int:
    """Bucket bits of the Step-3 keys' sort for batches of w edges."""
    bw = max(1, (w - 1).bit_length())
    return bw - 2 if bw > 3 else 1


def candidates(vertex_bits: int, w: int | None = None):
    """Tunings worth timing: for the arcs (vertex_bits key bits) and, when the
    batch size is known, the Step-3 keys, the widths that save a pass; every
    warp ranking method."""
    arc = _widths(vertex_bits)
    edge = _widths(step3_bits(w)) if w else list(DIGITS)
    return [(ba, be, rk) for ba, be, rk in itertools.product(arc, edge, RANKINGS)]


def tune(dev_batches, r: int, vertex_bits: int, seed: int = 1, reps: int = 2,
         stream: int = 0, candidates_list=None):
    """Time each tuning on the given device batches; return (best, table).

    ``dev_batches``: list of device arrays (torch tensors) of packed edges.
    ``table`` maps (arc_bits, edge_bits, ranking) to milliseconds per batch
    of the two sorts' digit passes (wall time; they run side by side).
    """
    w_max = max(int(b.numel()) for b in dev_batches)
    table = {}
    for cand in candidates_list or candidates(vertex_bits, w_max):
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


SWEEP_BLOCKS = (2, 3, 4, 6)


def tune_sweep(dev_batches, r: int, vertex_bits: int, tuning, seed: int = 1, stream: int = 0,
               warm: int = 2, candidates_list=SWEEP_BLOCKS):
    """Time whole pipelined batches (tc_process_batch_ready_async) for each
    sweep shape in blocks per SM; return (best, table of ms per batch).
    ``dev_batches``: device batches already in place; the first ``warm``
    run untimed, the rest are timed with CUDA events on ``stream``."""
    import torch
    w_max = max(int(b.numel()) for b in dev_batches)
    table = {}
    st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.current_stream()
    for bps in candidates_list:
        ctx = tc_create_ex(r, seed, 0, w_max, vertex_bits)
        try:
            tc_tune(ctx, *tuning)
            tc_tune_sweep(ctx, bps)
            for b in dev_batches[:warm]:
                tc_process_batch_ready_async(ctx, b, stream=stream)
            tc_sync(ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for b in dev_batches[warm:]:
                tc_process_batch_ready_async(ctx, b, stream=stream)
            e1.record(st)
            st.synchronize()
            tc_sync(ctx)
            table[bps] = e0.elapsed_time(e1) / max(1, len(dev_batches) - warm)
        finally:
            tc_destroy(ctx)
    best = min(table, key=table.get)
    return best, table


def tune_pipeline(dev_batches, r: int, vertex_bits: int, tuning, sweep_blocks: int = 0,
                  seed: int = 1, stream: int = 0, warm: int = 2):
    """Time whole batches stream-ordered (tc_process_batch_async) and
    pipelined (tc_process_batch_ready_async: each batch's sorts beside the
    previous batch's sweep) on scratch contexts; return ("on" | "off",
    table of ms per batch).  Results are identical either way."""
    import torch
    w_max = max(int(b.numel()) for b in dev_batches)
    st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.current_stream()
    table = {}
    for mode, fn in (("off", tc_process_batch_async), ("on", tc_process_batch_ready_async)):
        ctx = tc_create_ex(r, seed, 0, w_max, vertex_bits)
        try:
            tc_tune(ctx, *tuning)
            tc_tune_sweep(ctx, sweep_blocks)
            for b in dev_batches[:warm]:
                fn(ctx, b, stream=stream)
            tc_sync(ctx)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for b in dev_batches[warm:]:
                fn(ctx, b, stream=stream)
            e1.record(st)
            st.synchronize()
            tc_sync(ctx)
            table[mode] = e0.elapsed_time(e1) / max(1, len(dev_batches) - warm)
        finally:
            tc_destroy(ctx)
    return min(table, key=table.get), table
