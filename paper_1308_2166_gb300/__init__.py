"""Thin Python binding of libtc.so (the C ABI in include/tc.h).

Argument marshalling only: every step of the estimator update runs in the
library's CUDA kernels.  Functions carry the C names; arrays may be numpy
arrays (host) or torch tensors (host or CUDA, int64/uint64 holding the packed
edge keys' bit patterns).  Errors raise ``TcError``.  If the compiled library
is missing this module raises on first use -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libtc.so")

TC_OK = 0
TC_ERR_INVAL = -1
TC_ERR_NOMEM = -2
TC_ERR_INPUT = -3
TC_ERR_CUDA = -4
TC_ERR_TIMEOUT = -5
TC_ERR_RANGE = -6
TC_NOALLOC_MAX_EDGES = 1 << 18
TC_EMPTY_EDGE = (1 << 64) - 1
TC_FLAG_CLOSED = 1

# Every symbol include/tc.h declares (checked by tests/test_abi.py).
EXPORTS = (
    "tc_create", "tc_create_ex", "tc_process_batch", "tc_process_batch_async",
    "tc_sync", "tc_estimate", "tc_estimate_async", "tc_estimate_mom", "tc_get_state",
    "tc_get_counters", "tc_profile_begin", "tc_profile_end", "tc_tune", "tc_destroy",
    "tc_strerror", "tc_rank_all", "tc_rank_all_noalloc",
    "tc_multi_create", "tc_multi_process_async", "tc_multi_sync", "tc_multi_estimate",
    "tc_multi_estimates_async", "tc_multi_get_state", "tc_multi_get_counters",
    "tc_multi_tune", "tc_multi_launches", "tc_multi_destroy", "tc_multi_capture",
    "tc_multi_replay", "tc_process_batches_async", "tc_multi_process_ptrs_async",
    "tc_server_create", "tc_server_open", "tc_server_submit", "tc_server_query",
    "tc_server_close", "tc_server_poll", "tc_server_drain", "tc_server_stats",
    "tc_server_destroy", "tc_selftest_wait_timeout", "tc_save_size", "tc_save", "tc_load",
    "tc_process_batch_host_async", "tc_process_batch_ready_async",
    "tc_multi_process_ready_async", "tc_server_submit_many", "tc_set_hash_key",
    "tc_multi_set_hash_key", "tc_tune_sweep",
)

TC_REQ_OPEN, TC_REQ_BATCH, TC_REQ_QUERY, TC_REQ_CLOSE = 1, 2, 3, 4


class TcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {tc_strerror(code)} ({code})")


class tc_estimate_t(ctypes.Structure):
    _fields_ = [("num_lo", ctypes.c_uint64), ("num_hi", ctypes.c_uint64),
                ("r", ctypes.c_uint64), ("m", ctypes.c_uint64),
                ("n_closed", ctypes.c_uint64), ("tau_hat", ctypes.c_double),
                ("sum_lo", ctypes.c_uint64), ("sum_hi", ctypes.c_uint64),
                ("batches", ctypes.c_uint64)]


# Bytes of one tc_estimate_t record (tc_estimate_async writes one to device
# memory, tc_multi_estimates_async one per stream).
ESTIMATE_BYTES = ctypes.sizeof(tc_estimate_t)


def _estimate_dict(out: tc_estimate_t) -> dict:
    return {"N": out.num_lo | (out.num_hi << 64), "r": out.r, "m": out.m,
            "n_closed": out.n_closed, "tau_hat": out.tau_hat,
            "S": out.sum_lo | (out.sum_hi << 64), "batches": out.batches}


def estimate_records(buf) -> list:
    """Field view of tc_estimate_t records copied to host memory (a numpy
    array or CPU tensor holding n * ESTIMATE_BYTES bytes): one dict per
    record.  Reads the fields only; the library formed every value."""
    import numpy as np
    raw = np.ascontiguousarray(buf.numpy() if hasattr(buf, "numpy") else buf).view(np.uint8)
    n = raw.size // ESTIMATE_BYTES
    return [_estimate_dict(tc_estimate_t.from_buffer_copy(
        raw[k * ESTIMATE_BYTES:(k + 1) * ESTIMATE_BYTES].tobytes())) for k in range(n)]


class tc_profile_t(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("sort_pass_launches", ctypes.c_uint64), ("sort_pass_bytes", ctypes.c_uint64),
                ("sort_pass_skipped", ctypes.c_uint64), ("overflow", ctypes.c_uint64),
                ("ms_prep", ctypes.c_double), ("ms_arc_sort", ctypes.c_double),
                ("ms_edge_sort", ctypes.c_double), ("ms_dups", ctypes.c_double),
                ("ms_sweep", ctypes.c_double), ("ms_finish", ctypes.c_double),
                ("ms_estimate", ctypes.c_double), ("ms_sort_wall", ctypes.c_double)]


class tc_server_config_t(ctypes.Structure):
    _fields_ = [("max_streams", ctypes.c_uint32), ("vertex_bits", ctypes.c_uint32),
                ("budget_bytes", ctypes.c_uint64), ("w_max_round", ctypes.c_uint64),
                ("depth", ctypes.c_uint32), ("max_round_streams", ctypes.c_uint32)]


class tc_completion_t(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("handle", ctypes.c_uint32),
                ("kind", ctypes.c_int32), ("status", ctypes.c_int32), ("pad", ctypes.c_uint32),
                ("batches", ctypes.c_uint64), ("sum_lo", ctypes.c_uint64),
                ("sum_hi", ctypes.c_uint64), ("n_closed", ctypes.c_uint64),
                ("m", ctypes.c_uint64), ("t_submit_ns", ctypes.c_uint64),
                ("t_admit_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64),
                ("num_lo", ctypes.c_uint64), ("num_hi", ctypes.c_uint64),
                ("tau_hat", ctypes.c_double), ("t_round_ns", ctypes.c_uint64)]


_STATS_FIELDS = ("rounds", "kernel_launches", "batches", "rejected", "edges", "queries", "opens",
                 "closes", "streams_open", "requests_waiting", "admission_waits",
                 "max_round_edges", "max_round_streams", "bytes_budget", "bytes_fixed",
                 "bytes_reserved", "bytes_peak", "sched_gap_max_ns", "sched_gaps_over_5ms",
                 "inflight_full_max_ns", "pool_reserved_high", "pool_used_high",
                 "round_gpu_max_ns", "rounds_gpu_over_5ms", "round_max_wait_ns",
                 "round_max_sort_ns", "round_max_sweep_ns")


class tc_server_stats_t(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in _STATS_FIELDS]


_lib = None


def load(path: str | None = None):
    """Load libtc.so (built by ``paper_1308_2166_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libtc.so not built ({path}); run paper_1308_2166_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    sig = {
        "tc_create": (I, [U64, U64, ctypes.POINTER(P)]),
        "tc_create_ex": (I, [U64, U64, U32, U64, U32, ctypes.POINTER(P)]),
        "tc_process_batch": (I, [P, P, U64]),
        "tc_process_batch_async": (I, [P, P, U64, P]),
        "tc_sync": (I, [P]),
        "tc_estimate": (I, [P, ctypes.POINTER(tc_estimate_t)]),
        "tc_estimate_async": (I, [P, P, P]),
        "tc_profile_begin": (I, [P]),
        "tc_profile_end": (I, [P, ctypes.POINTER(tc_profile_t)]),
        "tc_tune": (I, [P, U32, U32, U32]),
        "tc_set_hash_key": (I, [P, U64]),
        "tc_tune_sweep": (I, [P, U32]),
        "tc_multi_set_hash_key": (I, [P, U64]),
        "tc_estimate_mom": (I, [P, U32, ctypes.POINTER(U64), ctypes.POINTER(U64),
                                ctypes.POINTER(U64), ctypes.POINTER(ctypes.c_double)]),
        "tc_get_state": (I, [P, P, P, P, P]),
        "tc_get_counters": (I, [P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64)]),
        "tc_destroy": (None, [P]),
        "tc_strerror": (ctypes.c_char_p, [I]),
        "tc_rank_all": (I, [P, U64, U32, P, P, P, P, P]),
        "tc_rank_all_noalloc": (I, [P, U64, U32, P, P, P, P, P]),
        "tc_multi_create": (I, [U32, P, P, P, U64, U32, ctypes.POINTER(P)]),
        "tc_multi_process_async": (I, [P, P, P, P]),
        "tc_multi_sync": (I, [P, P]),
        "tc_multi_estimate": (I, [P, U32, ctypes.POINTER(tc_estimate_t)]),
        "tc_multi_estimates_async": (I, [P, P, P]),
        "tc_multi_get_state": (I, [P, U32, P, P, P, P]),
        "tc_multi_get_counters": (I, [P, U32, ctypes.POINTER(U64), ctypes.POINTER(U64),
                                      ctypes.POINTER(U64)]),
        "tc_multi_tune": (I, [P, U32, U32, U32]),
        "tc_multi_launches": (I, [P, ctypes.POINTER(U64)]),
        "tc_multi_destroy": (None, [P]),
        "tc_multi_capture": (I, [P, P, P, P]),
        "tc_multi_replay": (I, [P, P]),
        "tc_process_batches_async": (I, [P, P, P, U32, P]),
        "tc_multi_process_ptrs_async": (I, [P, P, P, P]),
        "tc_server_create": (I, [ctypes.POINTER(tc_server_config_t), ctypes.POINTER(P)]),
        "tc_server_open": (I, [P, U64, U64, U32, ctypes.POINTER(U32), ctypes.POINTER(U64)]),
        "tc_server_submit": (I, [P, U32, P, U64, ctypes.POINTER(U64)]),
        "tc_server_query": (I, [P, U32, ctypes.POINTER(U64)]),
        "tc_server_submit_many": (I, [P, U32, P, P, P, P, P]),
        "tc_server_close": (I, [P, U32, ctypes.POINTER(U64)]),
        "tc_server_poll": (I, [P, P, U32, U32, ctypes.POINTER(U32)]),
        "tc_server_drain": (I, [P, U32]),
        "tc_server_stats": (I, [P, ctypes.POINTER(tc_server_stats_t)]),
        "tc_server_destroy": (None, [P]),
        "tc_selftest_wait_timeout": (I, []),
        "tc_process_batch_host_async": (I, [P, P, U64, P]),
        "tc_process_batch_ready_async": (I, [P, P, U64, P]),
        "tc_multi_process_ready_async": (I, [P, P, P, P]),
        "tc_save_size": (U64, [P]),
        "tc_save": (I, [P, P, U64]),
        "tc_load": (I, [P, U64, U64, ctypes.POINTER(P)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != TC_OK:
        raise TcError(rc, where)


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (contiguous)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _len(a) -> int:
    return a.numel() if hasattr(a, "numel") else a.size


def tc_strerror(code: int) -> str:
    return load().tc_strerror(code).decode()


def tc_create(r: int, seed: int) -> int:
    h = ctypes.c_void_p()
    _check(load().tc_create(r, seed, ctypes.byref(h)), "tc_create")
    return h.value


def tc_create_ex(r: int, seed: int, stream_id: int = 0, w_max: int = 1 << 22,
                 vertex_bits: int = 32) -> int:
    h = ctypes.c_void_p()
    _check(load().tc_create_ex(r, seed, stream_id, w_max, vertex_bits, ctypes.byref(h)),
           "tc_create_ex")
    return h.value


def tc_process_batch(ctx: int, edges, w: int | None = None) -> None:
    w = _len(edges) if w is None else w
    _check(load().tc_process_batch(ctx, _ptr(edges) if w else None, w), "tc_process_batch")


def tc_process_batch_async(ctx: int, d_edges, w: int | None = None, stream: int = 0) -> None:
    w = _len(d_edges) if w is None else w
    _check(load().tc_process_batch_async(ctx, _ptr(d_edges) if w else None, w, stream or None),
           "tc_process_batch_async")


def tc_process_batch_ready_async(ctx: int, d_edges, w: int | None = None,
                                 stream: int = 0) -> None:
    """Pipelined update for a device batch that is already in place: its sort
    phase overlaps the previous batch's sweep (bit-identical results)."""
    w = _len(d_edges) if w is None else w
    _check(load().tc_process_batch_ready_async(ctx, _ptr(d_edges) if w else None, w,
                                               stream or None),
           "tc_process_batch_ready_async")


def tc_process_batch_host_async(ctx: int, h_edges, w: int | None = None,
                                stream: int = 0) -> None:
    """Pipelined host-input update: the copy of this batch overlaps the
    update of the previous one (h_edges: pinned CPU tensor or numpy array,
    kept alive by the caller until the stream passes this batch)."""
    w = _len(h_edges) if w is None else w
    _check(load().tc_process_batch_host_async(ctx, _ptr(h_edges) if w else None, w,
                                              stream or None),
           "tc_process_batch_host_async")


def tc_process_batches_async(ctxs, d_edges, stream: int = 0) -> None:
    """One batch per context, enqueued back to back by the library."""
    n = len(ctxs)
    cp = (ctypes.c_void_p * n)(*ctxs)
    ep = (ctypes.c_void_p * n)(*[_ptr(d) if _len(d) else None for d in d_edges])
    wv = (ctypes.c_uint64 * n)(*[_len(d) for d in d_edges])
    _check(load().tc_process_batches_async(cp, ep, wv, n, stream or None),
           "tc_process_batches_async")


def tc_sync(ctx: int) -> None:
    _check(load().tc_sync(ctx), "tc_sync")


def tc_estimate(ctx: int) -> dict:
    out = tc_estimate_t()
    _check(load().tc_estimate(ctx, ctypes.byref(out)), "tc_estimate")
    return _estimate_dict(out)


def tc_estimate_async(ctx: int, d_out, stream: int = 0) -> None:
    """Enqueue the estimate record; d_out: device buffer of at least
    ESTIMATE_BYTES bytes (8-byte aligned), laid out as tc_estimate_t."""
    _check(load().tc_estimate_async(ctx, _ptr(d_out), stream or None), "tc_estimate_async")


def tc_profile_begin(ctx: int) -> None:
    _check(load().tc_profile_begin(ctx), "tc_profile_begin")


def tc_profile_end(ctx: int) -> dict:
    out = tc_profile_t()
    _check(load().tc_profile_end(ctx, ctypes.byref(out)), "tc_profile_end")
    return {name: getattr(out, name) for name, _ in tc_profile_t._fields_}


def tc_tune(ctx: int, arc_digit_bits: int = 0, edge_digit_bits: int = 0, ranking: int = 0) -> None:
    _check(load().tc_tune(ctx, arc_digit_bits, edge_digit_bits, ranking), "tc_tune")


def tc_tune_sweep(ctx: int, blocks_per_sm: int = 0) -> None:
    _check(load().tc_tune_sweep(ctx, blocks_per_sm), "tc_tune_sweep")


def tc_set_hash_key(ctx: int, key: int) -> None:
    _check(load().tc_set_hash_key(ctx, key), "tc_set_hash_key")


def tc_estimate_mom(ctx: int, g: int) -> dict:
    lo, hi, den = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    val = ctypes.c_double()
    _check(load().tc_estimate_mom(ctx, g, ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(den),
                                  ctypes.byref(val)), "tc_estimate_mom")
    return {"num": lo.value | (hi.value << 64), "den": den.value, "value": val.value}


def tc_get_state(ctx: int):
    """(f1, f2, chi, flags) as numpy uint64/uint32 arrays of length r."""
    import numpy as np
    r, _, _ = tc_get_counters(ctx)
    f1 = np.empty(r, dtype=np.uint64)
    f2 = np.empty(r, dtype=np.uint64)
    chi = np.empty(r, dtype=np.uint64)
    fl = np.empty(r, dtype=np.uint32)
    _check(load().tc_get_state(ctx, f1.ctypes.data, f2.ctypes.data, chi.ctypes.data,
                               fl.ctypes.data), "tc_get_state")
    return f1, f2, chi, fl


def tc_get_counters(ctx: int):
    r, m, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().tc_get_counters(ctx, ctypes.byref(r), ctypes.byref(m), ctypes.byref(b)),
           "tc_get_counters")
    return r.value, m.value, b.value


def tc_destroy(ctx: int) -> None:
    if ctx:
        load().tc_destroy(ctx)


def tc_rank_all(d_edges, w: int, vertex_bits: int, d_src, d_dst, d_pos, d_rank,
                stream: int = 0) -> None:
    _check(load().tc_rank_all(_ptr(d_edges), w, vertex_bits, _ptr(d_src), _ptr(d_dst),
                              _ptr(d_pos), _ptr(d_rank), stream or None), "tc_rank_all")


class TriangleStream:
    """Owning wrapper around one tc_ctx (same calls, Python lifetime)."""

    def __init__(self, r: int, seed: int = 1, stream_id: int = 0, w_max: int = 1 << 22,
                 vertex_bits: int = 32):
        self.ctx = tc_create_ex(r, seed, stream_id, w_max, vertex_bits)
        self.r = r

    def process_batch(self, edges, w=None):
        tc_process_batch(self.ctx, edges, w)

    def process_batch_async(self, d_edges, w=None, stream=0):
        tc_process_batch_async(self.ctx, d_edges, w, stream)

    def sync(self):
        tc_sync(self.ctx)

    def estimate(self):
        return tc_estimate(self.ctx)

    def estimate_mom(self, g):
        return tc_estimate_mom(self.ctx, g)

    def state(self):
        return tc_get_state(self.ctx)

    def counters(self):
        return tc_get_counters(self.ctx)

    def close(self):
        if self.ctx:
            tc_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_save(ctx: int) -> bytes:
    """The context's whole state as a checkpoint blob (see tc.h)."""
    n = load().tc_save_size(ctx)
    buf = ctypes.create_string_buffer(n)
    _check(load().tc_save(ctx, buf, n), "tc_save")
    return buf.raw


def tc_load(blob: bytes, w_max: int) -> int:
    """A new context resumed from a tc_save blob."""
    h = ctypes.c_void_p()
    _check(load().tc_load(blob, len(blob), w_max, ctypes.byref(h)), "tc_load")
    return h.value


def tc_selftest_wait_timeout() -> int:
    """Run the bounded-wait self-test; returns its TC_* code (TC_ERR_TIMEOUT
    is the expected result)."""
    return load().tc_selftest_wait_timeout()


def tc_rank_all_noalloc(d_edges, w: int, vertex_bits: int, d_src, d_dst, d_pos, d_rank,
                        stream: int = 0) -> None:
    """tc_rank_all for callers that cannot allocate device memory at call time.

    Same outputs as ``tc_rank_all``; the scratch is a fixed array inside the
    library's device image (held by every GPU that loads the library until
    the process exits), so nothing is allocated or freed.  At most
    ``TC_NOALLOC_MAX_EDGES`` edges; calls must not overlap on the GPU.
    """
    _check(load().tc_rank_all_noalloc(_ptr(d_edges), w, vertex_bits, _ptr(d_src), _ptr(d_dst),
                                      _ptr(d_pos), _ptr(d_rank), stream or None),
           "tc_rank_all_noalloc")


class MultiStream:
    """Owning wrapper around a tc_multi: S independent streams, one round at a
    time (one batch per stream, concatenated on the device)."""

    def __init__(self, r, seeds, stream_ids, w_max_round: int, vertex_bits: int = 32):
        import numpy as np
        self.S = len(r)
        self.r = np.ascontiguousarray(r, dtype=np.uint64)
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        si = np.ascontiguousarray(stream_ids, dtype=np.uint32)
        h = ctypes.c_void_p()
        _check(load().tc_multi_create(self.S, self.r.ctypes.data, sd.ctypes.data, si.ctypes.data,
                                      w_max_round, vertex_bits, ctypes.byref(h)),
               "tc_multi_create")
        self.h = h.value

    def process_async(self, d_edges, offsets, stream: int = 0):
        import numpy as np
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        if off.size != self.S + 1:
            raise ValueError("offsets needs S+1 entries")
        ptr = _ptr(d_edges) if int(off[-1]) else None
        _check(load().tc_multi_process_async(self.h, ptr, off.ctypes.data, stream or None),
               "tc_multi_process_async")

    def process_ready_async(self, d_edges, offsets, stream: int = 0):
        """Pipelined round for batches already in place: sorted beside the
        previous round's sweep (bit-identical results)."""
        import numpy as np
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        if off.size != self.S + 1:
            raise ValueError("offsets needs S+1 entries")
        ptr = _ptr(d_edges) if int(off[-1]) else None
        _check(load().tc_multi_process_ready_async(self.h, ptr, off.ctypes.data, stream or None),
               "tc_multi_process_ready_async")

    def process_ptrs_async(self, d_batches, stream: int = 0):
        """One round with each stream's batch in its own device tensor
        (None or an empty tensor sits the stream out)."""
        import numpy as np
        if len(d_batches) != self.S:
            raise ValueError("need one batch (or None) per stream")
        ptrs = np.zeros(self.S, dtype=np.uint64)
        w = np.zeros(self.S, dtype=np.uint64)
        for s, b in enumerate(d_batches):
            if b is not None and b.numel():
                ptrs[s] = _ptr(b)
                w[s] = b.numel()
        _check(load().tc_multi_process_ptrs_async(self.h, ptrs.ctypes.data, w.ctypes.data,
                                                  stream or None),
               "tc_multi_process_ptrs_async")

    def capture(self, d_edges, offsets, stream: int):
        """Capture one round (fixed buffer and offsets) as a CUDA graph."""
        import numpy as np
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        _check(load().tc_multi_capture(self.h, _ptr(d_edges), off.ctypes.data, stream or None),
               "tc_multi_capture")

    def replay(self, stream: int = 0):
        _check(load().tc_multi_replay(self.h, stream or None), "tc_multi_replay")

    def sync(self):
        """Per-stream error codes since the last sync."""
        import numpy as np
        errs = np.zeros(self.S, dtype=np.int32)
        load().tc_multi_sync(self.h, errs.ctypes.data)
        return errs

    def estimate(self, s: int) -> dict:
        out = tc_estimate_t()
        _check(load().tc_multi_estimate(self.h, s, ctypes.byref(out)), "tc_multi_estimate")
        return _estimate_dict(out)

    def estimates_async(self, d_out, stream: int = 0):
        """Every stream's tc_estimate_t record into the device buffer d_out
        (at least S * ESTIMATE_BYTES bytes)."""
        _check(load().tc_multi_estimates_async(self.h, _ptr(d_out), stream or None),
               "tc_multi_estimates_async")

    def state(self, s: int):
        import numpy as np
        n = int(self.r[s])
        f1 = np.empty(n, dtype=np.uint64)
        f2 = np.empty(n, dtype=np.uint64)
        chi = np.empty(n, dtype=np.uint64)
        fl = np.empty(n, dtype=np.uint32)
        _check(load().tc_multi_get_state(self.h, s, f1.ctypes.data, f2.ctypes.data,
                                         chi.ctypes.data, fl.ctypes.data), "tc_multi_get_state")
        return f1, f2, chi, fl

    def counters(self, s: int):
        r, m, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().tc_multi_get_counters(self.h, s, ctypes.byref(r), ctypes.byref(m),
                                            ctypes.byref(b)), "tc_multi_get_counters")
        return r.value, m.value, b.value

    def tune(self, arc_digit_bits=0, edge_digit_bits=0, ranking=0):
        _check(load().tc_multi_tune(self.h, arc_digit_bits, edge_digit_bits, ranking),
               "tc_multi_tune")

    def set_hash_key(self, key: int):
        _check(load().tc_multi_set_hash_key(self.h, key), "tc_multi_set_hash_key")

    def launches(self) -> int:
        v = ctypes.c_uint64()
        _check(load().tc_multi_launches(self.h, ctypes.byref(v)), "tc_multi_launches")
        return v.value

    def close(self):
        if self.h:
            load().tc_multi_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# numpy view of tc_completion_t
COMPLETION_DTYPE = None


def _completion_dtype():
    global COMPLETION_DTYPE
    if COMPLETION_DTYPE is None:
        import numpy as np
        COMPLETION_DTYPE = np.dtype([
            ("ticket", "<u8"), ("handle", "<u4"), ("kind", "<i4"), ("status", "<i4"),
            ("pad", "<u4"), ("batches", "<u8"), ("sum_lo", "<u8"), ("sum_hi", "<u8"),
            ("n_closed", "<u8"), ("m", "<u8"), ("t_submit_ns", "<u8"), ("t_admit_ns", "<u8"),
            ("t_done_ns", "<u8"), ("num_lo", "<u8"), ("num_hi", "<u8"), ("tau_hat", "<f8"),
            ("t_round_ns", "<u8")])
        assert COMPLETION_DTYPE.itemsize == ctypes.sizeof(tc_completion_t)
    return COMPLETION_DTYPE


class Server:
    """Owning wrapper around a tc_server (continuous-batching request server).

    Host batch buffers are kept alive here until their completion is polled.
    """

    def __init__(self, max_streams: int, vertex_bits: int, budget_bytes: int,
                 w_max_round: int, depth: int = 0, max_round_streams: int = 0):
        import numpy as np
        cfg = tc_server_config_t(max_streams, vertex_bits, budget_bytes, w_max_round, depth,
                                 max_round_streams)
        h = ctypes.c_void_p()
        _check(load().tc_server_create(ctypes.byref(cfg), ctypes.byref(h)), "tc_server_create")
        self.h = h.value
        self._keep = {}
        self._buf = np.zeros(4096, dtype=_completion_dtype())

    def open(self, r: int, seed: int, stream_id: int):
        """Returns (handle, ticket)."""
        hd, t = ctypes.c_uint32(), ctypes.c_uint64()
        _check(load().tc_server_open(self.h, r, seed, stream_id, ctypes.byref(hd),
                                     ctypes.byref(t)), "tc_server_open")
        return hd.value, t.value

    def submit(self, handle: int, edges) -> int:
        """Submit a host batch (numpy uint64 array or CPU torch tensor,
        ideally pinned); returns the ticket."""
        t = ctypes.c_uint64()
        w = int(edges.numel() if hasattr(edges, "numel") else edges.size)
        ptr = _ptr(edges) if w else None
        _check(load().tc_server_submit(self.h, handle, ptr, w, ctypes.byref(t)),
               "tc_server_submit")
        if w:
            self._keep[t.value] = edges
        return t.value

    def query(self, handle: int) -> int:
        t = ctypes.c_uint64()
        _check(load().tc_server_query(self.h, handle, ctypes.byref(t)), "tc_server_query")
        return t.value

    def submit_many(self, kinds, handles, ptrs, ws):
        """Submit many batches and queries in one call (tc_server_submit_many).
        kinds: TC_REQ_BATCH / TC_REQ_QUERY per request; ptrs: host addresses
        of the batches (ints; ignored for queries), ws: their lengths.  The
        caller keeps every batch buffer alive until its completion.  Returns
        the tickets (numpy uint64)."""
        import numpy as np
        kinds = np.ascontiguousarray(kinds, dtype=np.uint32)
        handles = np.ascontiguousarray(handles, dtype=np.uint32)
        ptrs = np.ascontiguousarray(ptrs, dtype=np.uint64)
        ws = np.ascontiguousarray(ws, dtype=np.uint64)
        n = kinds.size
        if not (handles.size == ptrs.size == ws.size == n):
            raise ValueError("submit_many: arrays of different lengths")
        tickets = np.zeros(n, dtype=np.uint64)
        _check(load().tc_server_submit_many(self.h, n, kinds.ctypes.data, handles.ctypes.data,
                                            ptrs.ctypes.data, ws.ctypes.data,
                                            tickets.ctypes.data), "tc_server_submit_many")
        return tickets

    def close(self, handle: int) -> int:
        t = ctypes.c_uint64()
        _check(load().tc_server_close(self.h, handle, ctypes.byref(t)), "tc_server_close")
        return t.value

    def poll(self, wait_us: int = 0):
        """Completions ready now (numpy structured array, COMPLETION_DTYPE)."""
        n = ctypes.c_uint32()
        _check(load().tc_server_poll(self.h, self._buf.ctypes.data, self._buf.size, wait_us,
                                     ctypes.byref(n)), "tc_server_poll")
        out = self._buf[:n.value].copy()
        if self._keep:
            for t in out["ticket"]:
                self._keep.pop(int(t), None)
        return out

    def drain(self, timeout_ms: int = 600000):
        _check(load().tc_server_drain(self.h, timeout_ms), "tc_server_drain")

    def stats(self) -> dict:
        st = tc_server_stats_t()
        _check(load().tc_server_stats(self.h, ctypes.byref(st)), "tc_server_stats")
        return {f: getattr(st, f) for f in _STATS_FIELDS}

    def destroy(self):
        if self.h:
            load().tc_server_destroy(self.h)
            self.h = 0
            self._keep.clear()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
