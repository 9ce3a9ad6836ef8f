/*
 * tc.h -- C ABI of the GB300 streaming triangle-count library (libtc.so).
 *
 * Implements the bulk update of r neighborhood-sampling estimators of
 * Tangwongsan, Pavan and Tirthapura, "Parallel Triangle Counting in Massive
 * Streaming Graphs" (CIKM'13, arXiv:1308.2166): each estimator keeps the
 * tuple (f1, f2, f3, chi) of Invariant 3.1 (Sec. 3.1); a batch W of edges is
 * folded in by Steps 1-3 of Sec. 4 (procedure bulkUpdateAll, Thm. 4.1); the
 * estimate is the mean of the per-estimator values of Lemma 3.1.
 *
 * Conventions shared by every call:
 *   - Edges are uint64 keys (u << 32) | v with u < v (undirected, packed
 *     smaller id first).  Vertex ids are < 2^vertex_bits.  The order of an
 *     edge array is arrival order (Sec. 2: the stream's total order).
 *   - Every call returns 0 (TC_OK) or a negative TC_ERR_* code; no C++
 *     exception crosses the ABI.  tc_strerror() names a code.
 *   - Randomness is Philox4x32-10 keyed by (seed, stream id, estimator,
 *     batch, slot): the same inputs, seed and batch boundaries give the same
 *     state bit for bit, on any launch configuration.
 *   - Device memory for the estimator state and all per-batch scratch is
 *     owned by the library (cudaMalloc on the device that is current when
 *     the context is created).  Input arrays are borrowed for the duration
 *     of the call (or, for *_async calls, until the given CUDA stream
 *     reaches that point).
 *   - A rejected batch (TC_ERR_INPUT) leaves the estimator state, |E| and
 *     the batch counter unchanged: validation results are checked on the
 *     device before any state is written.
 */
#ifndef TC_H
#define TC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TC_OK 0
#define TC_ERR_INVAL (-1)   /* bad argument: null pointer, r == 0, bad sizes */
#define TC_ERR_NOMEM (-2)   /* device or host allocation failed */
#define TC_ERR_INPUT (-3)   /* batch breaks the stream model: self-loop, key
                               not (min,max), id >= 2^vertex_bits, or an edge
                               repeated inside the batch */
#define TC_ERR_CUDA (-4)    /* a CUDA runtime call failed */
#define TC_ERR_TIMEOUT (-5) /* a bounded device-side wait gave up */
#define TC_ERR_RANGE (-6)   /* size beyond a fixed maximum: tc_rank_all_noalloc's
                               scratch, a tc_server's round or memory budget */

/* Empty level-1 / level-2 edge in tc_get_state output. */
#define TC_EMPTY_EDGE 0xFFFFFFFFFFFFFFFFull
/* Bit 0 of a state flag word: the wedge (f1, f2) is closed (f3 present). */
#define TC_FLAG_CLOSED 1u

typedef struct tc_ctx tc_ctx;

/* Result of tc_estimate (Lemma 3.1 aggregated by the plain mean).
 *   S = sum of chi over the estimators whose wedge is closed (128-bit),
 *   N = |E| * S (128-bit, exact), tau_hat = N / r as a double computed as
 *   q + rem / r with q = N div r (q rounded to nearest, rem / r one correctly
 *   rounded division, then one rounded addition).  The first six fields are
 *   the problem statement's result (N, r, |E|, closed count, tau_hat); S and
 *   the batch count follow.  Every call that returns an estimate -- host or
 *   device record, one stream or many -- forms it with the same arithmetic,
 *   so the records agree bit for bit.  72 bytes, no padding. */
typedef struct {
    uint64_t num_lo, num_hi;   /* N = m * S */
    uint64_t r;                /* estimators */
    uint64_t m;                /* |E|: edges folded in so far */
    uint64_t n_closed;         /* estimators with a closed wedge */
    double tau_hat;            /* N / r (display value; N is exact) */
    uint64_t sum_lo, sum_hi;   /* S */
    uint64_t batches;          /* batches folded in so far */
} tc_estimate_t;

/* Create a stream of r >= 1 estimators (Sec. 4.1: est_1..est_r), all empty,
 * |E| = 0, stream id 0, 32-bit vertex ids, scratch for batches of up to
 * 2^22 edges (grown on demand by tc_process_batch).  *out receives the
 * context.  Errors: TC_ERR_INVAL (r == 0, out == NULL), TC_ERR_NOMEM,
 * TC_ERR_CUDA. */
int tc_create(uint64_t r, uint64_t seed, tc_ctx **out);

/* As tc_create with explicit stream id (part of the Philox counter, so
 * independent streams may share a seed), maximum batch size w_max >= 1
 * (scratch is sized for it up front) and vertex_bits in [1, 32] (a promise
 * that every id is < 2^vertex_bits; it shortens the radix-sort keys).
 * r must be < 2^32 (the estimator index is a 32-bit Philox counter word). */
int tc_create_ex(uint64_t r, uint64_t seed, uint32_t stream_id, uint64_t w_max,
                 uint32_t vertex_bits, tc_ctx **out);

/* bulkUpdateAll (Sec. 4, Thm. 4.1): fold the batch edges[0..w) into every
 * estimator -- Step 1 level-1 reservoir (Sec. 4.2), Step 2 rankAll, chi+
 * and level-2 rank-select (Sec. 4.3, Lemma 4.3, Def. 4.2), Step 3 closing
 * edges (Sec. 4.4) -- then |E| += w.  `edges` may be a host pointer (copied
 * to the device inside the call) or a device pointer.  Synchronous: returns
 * once the update is complete.  w == 0 is a no-op (no batch is counted).
 * w above 2^28 is TC_ERR_INVAL.  Errors: TC_ERR_INPUT (state unchanged),
 * TC_ERR_INVAL, TC_ERR_NOMEM, TC_ERR_CUDA, TC_ERR_TIMEOUT. */
int tc_process_batch(tc_ctx *c, const uint64_t *edges, uint64_t w);

/* Enqueue the same update on `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream) for a DEVICE array d_edges, without waiting.
 * w must not exceed the context's current scratch capacity (w_max of
 * tc_create_ex, or the largest w seen by tc_process_batch), else
 * TC_ERR_INVAL.  Device-side errors (a rejected batch, a timeout) are
 * reported by the next tc_sync / tc_estimate on this context; a rejected
 * batch leaves the state unchanged and later batches proceed. */
int tc_process_batch_async(tc_ctx *c, const uint64_t *d_edges, uint64_t w,
                           void *cuda_stream);

/* Pipelined form of tc_process_batch_async for a DEVICE array that already
 * holds the batch when the call is made (filled and synchronised before, not
 * by work still queued on `cuda_stream`).  The batch's sort phase -- key
 * build, both sorts and their directories -- starts on the library's own
 * streams at once, into a second scratch set, so it overlaps the sweep of the
 * previous batch; the sweep and bookkeeping are ordered on `cuda_stream` as
 * usual, so results are bit-identical to the stream-ordered call.  The first
 * call allocates the second scratch set.  d_edges is borrowed until the work
 * on `cuda_stream` passes this batch.  Errors as tc_process_batch_async. */
int tc_process_batch_ready_async(tc_ctx *c, const uint64_t *d_edges, uint64_t w,
                                 void *cuda_stream);

/* tc_process_batch_async for a HOST array (pinned memory for the copy to
 * run asynchronously): the batch is copied to one of two device staging
 * buffers on an internal copy stream, so the copy of each batch overlaps the
 * update of the one before it; the batch is then sorted as soon as its copy
 * lands (pipelined as tc_process_batch_ready_async) and swept on
 * `cuda_stream`.  Returns without waiting.  h_edges is borrowed until the
 * work on `cuda_stream` passes this batch.  w must not exceed the context's
 * scratch capacity, else TC_ERR_INVAL; errors are reported as for
 * tc_process_batch_async.  Do not interleave with tc_process_batch from
 * another host thread. */
int tc_process_batch_host_async(tc_ctx *c, const uint64_t *h_edges, uint64_t w,
                                void *cuda_stream);

/* tc_process_batch_async for n contexts in turn (a native loop, so that
 * many independent streams can be advanced back to back without per-call
 * host overhead): batch k = d_edges[k][0..w[k]) goes to ctxs[k]; w[k] == 0
 * skips it.  Stops at the first error and returns it.  HOST arrays of n
 * entries; the edge arrays are DEVICE pointers. */
int tc_process_batches_async(tc_ctx *const *ctxs, const uint64_t *const *d_edges,
                             const uint64_t *w, uint32_t n, void *cuda_stream);

/* Wait for all work enqueued on the context and return the first
 * device-side error recorded since the last tc_sync (then clear it). */
int tc_sync(tc_ctx *c);

/* The estimate of Lemma 3.1 averaged over the r estimators: S (128-bit) and
 * the closed count are reduced on the device inside every accepted batch
 * update, from the estimators' new state; N = m * S is formed exactly.
 * Synchronises (returns a pending device-side error first, as tc_sync). */
int tc_estimate(tc_ctx *c, tc_estimate_t *out);

/* Enqueue, on `cuda_stream`, one small kernel that writes the current
 * estimate -- as of the last batch enqueued before it on the same stream --
 * to the DEVICE record *d_out, laid out as tc_estimate_t (N, tau_hat and
 * all), without waiting.  The record equals what tc_estimate would return at
 * that point.  d_out must be 8-byte aligned and is borrowed until the stream
 * passes this point.  Errors: TC_ERR_INVAL, TC_ERR_CUDA. */
int tc_estimate_async(tc_ctx *c, tc_estimate_t *d_out, void *cuda_stream);

/* Median-of-means aggregate (Sec. 3.1; the paper's implementation, Sec. 5):
 * estimators are split into g contiguous groups, group k holding indices
 * [k*r/g, (k+1)*r/g); each group's exact mean m * S_k / |group k| is formed
 * and the lower median of the g means is returned as the exact fraction
 * num / den (num 128-bit, den = that group's size) and as a double.
 * Requires 1 <= g <= r.  Synchronises. */
int tc_estimate_mom(tc_ctx *c, uint32_t g, uint64_t *num_lo, uint64_t *num_hi,
                    uint64_t *den, double *value);

/* Copy the estimator state to HOST arrays of r entries each (any may be
 * NULL): f1, f2 as packed keys (TC_EMPTY_EDGE when empty), chi, and flags
 * (TC_FLAG_CLOSED).  Synchronises. */
int tc_get_state(tc_ctx *c, uint64_t *f1, uint64_t *f2, uint64_t *chi,
                 uint32_t *flags);

/* Counters: r, |E| and batches folded in so far.  Synchronises. */
int tc_get_counters(tc_ctx *c, uint64_t *r, uint64_t *m, uint64_t *batches);

/* Per-stage device time of the update (the paper's time breakdown of
 * Sec. 5, Fig. 6: sort vs. multisearch vs. the rest).  Between
 * tc_profile_begin and tc_profile_end every batch and estimate enqueued on
 * this context records CUDA events around each stage on the stream it runs
 * on; tc_profile_end waits for them and returns the sums.  `launches` counts
 * the library kernels launched in that window; `sort_pass_bytes` is the
 * algorithmic traffic of the onesweep digit passes (each launched pass reads
 * and writes its n keys and values once).  Errors: TC_ERR_INVAL,
 * TC_ERR_CUDA. */
typedef struct {
    uint64_t batches;             /* batches recorded */
    uint64_t launches;            /* library kernels launched */
    uint64_t sort_pass_launches;  /* onesweep digit-pass launches */
    uint64_t sort_pass_bytes;     /* algorithmic bytes of those launches */
    uint64_t sort_pass_skipped;   /* passes that found one digit value and did no work */
    uint64_t overflow;            /* 1 if events ran out and some stages went unrecorded */
    double ms_prep;               /* key build, histograms, validation, sort plans */
    /* The two sorts run side by side (the Step-3 `edges` sort and its index
     * on a second CUDA stream); the next four stages partition the main
     * stream's time between the sort plans and the sweep: */
    double ms_arc_sort;           /* rankAll digit passes (Lemma 4.3), with the
                                     `edges` passes (Sec. 4.4) beside them */
    double ms_edge_sort;          /* what is left of the `edges` passes and
                                     their directory after the arc index */
    double ms_dups;               /* arc directory, beside the `edges` branch */
    double ms_sweep;              /* fused Steps 1-3 per estimator (searches) */
    double ms_finish;             /* batch bookkeeping */
    double ms_estimate;           /* tc_estimate / tc_estimate_async reductions */
    double ms_sort_wall;          /* wall time of both sorts' digit passes:
                                     from their start to the later end */
} tc_profile_t;
/* Batches enqueued by the pipelined calls (tc_process_batch_ready_async,
 * tc_process_batch_host_async) run their sort phase on the library's own
 * streams: for them only ms_sweep, ms_finish, ms_estimate and ms_sort_wall
 * are recorded. */

int tc_profile_begin(tc_ctx *c);
int tc_profile_end(tc_ctx *c, tc_profile_t *out);

/* Launch tuning of the two radix sorts (rankAll's arcs, Lemma 4.3; Step 3's
 * edges, Sec. 4.4).  arc_digit_bits / edge_digit_bits: 0 (automatic: 8-bit
 * digits over the live key bits, or 9-bit ones where they save a pass), 8,
 * 9, 10 or 11.  ranking (how a warp
 * finds the lanes holding equal digits): 0 or 2 = one ballot per digit bit
 * (the default), 1 = one match.any per key, 3 = lanes OR their bit into a
 * shared-memory word per (warp, digit; 8-bit digits only, else match.any).
 * Results do not depend on the tuning.  Applies to batches enqueued
 * afterwards.
 * Errors: TC_ERR_INVAL for other values. */
int tc_tune(tc_ctx *c, uint32_t arc_digit_bits, uint32_t edge_digit_bits, uint32_t ranking);

/* Launch shape of the estimator sweep (fused Steps 1-3): blocks of 256
 * threads per SM, 1..6 (0 = 6, the default: one resident wave).  The sweep
 * is bound by random DRAM reads and the digit passes by integer issue, so a
 * wave of fewer blocks per SM leaves room for the next batch's sort passes
 * to run beside it when batches are pipelined.  Results do not depend on
 * it.  Applies to batches enqueued afterwards.  Errors: TC_ERR_INVAL. */
int tc_tune_sweep(tc_ctx *c, uint32_t blocks_per_sm);

/* Key of the 32-bit edge hash that orders the Step-3 lookup keys (Sec. 4.4's
 * `edges` array, sorted here by hash bucket).  Results never depend on the
 * key: a lookup checks every candidate against the batch itself.  Each
 * context starts with a key drawn from the operating system's entropy
 * source, so that no batch can be crafted to crowd its edges into a few
 * hash runs (the repeat check and the lookups scan a run, so crowded runs
 * would cost time quadratic in their length); a fixed key makes the bucket
 * layout reproducible, for tests that build such runs on purpose.  Applies
 * to batches enqueued afterwards.  Errors: TC_ERR_INVAL. */
int tc_set_hash_key(tc_ctx *c, uint64_t key);

/* Free the context and its device memory (NULL is a no-op). */
void tc_destroy(tc_ctx *c);

/* Static description of an error code. */
const char *tc_strerror(int code);

/* rankAll (Lemma 4.3, Fig. 2) as a standalone call: for the DEVICE batch
 * d_edges[0..w), write the 2w arcs ordered by src ascending then pos
 * descending into DEVICE arrays of 2w uint32 each: src, dst, pos (0-based
 * arrival index) and rank = rank(src -> dst) of Def. 4.2 (the number of
 * batch edges on src that arrive after this one).  Work runs on
 * `cuda_stream` and the call returns once it is complete.  Scratch (about
 * 16 bytes per arc) is taken from and returned to the stream-ordered
 * allocator inside the call.  The batch is not validated: its edges must be
 * distinct (min,max) keys without self-loops and ids < 2^vertex_bits, and
 * w <= 2^28.  Errors: TC_ERR_INVAL, TC_ERR_NOMEM, TC_ERR_CUDA,
 * TC_ERR_TIMEOUT. */
int tc_rank_all(const uint64_t *d_edges, uint64_t w, uint32_t vertex_bits,
                uint32_t *d_src, uint32_t *d_dst, uint32_t *d_pos,
                uint32_t *d_rank, void *cuda_stream);

/* ---- Many streams at once -------------------------------------------------
 * A tc_multi holds S independent streams (Sec. 4's bulkUpdateAll applied to
 * each stream's own edges with its own r_s estimators) whose state stays
 * resident in HBM.  One round folds one batch per stream into all of them
 * with a single segmented launch sequence (one key build, one pair of radix
 * sorts over every stream's keys, one repeat check, one estimator sweep,
 * one bookkeeping launch).  Every stream's state is bit-identical to running
 * it alone through tc_create_ex / tc_process_batch with the same seed,
 * stream id and batch boundaries. */
typedef struct tc_multi tc_multi;

/* S = n_streams >= 1 streams; HOST arrays r[S] (estimators, 1..2^32-1),
 * seeds[S], stream_ids[S]; w_max_round = most edges one round may carry in
 * total; vertex_bits as in tc_create_ex.  Requires bits(S-1) + vertex_bits +
 * bits(w_max_round-1) + 1 <= 64 (the rankAll sort keys carry the stream
 * index; the Step-3 keys carry it beside a 32-bit hash of the edge).
 * Errors: TC_ERR_INVAL, TC_ERR_NOMEM, TC_ERR_CUDA. */
int tc_multi_create(uint32_t n_streams, const uint64_t *r, const uint64_t *seeds,
                    const uint32_t *stream_ids, uint64_t w_max_round, uint32_t vertex_bits,
                    tc_multi **out);

/* Enqueue one round on `cuda_stream`: d_edges (DEVICE) holds the streams'
 * batches concatenated in stream order; offsets (HOST, S+1 entries,
 * offsets[0] = 0, non-decreasing) delimit stream s's batch as
 * [offsets[s], offsets[s+1]); an empty range leaves the stream untouched.
 * A batch that breaks the stream model (see TC_ERR_INPUT) is rejected for
 * its stream only; that stream's state stays as it was and tc_multi_sync
 * reports it.  d_edges is borrowed until the stream passes this round. */
int tc_multi_process_async(tc_multi *M, const uint64_t *d_edges, const uint64_t *offsets,
                           void *cuda_stream);

/* Pipelined form of tc_multi_process_async for batches already in place in
 * d_edges when the call is made: the round's sort phase runs on the
 * engine's own streams, into a second round scratch set (allocated by the
 * first call), beside the previous round's sweep; the sweep and bookkeeping
 * stay ordered on `cuda_stream`, so results are bit-identical. */
int tc_multi_process_ready_async(tc_multi *M, const uint64_t *d_edges, const uint64_t *offsets,
                                 void *cuda_stream);

/* As tc_multi_process_async, with each stream's batch in its own DEVICE
 * buffer: d_batches (HOST array of S device pointers) and w (HOST array of
 * S batch lengths; w[s] = 0 sits stream s out and d_batches[s] may then be
 * NULL).  Lets a caller fold batches where they already lie without
 * gathering them into one buffer.  Buffers are borrowed until the stream
 * passes this round.  Errors as tc_multi_process_async. */
int tc_multi_process_ptrs_async(tc_multi *M, const uint64_t *const *d_batches,
                                const uint64_t *w, void *cuda_stream);

/* Capture one round as a CUDA graph on `cuda_stream` (which must not be
 * capturing already) for the DEVICE buffer d_edges and the HOST offsets
 * given here, without running it; tc_multi_replay then launches the whole
 * round -- every kernel of it -- with one graph launch.  Each replay folds
 * whatever d_edges holds at that moment into the streams (the caller
 * refills the buffer between replays; the offsets stay fixed).  A new
 * capture replaces the old one.  Errors: TC_ERR_INVAL (empty round, bad
 * offsets), TC_ERR_CUDA. */
int tc_multi_capture(tc_multi *M, const uint64_t *d_edges, const uint64_t *offsets,
                     void *cuda_stream);
int tc_multi_replay(tc_multi *M, void *cuda_stream);

/* Wait for all rounds; write each stream's first error since the last sync
 * (TC_OK or a TC_ERR_* code) to the HOST array stream_errors[S] (may be
 * NULL), clear them, and return the first nonzero one. */
int tc_multi_sync(tc_multi *M, int32_t *stream_errors);

/* Lemma 3.1's estimate of stream s, as tc_estimate.  Synchronises. */
int tc_multi_estimate(tc_multi *M, uint32_t s, tc_estimate_t *out);

/* Enqueue, on `cuda_stream`, one kernel that writes every stream's estimate
 * record (as tc_multi_estimate would return it) to the DEVICE array
 * d_out[S] of tc_estimate_t.  A slot that holds no stream gets a zero record
 * with r = 0. */
int tc_multi_estimates_async(tc_multi *M, tc_estimate_t *d_out, void *cuda_stream);

/* Stream s's estimator state into HOST arrays of r[s] entries (as
 * tc_get_state), and its counters.  Synchronise. */
int tc_multi_get_state(tc_multi *M, uint32_t s, uint64_t *f1, uint64_t *f2, uint64_t *chi,
                       uint32_t *flags);
int tc_multi_get_counters(tc_multi *M, uint32_t s, uint64_t *r, uint64_t *m,
                          uint64_t *batches);

/* Sort tuning for later rounds, as tc_tune (ranking 3 is treated as 2). */
int tc_multi_tune(tc_multi *M, uint32_t arc_digit_bits, uint32_t edge_digit_bits,
                  uint32_t ranking);

/* Key of the Step-3 edge hash for later rounds, as tc_set_hash_key (each
 * engine starts with a random key). */
int tc_multi_set_hash_key(tc_multi *M, uint64_t key);

/* Library kernels launched by this object so far. */
int tc_multi_launches(tc_multi *M, uint64_t *launches);

void tc_multi_destroy(tc_multi *M);

/* ---- Serving ---------------------------------------------------------------
 * A tc_server takes requests from many concurrent streams as they arrive --
 * open a stream, fold an edge batch, query the estimate, close -- and serves
 * them with continuous batching: a native scheduler thread admits requests
 * in arrival order as stream slots and device memory (within budget_bytes)
 * free up, copies admitted batches to HBM on a copy stream while earlier
 * rounds run, and, whenever fewer than `depth` rounds are in flight, forms
 * the next round from every stream with admitted work (its queued queries,
 * then at most one batch; round robin, up to w_max_round edges) and folds it
 * with the multi-stream engine.  Estimator state stays in HBM from open to
 * close.  A query is answered with the stream's Lemma 3.1 sums after exactly
 * the batches submitted before it, so every result equals that of running
 * the stream alone (tc_create_ex / tc_process_batch, same seed, stream id
 * and batch boundaries), whatever else is in the mix.
 *
 * All calls are thread-safe.  Requests return a ticket at once; each request
 * later yields one tc_completion_t through tc_server_poll. */
typedef struct tc_server tc_server;

#define TC_REQ_OPEN 1
#define TC_REQ_BATCH 2
#define TC_REQ_QUERY 3
#define TC_REQ_CLOSE 4

typedef struct {
    uint32_t max_streams;  /* stream slots open at once, >= 1 */
    uint32_t vertex_bits;  /* every stream's vertex ids < 2^vertex_bits (1..32) */
    uint64_t budget_bytes; /* device memory the server may hold: engine scratch,
                              round buffers, open streams' state (28 B per
                              estimator) and admitted batches (8 B per edge) */
    uint64_t w_max_round;  /* most edges one round folds (and the largest batch) */
    uint32_t depth;        /* rounds in flight, 1..8; 0 means 2.  With more than
                              one, a round's sorts run beside the previous round's
                              sweep (9% more throughput at saturation, measured
                              at depth 2 against 1) */
    uint32_t max_round_streams; /* most streams one round folds; 0 = max_streams
                                   (1 serves one batch per round, back to back) */
} tc_server_config_t;

typedef struct {
    uint64_t ticket;
    uint32_t handle;
    int32_t kind;          /* TC_REQ_* */
    int32_t status;        /* TC_OK, TC_ERR_INPUT (batch rejected, stream
                              unchanged), or the error that stopped the server */
    uint32_t pad;
    /* batch and query: the stream's state after this request, as
     * tc_estimate: batch count, S = sum of closed chi (128-bit), closed
     * count, |E|; zero for open and close */
    uint64_t batches, sum_lo, sum_hi, n_closed, m;
    /* host steady-clock nanoseconds since tc_server_create: submitted,
     * admitted (slot/memory granted), completion recorded */
    uint64_t t_submit_ns, t_admit_ns, t_done_ns;
    /* batch and query: N = m * S (128-bit) and tau_hat = N / r, formed as in
     * tc_estimate_t; zero for open and close */
    uint64_t num_lo, num_hi;
    double tau_hat;
    /* host steady-clock nanoseconds when the request's round was formed and
     * enqueued (zero for an open): t_round - t_admit is the wait for a round
     * slot, t_done - t_round the round itself */
    uint64_t t_round_ns;
} tc_completion_t;

typedef struct {
    uint64_t rounds, kernel_launches;
    uint64_t batches, rejected, edges, queries, opens, closes;
    uint64_t streams_open;      /* now */
    uint64_t requests_waiting;  /* not yet admitted, now */
    uint64_t admission_waits;   /* head requests that had to wait for memory or a slot */
    uint64_t max_round_edges, max_round_streams;
    uint64_t bytes_budget, bytes_fixed, bytes_reserved, bytes_peak;
    /* the longest stretch between two scheduler passes while work was in
     * flight or waiting (beyond the scheduler's own bounded waits), and how
     * many stretches exceeded 5 ms: stalls of the scheduler thread itself */
    uint64_t sched_gap_max_ns, sched_gaps_over_5ms;
    /* the longest stretch with `depth` rounds in flight, i.e. the scheduler
     * waiting for the GPU before it may form the next round */
    uint64_t inflight_full_max_ns;
    /* the server's memory pool (stream state and batch copies): physical
     * memory it holds and the most it had in use at once, high-water marks */
    uint64_t pool_reserved_high, pool_used_high;
    /* device time of the rounds (CUDA events): the longest round, from the
     * start of its work on the compute stream to its records; how many took
     * more than 5 ms; and the longest round's split into waiting (for its
     * batches' copies and, with depth > 1, the previous round's sweep), its
     * sorts and directories, and its sweep and records */
    uint64_t round_gpu_max_ns, rounds_gpu_over_5ms;
    uint64_t round_max_wait_ns, round_max_sort_ns, round_max_sweep_ns;
} tc_server_stats_t;

/* Errors: TC_ERR_INVAL (bad config; key bits as tc_multi_create with
 * S = max_streams), TC_ERR_RANGE (budget below the fixed scratch),
 * TC_ERR_NOMEM, TC_ERR_CUDA.  Uses the current CUDA device.  The server's
 * memory pool (stream state and batch copies) maps min(16 GB, budget minus
 * the fixed scratch) at creation, so admitting requests never waits for the
 * pool to grow that far; it keeps what it maps until tc_server_destroy. */
int tc_server_create(const tc_server_config_t *cfg, tc_server **out);

/* Request a new stream with r estimators (1..2^32-1), Philox seed and stream
 * id; *handle names it in later calls at once (requests may follow before
 * the open is admitted).  TC_ERR_RANGE if its state can never fit. */
int tc_server_open(tc_server *S, uint64_t r, uint64_t seed, uint32_t stream_id,
                   uint32_t *handle, uint64_t *ticket);

/* Submit a batch of w edges (HOST memory, (min << 32) | max, arrival order).
 * The buffer is borrowed until the batch's completion.  Pinned memory (and,
 * on a device that reads pageable host memory, any host memory) is uploaded
 * when the batch is admitted by the server's own copy kernel, one launch for
 * every batch admitted together; other memory by cudaMemcpyAsync.  w = 0 completes as a no-op.  TC_ERR_INVAL for an
 * unknown or closed handle, TC_ERR_RANGE for w > w_max_round or a batch that
 * can never fit the budget.  A batch that breaks the stream model completes
 * with TC_ERR_INPUT and leaves its stream as it was. */
int tc_server_submit(tc_server *S, uint32_t handle, const uint64_t *h_edges, uint64_t w,
                     uint64_t *ticket);

/* Ask for the stream's estimate after every batch submitted before this call. */
int tc_server_query(tc_server *S, uint32_t handle, uint64_t *ticket);

/* Submit n requests in one call, in array order, as if by n calls of
 * tc_server_submit (kinds[i] = TC_REQ_BATCH) or tc_server_query
 * (TC_REQ_QUERY), under one lock and one wake-up of the scheduler.  All HOST
 * arrays of n entries; h_edges[i] and w[i] are ignored for queries.
 * tickets[i] receives request i's ticket.  Every request is checked first:
 * on an error (as those calls give, or TC_ERR_INVAL for another kind) none is
 * submitted. */
int tc_server_submit_many(tc_server *S, uint32_t n, const uint32_t *kinds,
                          const uint32_t *handles, const uint64_t *const *h_edges,
                          const uint64_t *w, uint64_t *tickets);

/* Close the stream after its earlier requests; its slot and state memory
 * return to the server.  The handle is invalid from this call on. */
int tc_server_close(tc_server *S, uint32_t handle, uint64_t *ticket);

/* Copy up to max_n completions, in completion order, to the HOST array out;
 * wait up to wait_us microseconds if none is ready.  *n_out = count. */
int tc_server_poll(tc_server *S, tc_completion_t *out, uint32_t max_n, uint32_t wait_us,
                   uint32_t *n_out);

/* Wait until every request submitted so far has completed (TC_ERR_TIMEOUT
 * after timeout_ms milliseconds).  Returns the server's failure code, if any. */
int tc_server_drain(tc_server *S, uint32_t timeout_ms);

int tc_server_stats(tc_server *S, tc_server_stats_t *out);

/* Stop the scheduler, wait for the rounds in flight and free everything;
 * requests not yet in a round are dropped without completion. */
void tc_server_destroy(tc_server *S);

/* ---- Checkpoint / resume ----------------------------------------------------
 * A stream's whole state -- the estimator tuples (f1, f2, f3 as the closed
 * bit, chi), |E|, the batch counter, seed, stream id and vertex bits -- as
 * one host blob: a 128-byte header (magic "TCSTATE1", version 1, then r,
 * seed, stream id, vertex bits, |E|, batches, S low, S high, closed count,
 * as little-endian uint64) followed by f1[r], f2[r], chi[r] (uint64) and
 * flags[r] (uint32).  Because every draw is a function of (seed, stream id,
 * estimator, batch, slot), a stream loaded from a blob continues bit for bit
 * as if it had never stopped.  (The paper keeps its state in memory only;
 * this is the library's own.) */

/* Bytes tc_save writes for this context: 128 + 28 r. */
uint64_t tc_save_size(tc_ctx *c);

/* Write the blob to the HOST buffer buf of `size` bytes (>= tc_save_size).
 * Synchronises.  Errors: TC_ERR_INVAL, TC_ERR_CUDA. */
int tc_save(tc_ctx *c, void *buf, uint64_t size);

/* Create a context from a blob (scratch for batches of up to w_max edges,
 * as tc_create_ex).  TC_ERR_INVAL if the header is not a version-1 blob,
 * `size` is short, a flag word has bits other than TC_FLAG_CLOSED, a tuple
 * is not one the update can reach (with |E| = 0 every tuple empty; else f1
 * an edge u < v < 2^vertex_bits, f2 empty with chi = 0 or another such
 * edge sharing an endpoint with f1 with chi >= 1, closed only with f2), or
 * the stored S and
 * closed count disagree with the state; TC_ERR_NOMEM, TC_ERR_CUDA as
 * tc_create_ex. */
int tc_load(const void *buf, uint64_t size, uint64_t w_max, tc_ctx **out);

/* Self-test of the bounded device-side waits (no counterpart in the paper;
 * the radix sort's look-back is the library's only spin-wait).  Runs one
 * digit pass over two tiles of keys with a single CTA that is handed tile 1,
 * so the predecessor its look-back waits for never publishes; the wait gives
 * up after its iteration limit (about a second), records the timeout and the
 * CTA finishes.  Returns TC_ERR_TIMEOUT when that happened (the expected
 * result), TC_OK if the wait somehow completed, TC_ERR_CUDA on a CUDA error.
 * The device stays usable afterwards.  Synchronises the device. */
int tc_selftest_wait_timeout(void);

/* Largest batch tc_rank_all_noalloc accepts. */
#define TC_NOALLOC_MAX_EDGES (1u << 18)

/* tc_rank_all without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they need rankAll -- a process whose HBM another allocator already
 * owns, a latency-critical loop where cudaMalloc/cudaFree would synchronise
 * the device or could fail with out-of-memory halfway through, or code that
 * must not run out of memory once started.  Same arguments and output as
 * tc_rank_all, for batches of at most TC_NOALLOC_MAX_EDGES edges (larger w
 * returns TC_ERR_RANGE before any GPU work).  Its scratch (about 12.3 MB) is
 * a fixed array in the library's device image, so every GPU that loads
 * libtc.so holds it from module load until the process exits; no call
 * allocates or frees anything.  The first call on a device looks the
 * array's device address up (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the one array and each clears what must start at zero, but calls whose
 * work overlaps on the GPU (other streams, other host threads) race on it:
 * issue them one after another.  Returns after the work on `cuda_stream` is
 * complete.  Errors: TC_ERR_INVAL, TC_ERR_RANGE, TC_ERR_CUDA,
 * TC_ERR_TIMEOUT. */
int tc_rank_all_noalloc(const uint64_t *d_edges, uint64_t w, uint32_t vertex_bits,
                        uint32_t *d_src, uint32_t *d_dst, uint32_t *d_pos,
                        uint32_t *d_rank, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
