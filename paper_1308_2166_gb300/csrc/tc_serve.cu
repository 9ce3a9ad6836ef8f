// Request server: many concurrent streams send edge batches and estimate
// queries as they arrive; a native scheduler thread keeps every open stream's
// estimator state resident in HBM and folds the batches in with continuous
// batching over the multi-stream round engine.
//
// Pipeline (one scheduler thread, two CUDA streams):
//   admission   requests leave the submission queue in arrival order.  An
//               open needs a free stream slot and its state bytes, a batch
//               its own bytes, within the device-memory budget; the head
//               request waits until earlier work completes and frees them.
//               An admitted batch is copied host -> device on the copy
//               stream at once, overlapping the rounds in flight.
//   rounds      whenever fewer than `depth` rounds are in flight, the next
//               round takes, from each stream with admitted work (round
//               robin), the queries at the head of its queue and then at
//               most one batch, up to w_max_round edges.  The queries are
//               answered from the stream records at the start of the round,
//               i.e. after exactly the batches submitted before them; the
//               batches are folded by one segmented launch sequence on the
//               compute stream, which waits only for their own copies.
//   completion  when a round's event has fired, every request in it gets a
//               completion record (status, the stream's batch count and
//               Lemma 3.1 sums, host timestamps) and its batch memory goes
//               back to the budget.
// Each stream's results are those of running it alone with the same seed,
// stream id and batch boundaries: rounds keep every stream's batches in
// submission order and a stream's arithmetic never depends on the others.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

#include "tc_multi_impl.cuh"
#include "tc_nvtx.h"

using namespace tc;

namespace {

// Bytes of pool memory mapped when a server starts (at most the budget left
// after the fixed scratch).
constexpr u64 kPoolWarmBytes = 16ull << 30;

struct Req {
    u64 ticket = 0;
    int kind = 0;
    u32 handle = 0;
    const u64 *h_edges = nullptr;
    const u64 *h_dev = nullptr;  // h_edges as the device reads it (null: copy engine)
    u64 w = 0;
    u64 r = 0, seed = 0;
    u32 stream_id = 0;
    u64 t_submit = 0, t_admit = 0, t_round = 0;
    u64 *d_edges = nullptr;  // device copy of an admitted batch
    u64 bytes = 0;           // budget bytes it holds until completion
    int ev = -1;             // copy event
    u64 seq = 0;             // copy order
    bool waited = false;     // had to wait for admission
};

struct Slot {
    u32 handle = 0;
    u64 r = 0;  // the stream's estimators
    void *state = nullptr;
    u64 state_bytes = 0;
    bool used = false;
    bool in_ready = false;
    std::deque<Req> q;
};

struct Round {
    int buf = 0;
    bool sorted = false;  // has batches: a sort phase with its own timing events
    std::vector<Req> queries;
    std::vector<Req> batches;
    std::vector<Req> closes;
};

u64 round_up(u64 x) { return (x + 255) & ~255ull; }
u64 state_bytes_for(u64 r) { return round_up(28 * r); }

// Batches admitted in one scheduler pass are uploaded together by a few
// kernel launches: SMs read the host memory (pinned, or pageable where the
// device can read it) in chunks of kUploadWords.  A cudaMemcpyAsync per
// batch cost about 9 us of the scheduler thread each (20,000 batches of
// log-uniform [1e3, 1e6] edges took 171 ms to issue, 130 GB/s), while one
// gather kernel per 50 batches issued the same in 0.6 ms and copied at
// 191 GB/s.  Under serving load the copy-engine path also left rounds
// waiting tens of milliseconds for their batches (p99 batch latency 8-82 ms
// at 70% of saturation against 3.7-16 ms with the kernel, A/B on the same
// boxes), even when only the largest batches took it.
struct UploadChunk {
    const u64 *src;
    u64 *dst;
    u32 n;
    u32 pad;
};
constexpr u32 kUploadWords = 16384;   // words per chunk (128 KB)
constexpr u32 kUploadChunks = 16384;  // chunks per ring slot
constexpr int kUploadSlots = 4;
// One launch per group of at most kUploadGroup chunks (8 MB), each batch's
// copy event recorded behind the group holding its last chunk, so a batch is
// ready as soon as its own group has landed; a block per chunk, eight loads
// in flight per thread.
constexpr u32 kUploadGroup = 64;
constexpr u32 kUploadUnroll = 8;

__global__ void __launch_bounds__(256) upload_kernel(const UploadChunk *__restrict__ chunks,
                                                     u32 nchunks) {
    for (u32 c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const UploadChunk ch = chunks[c];
        for (u32 i0 = threadIdx.x; i0 < ch.n; i0 += 256 * kUploadUnroll) {
            u64 v[kUploadUnroll];
#pragma unroll
            for (u32 k = 0; k < kUploadUnroll; ++k) {
                const u32 i = i0 + k * 256;
                v[k] = i < ch.n ? __ldcs(ch.src + i) : 0ull;
            }
#pragma unroll
            for (u32 k = 0; k < kUploadUnroll; ++k) {
                const u32 i = i0 + k * 256;
                if (i < ch.n) ch.dst[i] = v[k];
            }
        }
    }
}

// The address at which the device reads host buffer h, or nullptr when it
// cannot (then the copy engine uploads it).
const u64 *device_readable(const u64 *h, bool pageable_ok) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice ||
        a.type == cudaMemoryTypeManaged)
        return static_cast<const u64 *>(a.devicePointer);
    return pageable_ok ? h : nullptr;
}

int status_of(u64 e) {
    return e == 0 ? TC_OK : e == kErrInput ? TC_ERR_INPUT : e == kErrTimeout ? TC_ERR_TIMEOUT
                                                                               : TC_ERR_CUDA;
}

}  // namespace

struct tc_server {
    tc_server_config_t cfg{};
    int dev = 0;
    int depth = 2;
    tc_multi *M = nullptr;
    cudaStream_t cs = nullptr;  // rounds
    cudaStream_t xs = nullptr;  // host -> device batch copies
    cudaMemPool_t pool = nullptr;
    std::chrono::steady_clock::time_point t0;
    u64 fixed = 0;

    // ---- shared with client threads (mu)
    std::mutex mu;
    std::condition_variable cv_in, cv_out;
    std::deque<Req> inbox;
    std::deque<tc_completion_t> done;
    std::unordered_map<u32, bool> handles;  // open handles
    u64 next_ticket = 1;
    u32 next_handle = 1;
    u64 submitted = 0, completed = 0;
    int fatal = TC_OK;
    bool stop = false;
    tc_server_stats_t stats{};

    // ---- scheduler thread only
    std::thread th;
    std::deque<Req> pending;
    std::vector<Slot> slots;
    std::vector<u32> free_slots;
    std::unordered_map<u32, u32> slot_of;  // handle -> slot
    std::deque<u32> ready;                 // slots with queued work, round-robin
    std::deque<Round> inflight;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_free;
    bool pageable_ok = false;  // the device reads pageable host memory
    // upload ring: chunk lists in mapped pinned memory, one kernel per list
    UploadChunk *up_ring = nullptr, *up_ring_dev = nullptr;
    cudaEvent_t up_ev[kUploadSlots] = {};
    int up_slot = 0;
    std::vector<UploadChunk> up_chunks;
    // (index of the batch's last chunk, its copy event): recorded after the
    // launch covering that chunk
    std::vector<std::pair<size_t, int>> up_events;
    u64 copy_seq = 0;
    int nbuf = 0;
    std::vector<u64 *> d_out, h_out, d_desc, h_desc;
    std::vector<u32 *> h_qs;
    // device addresses of the mapped pinned buffers: the round's descriptor
    // and query slots are read, and its records written, by kernels, so no
    // round work waits for a copy engine busy with later rounds' batches
    std::vector<u64 *> h_out_dev, h_desc_dev;
    std::vector<u32 *> h_qs_dev;
    std::vector<cudaEvent_t> round_ev;            // a round's records are back (timing)
    std::vector<cudaEvent_t> ev_start, ev_sort0, ev_sort1;  // its start; its sort phase
    u64 round_no = 0;
    u64 reserved = 0, peak = 0;
    int err = TC_OK;          // first CUDA failure seen by the scheduler
    bool dirty = false;       // arrivals or freed slots/memory since the last admission pass
    tc_server_stats_t local{};
    std::vector<tc_completion_t> outbox;

    u64 now() const {
        return (u64)std::chrono::duration_cast<std::chrono::nanoseconds>(
                   std::chrono::steady_clock::now() - t0)
            .count();
    }
    void run();
    bool admit();
    bool form_round();
    bool retire();
    void publish();
    void fail_all(int code);
    int get_event();
    void complete(const Req &q, int status, const u64 *rec);
    void note_round_time(const Round &R);
    bool flush_uploads();
};

void tc_server::complete(const Req &q, int status, const u64 *rec) {
    tc_completion_t c{};
    c.ticket = q.ticket;
    c.handle = q.handle;
    c.kind = q.kind;
    c.status = status;
    if (rec) {
        c.batches = rec[1];
        c.sum_lo = rec[2];
        c.sum_hi = rec[3];
        c.n_closed = rec[4];
        c.m = rec[5];
        if (q.r) {
            tc_estimate_t e;
            finish_estimate(c.sum_lo, c.sum_hi, c.n_closed, c.m, q.r, c.batches, &e);
            c.num_lo = e.num_lo;
            c.num_hi = e.num_hi;
            c.tau_hat = e.tau_hat;
        }
    }
    c.t_submit_ns = q.t_submit;
    c.t_admit_ns = q.t_admit;
    c.t_round_ns = q.t_round;
    c.t_done_ns = now();
    outbox.push_back(c);
}

int tc_server::get_event() {
    if (ev_free.empty()) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return -1;
        ev_pool.push_back(e);
        return (int)ev_pool.size() - 1;
    }
    const int k = ev_free.back();
    ev_free.pop_back();
    return k;
}

// Admit what can be admitted, in arrival order.  An open needs a free slot
// and its state bytes, a batch its own bytes; once an open (a batch) has to
// wait, no later open (batch) overtakes it.  Queries, closes and empty
// batches of admitted streams need nothing and pass waiting requests of
// other streams -- a close may be what frees the slot an open waits for --
// but no request overtakes an earlier one of its own stream.  Returns
// whether anything was admitted; a CUDA failure is left in `err`.
bool tc_server::admit() {
    const NvtxRange range("tc server admit");
    if (pending.empty() || !dirty) return false;
    dirty = false;
    bool moved = false, open_blocked = false, mem_blocked = false;
    std::unordered_set<u32> held;  // handles with an earlier request still waiting
    std::deque<Req> keep;
    while (!pending.empty()) {
        Req q = std::move(pending.front());
        pending.pop_front();
        bool wait = held.count(q.handle) != 0;
        if (!wait && q.kind == TC_REQ_OPEN) {
            const u64 b = state_bytes_for(q.r);
            wait = open_blocked || free_slots.empty() || reserved + b > cfg.budget_bytes;
            if (wait) {
                open_blocked = true;
            } else {
                void *p = nullptr;
                if (cudaMallocFromPoolAsync(&p, b, pool, cs) != cudaSuccess) {
                    err = TC_ERR_NOMEM;
                    pending.push_front(std::move(q));
                    break;
                }
                const u32 s = free_slots.back();
                free_slots.pop_back();
                if (multi_open_slot(M, s, q.r, q.seed, q.stream_id, p, cs) != TC_OK) {
                    err = TC_ERR_CUDA;
                    pending.push_front(std::move(q));
                    break;
                }
                Slot &sl = slots[s];
                sl.handle = q.handle;
                sl.r = q.r;
                sl.state = p;
                sl.state_bytes = b;
                sl.used = true;
                slot_of[q.handle] = s;
                reserved += b;
                q.t_admit = now();
                local.opens++;
                local.streams_open++;
                complete(q, TC_OK, nullptr);
            }
        } else if (!wait) {
            if (q.kind == TC_REQ_BATCH && q.w > 0) {
                const u64 b = round_up(8 * q.w);
                wait = mem_blocked || reserved + b > cfg.budget_bytes;
                if (wait) {
                    mem_blocked = true;
                } else {
                    if (cudaMallocFromPoolAsync((void **)&q.d_edges, 8 * q.w, pool, xs) !=
                        cudaSuccess) {
                        err = TC_ERR_NOMEM;
                        pending.push_front(std::move(q));
                        break;
                    }
                    q.ev = get_event();
                    bool ok = q.ev >= 0;
                    if (ok && q.h_dev) {
                        // uploaded by this pass's kernel; its event follows it
                        for (u64 o = 0; o < q.w; o += kUploadWords)
                            up_chunks.push_back(UploadChunk{
                                q.h_dev + o, q.d_edges + o,
                                (u32)std::min<u64>(kUploadWords, q.w - o), 0u});
                        up_events.emplace_back(up_chunks.size() - 1, q.ev);
                    } else if (ok) {
                        ok = cudaMemcpyAsync(q.d_edges, q.h_edges, 8 * q.w,
                                             cudaMemcpyHostToDevice, xs) == cudaSuccess &&
                             cudaEventRecord(ev_pool[q.ev], xs) == cudaSuccess;
                    }
                    if (!ok) {
                        err = TC_ERR_CUDA;
                        pending.push_front(std::move(q));
                        break;
                    }
                    q.bytes = b;
                    q.seq = ++copy_seq;
                    reserved += b;
                }
            }
            if (!wait) {
                q.t_admit = now();
                const u32 s = slot_of.at(q.handle);
                Slot &sl = slots[s];
                sl.q.push_back(std::move(q));
                if (!sl.in_ready) {
                    sl.in_ready = true;
                    ready.push_back(s);
                }
            }
        }
        if (wait) {
            if (!q.waited) local.admission_waits++;
            q.waited = true;
            held.insert(q.handle);
            keep.push_back(std::move(q));
        } else {
            moved = true;
            if (reserved > peak) peak = reserved;
        }
    }
    while (!keep.empty()) {  // waiting requests go back in arrival order
        pending.push_front(std::move(keep.back()));
        keep.pop_back();
    }
    if (!flush_uploads() && err == TC_OK) err = TC_ERR_CUDA;
    return moved;
}

// Launch the upload kernels for the chunks gathered by this pass on the copy
// stream, recording each uploaded batch's copy event behind the launch that
// covers its last chunk.
bool tc_server::flush_uploads() {
    bool ok = true;
    size_t done_chunks = 0, next_ev = 0;
    while (ok && done_chunks < up_chunks.size()) {
        const int k = up_slot;
        up_slot = (up_slot + 1) % kUploadSlots;
        // the slot's previous list has been read once its kernels finished
        ok &= cudaEventSynchronize(up_ev[k]) == cudaSuccess;
        const u32 n = (u32)std::min<size_t>(kUploadChunks, up_chunks.size() - done_chunks);
        UploadChunk *list = up_ring + (size_t)k * kUploadChunks;
        const UploadChunk *list_dev = up_ring_dev + (size_t)k * kUploadChunks;
        std::memcpy(list, up_chunks.data() + done_chunks, n * sizeof(UploadChunk));
        for (u32 g = 0; g < n && ok; g += kUploadGroup) {
            const u32 m = std::min<u32>(kUploadGroup, n - g);
            upload_kernel<<<m, 256, 0, xs>>>(list_dev + g, m);
            ok &= cudaGetLastError() == cudaSuccess;
            const size_t end = done_chunks + g + m;  // chunks uploaded so far
            while (ok && next_ev < up_events.size() && up_events[next_ev].first < end)
                ok &= cudaEventRecord(ev_pool[up_events[next_ev++].second], xs) == cudaSuccess;
        }
        ok &= ok && cudaEventRecord(up_ev[k], xs) == cudaSuccess;
        done_chunks += n;
    }
    up_chunks.clear();
    up_events.clear();
    return ok;
}

bool tc_server::form_round() {
    const NvtxRange range("tc server round");
    if (ready.empty()) return false;
    const u32 S = M->S;
    Round R;
    std::vector<RoundItem> items;
    std::vector<u32> qslots;
    std::vector<u32> closed_slots;
    u64 edges = 0, wait_seq = 0;
    int wait_ev = -1;
    std::deque<u32> again;
    size_t n = ready.size();
    bool full = false;
    while (n-- > 0 && !full) {
        const u32 s = ready.front();
        ready.pop_front();
        Slot &sl = slots[s];
        sl.in_ready = false;
        bool closing = false;
        while (!sl.q.empty()) {
            Req &h = sl.q.front();
            if (h.kind == TC_REQ_QUERY || (h.kind == TC_REQ_BATCH && h.w == 0)) {
                if (qslots.size() >= S) {
                    full = true;
                    break;
                }
                qslots.push_back(s);
                h.r = sl.r;
                R.queries.push_back(std::move(h));
                sl.q.pop_front();
                continue;
            }
            if (h.kind == TC_REQ_CLOSE) {
                R.closes.push_back(std::move(h));
                sl.q.pop_front();
                closing = true;
                break;
            }
            // a batch: at most one per stream per round; queries behind it
            // wait for the next round (they must see this batch)
            if (edges + h.w > cfg.w_max_round || items.size() >= cfg.max_round_streams) {
                full = true;
                break;
            }
            items.push_back(RoundItem{s, h.d_edges, h.w});
            edges += h.w;
            if (h.seq > wait_seq) {
                wait_seq = h.seq;
                wait_ev = h.ev;
            }
            h.r = sl.r;
            R.batches.push_back(std::move(h));
            sl.q.pop_front();
            break;
        }
        if (closing) {
            closed_slots.push_back(s);
        } else if (!sl.q.empty()) {
            sl.in_ready = true;
            if (full) ready.push_front(s);
            else again.push_back(s);
        }
    }
    for (u32 s : again) ready.push_back(s);
    if (items.empty() && qslots.empty() && R.closes.empty()) return false;
    {
        const u64 t = now();
        for (Req &q : R.queries) q.t_round = t;
        for (Req &q : R.batches) q.t_round = t;
        for (Req &q : R.closes) q.t_round = t;
    }

    const int b = (int)(round_no % (u64)nbuf);
    const u32 Q = (u32)qslots.size(), K = (u32)items.size();
    bool ok = cudaEventRecord(ev_start[b], cs) == cudaSuccess;
    if (Q && ok) {
        std::memcpy(h_qs[b], qslots.data(), Q * sizeof(u32));
        ok &= multi_gather(M, h_qs_dev[b], Q, d_out[b], cs) == TC_OK;
    }
    if (K && ok) {
        // pipelined: the round is sorted on the engine's own streams as soon as
        // its batches' copies have landed, beside the previous round's sweep;
        // its sweep and records are ordered on cs
        write_descriptor(M, items.data(), K, h_desc[b]);
        ok &= multi_enqueue(M, items.data(), K, d_desc[b], h_desc_dev[b],
                            d_out[b] + (u64)Q * kRecordWords, cs, true,
                            wait_ev >= 0 ? ev_pool[wait_ev] : nullptr, ev_sort0[b],
                            ev_sort1[b]) == TC_OK;
        for (Req &q : R.batches) {
            ok &= ok && cudaFreeAsync(q.d_edges, cs) == cudaSuccess;
            q.d_edges = nullptr;
            ev_free.push_back(q.ev);
            q.ev = -1;
        }
    }
    const u64 words = (u64)(Q + K) * kRecordWords;
    if (words && ok) ok &= copy_words_async(M, h_out_dev[b], d_out[b], words, cs) == TC_OK;
    for (u32 s : closed_slots) {
        Slot &sl = slots[s];
        ok &= ok && cudaFreeAsync(sl.state, cs) == cudaSuccess;
        reserved -= sl.state_bytes;
        slot_of.erase(sl.handle);
        sl.state = nullptr;
        sl.state_bytes = 0;
        sl.used = false;
        free_slots.push_back(s);
        dirty = true;
        local.closes++;
        local.streams_open--;
    }
    ok &= ok && cudaEventRecord(round_ev[b], cs) == cudaSuccess;
    if (!ok) {
        err = TC_ERR_CUDA;
        return false;
    }
    R.buf = b;
    R.sorted = K > 0;
    inflight.push_back(std::move(R));
    round_no++;
    local.rounds++;
    local.edges += edges;
    if (edges > local.max_round_edges) local.max_round_edges = edges;
    if (K > local.max_round_streams) local.max_round_streams = K;
    return true;
}

// Device time of a finished round and, for the longest so far, its split.
void tc_server::note_round_time(const Round &R) {
    const int b = R.buf;
    auto ns = [](cudaEvent_t a, cudaEvent_t z) -> u64 {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, z) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return ms > 0.f ? (u64)((double)ms * 1e6) : 0;
    };
    const u64 total = ns(ev_start[b], round_ev[b]);
    if (total > 5000000) local.rounds_gpu_over_5ms++;
    if (total <= local.round_gpu_max_ns) return;
    local.round_gpu_max_ns = total;
    if (R.sorted) {
        local.round_max_wait_ns = ns(ev_start[b], ev_sort0[b]);
        local.round_max_sort_ns = ns(ev_sort0[b], ev_sort1[b]);
        local.round_max_sweep_ns = ns(ev_sort1[b], round_ev[b]);
    } else {
        local.round_max_wait_ns = local.round_max_sort_ns = local.round_max_sweep_ns = 0;
    }
}

bool tc_server::retire() {
    bool any = false;
    while (!inflight.empty()) {
        Round &R = inflight.front();
        const cudaError_t e = cudaEventQuery(round_ev[R.buf]);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) {
            err = TC_ERR_CUDA;
            return any;
        }
        note_round_time(R);
        const u64 *o = h_out[R.buf];
        const size_t Q = R.queries.size();
        for (size_t i = 0; i < Q; ++i) {
            complete(R.queries[i], TC_OK, o + i * kRecordWords);
            local.queries++;
        }
        for (size_t k = 0; k < R.batches.size(); ++k) {
            const u64 *rec = o + (Q + k) * kRecordWords;
            const int st = status_of(rec[0]);
            complete(R.batches[k], st, rec);
            reserved -= R.batches[k].bytes;
            dirty = true;
            if (st) local.rejected++;
            else local.batches++;
        }
        for (const Req &q : R.closes) complete(q, TC_OK, nullptr);
        inflight.pop_front();
        any = true;
    }
    return any;
}

// Hand the completions gathered by this pass to the clients.
void tc_server::publish() {
    std::lock_guard<std::mutex> lk(mu);
    local.kernel_launches = M->launches;
    local.bytes_reserved = reserved;
    local.bytes_peak = peak;
    local.requests_waiting = pending.size() + inbox.size();
    stats = local;
    stats.bytes_budget = cfg.budget_bytes;
    stats.bytes_fixed = fixed;
    if (!outbox.empty()) {
        for (const tc_completion_t &c : outbox) done.push_back(c);
        completed += outbox.size();
        outbox.clear();
        cv_out.notify_all();
    }
}

// After a CUDA error: every request not yet completed fails with `code`.
void tc_server::fail_all(int code) {
    cudaStreamSynchronize(cs);
    cudaStreamSynchronize(xs);
    for (Round &R : inflight) {
        for (const Req &q : R.queries) complete(q, code, nullptr);
        for (const Req &q : R.batches) complete(q, code, nullptr);
        for (const Req &q : R.closes) complete(q, code, nullptr);
    }
    inflight.clear();
    for (Slot &sl : slots) {
        for (const Req &q : sl.q) complete(q, code, nullptr);
        sl.q.clear();
    }
    ready.clear();
    for (const Req &q : pending) complete(q, code, nullptr);
    pending.clear();
}

void tc_server::run() {
    cudaSetDevice(dev);
    u64 t_prev = now();
    u64 t_full = 0;  // since when `depth` rounds have been in flight (0: not full)
    for (;;) {
        {
            // the longest stretch with every round slot busy: the scheduler
            // waiting for the GPU to finish a round
            const u64 t = now();
            if ((int)inflight.size() >= depth) {
                if (!t_full) t_full = t;
                if (t - t_full > local.inflight_full_max_ns) local.inflight_full_max_ns = t - t_full;
            } else {
                t_full = 0;
            }
        }
        {
            // the longest stretch between two scheduler passes with work in
            // flight or waiting: where the scheduler thread itself stalled
            const u64 t = now();
            if (!inflight.empty() || !pending.empty()) {
                const u64 gap = t - t_prev;
                if (gap > local.sched_gap_max_ns) local.sched_gap_max_ns = gap;
                if (gap > 5000000) local.sched_gaps_over_5ms++;
            }
            t_prev = t;
        }
        bool stopping;
        {
            std::lock_guard<std::mutex> lk(mu);
            stopping = stop;
            if (!inbox.empty()) dirty = true;
            while (!inbox.empty()) {
                pending.push_back(std::move(inbox.front()));
                inbox.pop_front();
            }
        }
        if (stopping) break;
        if (err == TC_OK) {
            bool progress = retire();
            if (err == TC_OK) progress |= admit();
            while (err == TC_OK && (int)inflight.size() < depth && form_round()) progress = true;
            if (err != TC_OK) {
                {
                    std::lock_guard<std::mutex> lk(mu);
                    fatal = err;
                }
                fail_all(err);
            }
            publish();
            if (!progress && err == TC_OK) {
                std::unique_lock<std::mutex> lk(mu);
                const auto budget = std::chrono::microseconds(inflight.empty() ? 500 : 10);
                const u64 t_wait = now();
                cv_in.wait_for(lk, budget, [&] { return stop || !inbox.empty(); });
                // a wait up to its budget is the scheduler's own choice; only
                // time beyond it (the thread not running) counts as a gap
                const u64 waited = now() - t_wait;
                const u64 allowed = (u64)std::chrono::nanoseconds(budget).count();
                t_prev += waited < allowed ? waited : allowed;
            }
            continue;
        }
        // after a failure every request still arriving completes with it
        for (const Req &q : pending) complete(q, err, nullptr);
        pending.clear();
        publish();
        std::unique_lock<std::mutex> lk(mu);
        cv_in.wait(lk, [&] { return stop || !inbox.empty(); });
    }
    // leaving: let the rounds in flight finish before their memory goes
    cudaStreamSynchronize(xs);
    cudaStreamSynchronize(cs);
}

static void server_free(tc_server *S) {
    if (S->cs) cudaStreamSynchronize(S->cs);
    if (S->xs) cudaStreamSynchronize(S->xs);
    for (Slot &sl : S->slots) {
        for (Req &q : sl.q)
            if (q.d_edges) cudaFreeAsync(q.d_edges, S->cs);
        if (sl.state) cudaFreeAsync(sl.state, S->cs);
    }
    for (Req &q : S->pending)
        if (q.d_edges) cudaFreeAsync(q.d_edges, S->cs);
    if (S->cs) cudaStreamSynchronize(S->cs);
    for (int k = 0; k < S->nbuf; ++k) {
        cudaFree(S->d_out[k]);
        cudaFree(S->d_desc[k]);
        if (S->h_out[k]) cudaFreeHost(S->h_out[k]);
        if (S->h_desc[k]) cudaFreeHost(S->h_desc[k]);
        if (S->h_qs[k]) cudaFreeHost(S->h_qs[k]);
        if (S->round_ev[k]) cudaEventDestroy(S->round_ev[k]);
        if (S->ev_start[k]) cudaEventDestroy(S->ev_start[k]);
        if (S->ev_sort0[k]) cudaEventDestroy(S->ev_sort0[k]);
        if (S->ev_sort1[k]) cudaEventDestroy(S->ev_sort1[k]);
    }
    for (cudaEvent_t e : S->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : S->up_ev)
        if (e) cudaEventDestroy(e);
    if (S->up_ring) cudaFreeHost(S->up_ring);
    if (S->M) multi_free(S->M);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    if (S->cs) cudaStreamDestroy(S->cs);
    if (S->xs) cudaStreamDestroy(S->xs);
    delete S;
}

extern "C" {

int tc_server_create(const tc_server_config_t *cfg, tc_server **out) {
    if (!cfg || !out) return TC_ERR_INVAL;
    *out = nullptr;
    if (cfg->max_streams == 0 || cfg->depth > 8 || cfg->w_max_round == 0) return TC_ERR_INVAL;
    const u32 S = cfg->max_streams;
    // two rounds in flight unless asked: a round's sorts run beside the
    // previous round's sweep (8.51 against 7.80 G edges/s at saturation,
    // with p99 batch latency at 70% load of 1.3-4.3 ms against 1.5-2.4 ms
    // with one, on one box)
    const int depth = cfg->depth ? (int)cfg->depth : 2;
    const int nbuf = depth + 1;
    const u64 ring_bytes = (u64)nbuf * (2ull * S * kRecordWords * 8 + desc_words(S) * 8);
    const u64 fixed = multi_scratch_bytes(S, cfg->w_max_round, cfg->vertex_bits, 2) + ring_bytes;
    if (fixed >= cfg->budget_bytes) return TC_ERR_RANGE;

    tc_server *Sv = new (std::nothrow) tc_server();
    if (!Sv) return TC_ERR_NOMEM;
    Sv->cfg = *cfg;
    if (Sv->cfg.max_round_streams == 0 || Sv->cfg.max_round_streams > S)
        Sv->cfg.max_round_streams = S;
    Sv->depth = depth;
    Sv->nbuf = nbuf;
    Sv->fixed = fixed;
    Sv->reserved = fixed;
    Sv->peak = fixed;
    Sv->t0 = std::chrono::steady_clock::now();
    int rc = TC_OK;
    if (cudaGetDevice(&Sv->dev) != cudaSuccess) rc = TC_ERR_CUDA;
    if (!rc) rc = multi_alloc(S, cfg->w_max_round, cfg->vertex_bits, &Sv->M, 2);
    bool ok = rc == TC_OK;
    ok &= ok && cudaStreamCreateWithFlags(&Sv->cs, cudaStreamNonBlocking) == cudaSuccess;
    ok &= ok && cudaStreamCreateWithFlags(&Sv->xs, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = Sv->dev;
        ok &= cudaMemPoolCreate(&Sv->pool, &props) == cudaSuccess;
        u64 keep = ~0ull;
        int no = 0;
        ok &= ok && cudaMemPoolSetAttribute(Sv->pool, cudaMemPoolAttrReleaseThreshold, &keep) ==
                        cudaSuccess;
        // never make the copy stream wait for the compute stream to reuse memory
        ok &= ok && cudaMemPoolSetAttribute(Sv->pool, cudaMemPoolReuseAllowInternalDependencies,
                                            &no) == cudaSuccess;
        // map the pool's memory up front (up to 16 GB of the budget): growing
        // it while requests wait would stall the scheduler thread; the pool
        // keeps what it maps (release threshold: everything)
        const u64 warm = std::min<u64>(cfg->budget_bytes - fixed, kPoolWarmBytes);
        void *wp = nullptr;
        if (ok && warm && cudaMallocFromPoolAsync(&wp, warm, Sv->pool, Sv->cs) == cudaSuccess) {
            ok &= cudaFreeAsync(wp, Sv->cs) == cudaSuccess;
            ok &= ok && cudaStreamSynchronize(Sv->cs) == cudaSuccess;
        } else {
            cudaGetLastError();  // not enough memory to warm: the pool grows on demand
        }
    }
    Sv->d_out.assign(nbuf, nullptr);
    Sv->h_out.assign(nbuf, nullptr);
    Sv->d_desc.assign(nbuf, nullptr);
    Sv->h_desc.assign(nbuf, nullptr);
    Sv->h_qs.assign(nbuf, nullptr);
    Sv->round_ev.assign(nbuf, nullptr);
    Sv->h_out_dev.assign(nbuf, nullptr);
    Sv->h_desc_dev.assign(nbuf, nullptr);
    Sv->h_qs_dev.assign(nbuf, nullptr);
    Sv->ev_start.assign(nbuf, nullptr);
    Sv->ev_sort0.assign(nbuf, nullptr);
    Sv->ev_sort1.assign(nbuf, nullptr);
    for (int k = 0; k < nbuf && ok; ++k) {
        const u64 ob = 2ull * S * kRecordWords * 8;
        ok &= cudaMalloc(&Sv->d_out[k], ob) == cudaSuccess;
        ok &= ok && cudaHostAlloc(&Sv->h_out[k], ob, cudaHostAllocMapped) == cudaSuccess;
        ok &= ok && cudaMalloc(&Sv->d_desc[k], desc_words(S) * 8) == cudaSuccess;
        ok &= ok && cudaHostAlloc(&Sv->h_desc[k], desc_words(S) * 8, cudaHostAllocMapped) ==
                        cudaSuccess;
        ok &= ok && cudaHostAlloc(&Sv->h_qs[k], S * 4, cudaHostAllocMapped) == cudaSuccess;
        if (ok) {
            Sv->h_out_dev[k] = static_cast<u64 *>(mapped_device_ptr(Sv->h_out[k]));
            Sv->h_desc_dev[k] = static_cast<u64 *>(mapped_device_ptr(Sv->h_desc[k]));
            Sv->h_qs_dev[k] = static_cast<u32 *>(mapped_device_ptr(Sv->h_qs[k]));
            ok &= Sv->h_out_dev[k] && Sv->h_desc_dev[k] && Sv->h_qs_dev[k];
        }
        // timing events: the stats report each round's device time
        ok &= ok && cudaEventCreate(&Sv->round_ev[k]) == cudaSuccess;
        ok &= ok && cudaEventCreate(&Sv->ev_start[k]) == cudaSuccess;
        ok &= ok && cudaEventCreate(&Sv->ev_sort0[k]) == cudaSuccess;
        ok &= ok && cudaEventCreate(&Sv->ev_sort1[k]) == cudaSuccess;
    }
    if (!ok) {
        if (rc == TC_OK) rc = cudaGetLastError() == cudaErrorMemoryAllocation ? TC_ERR_NOMEM
                                                                              : TC_ERR_CUDA;
        server_free(Sv);
        return rc;
    }
    if (ok) {
        int pma = 0;
        if (cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, Sv->dev) == cudaSuccess)
            Sv->pageable_ok = pma != 0;
        cudaGetLastError();
        ok &= cudaHostAlloc(&Sv->up_ring, (size_t)kUploadSlots * kUploadChunks * sizeof(UploadChunk),
                            cudaHostAllocMapped) == cudaSuccess;
        Sv->up_ring_dev = ok ? static_cast<UploadChunk *>(mapped_device_ptr(Sv->up_ring)) : nullptr;
        ok &= Sv->up_ring_dev != nullptr;
        for (int k = 0; k < kUploadSlots && ok; ++k)
            ok &= cudaEventCreateWithFlags(&Sv->up_ev[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            server_free(Sv);
            return TC_ERR_CUDA;
        }
    }
    Sv->slots.resize(S);
    Sv->free_slots.reserve(S);
    for (u32 s = S; s-- > 0;) Sv->free_slots.push_back(s);
    try {
        Sv->th = std::thread([Sv] { Sv->run(); });
    } catch (...) {
        server_free(Sv);
        return TC_ERR_NOMEM;
    }
    *out = Sv;
    return TC_OK;
}

static int submit(tc_server *S, Req &&q, uint64_t *ticket) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal) return S->fatal;
    q.ticket = S->next_ticket++;
    q.t_submit = S->now();
    if (ticket) *ticket = q.ticket;
    S->inbox.push_back(std::move(q));
    S->submitted++;
    S->cv_in.notify_one();
    return TC_OK;
}

int tc_server_open(tc_server *S, uint64_t r, uint64_t seed, uint32_t stream_id,
                   uint32_t *handle, uint64_t *ticket) {
    if (!S || !handle || r == 0 || r > 0xFFFFFFFFull) return TC_ERR_INVAL;
    if (S->fixed + state_bytes_for(r) > S->cfg.budget_bytes) return TC_ERR_RANGE;
    Req q;
    q.kind = TC_REQ_OPEN;
    q.r = r;
    q.seed = seed;
    q.stream_id = stream_id;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->fatal) return S->fatal;
        q.handle = S->next_handle++;
        S->handles[q.handle] = true;
    }
    *handle = q.handle;
    return submit(S, std::move(q), ticket);
}

static bool handle_open(tc_server *S, uint32_t handle, bool closing) {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->handles.find(handle);
    if (it == S->handles.end()) return false;
    if (closing) S->handles.erase(it);
    return true;
}

int tc_server_submit(tc_server *S, uint32_t handle, const uint64_t *h_edges, uint64_t w,
                     uint64_t *ticket) {
    if (!S || (w && !h_edges)) return TC_ERR_INVAL;
    if (w > S->cfg.w_max_round || w > (1ull << 28) ||
        S->fixed + round_up(8 * w) > S->cfg.budget_bytes)
        return TC_ERR_RANGE;
    if (!handle_open(S, handle, false)) return TC_ERR_INVAL;
    Req q;
    q.kind = TC_REQ_BATCH;
    q.handle = handle;
    q.h_edges = h_edges;
    q.h_dev = w ? device_readable(h_edges, S->pageable_ok) : nullptr;
    q.w = w;
    return submit(S, std::move(q), ticket);
}

int tc_server_query(tc_server *S, uint32_t handle, uint64_t *ticket) {
    if (!S) return TC_ERR_INVAL;
    if (!handle_open(S, handle, false)) return TC_ERR_INVAL;
    Req q;
    q.kind = TC_REQ_QUERY;
    q.handle = handle;
    return submit(S, std::move(q), ticket);
}

int tc_server_submit_many(tc_server *S, uint32_t n, const uint32_t *kinds,
                          const uint32_t *handles, const uint64_t *const *h_edges,
                          const uint64_t *w, uint64_t *tickets) {
    if (!S) return TC_ERR_INVAL;
    if (n == 0) return TC_OK;
    if (!kinds || !handles || !tickets) return TC_ERR_INVAL;
    for (u32 i = 0; i < n; ++i) {
        if (kinds[i] == TC_REQ_BATCH) {
            if (!w || !h_edges || (w[i] && !h_edges[i])) return TC_ERR_INVAL;
            if (w[i] > S->cfg.w_max_round || w[i] > (1ull << 28) ||
                S->fixed + round_up(8 * w[i]) > S->cfg.budget_bytes)
                return TC_ERR_RANGE;
        } else if (kinds[i] != TC_REQ_QUERY) {
            return TC_ERR_INVAL;
        }
    }
    // where the device reads each batch, found before taking the lock
    std::vector<const u64 *> dev(n, nullptr);
    for (u32 i = 0; i < n; ++i)
        if (kinds[i] == TC_REQ_BATCH && w[i]) dev[i] = device_readable(h_edges[i], S->pageable_ok);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal) return S->fatal;
    for (u32 i = 0; i < n; ++i)
        if (S->handles.find(handles[i]) == S->handles.end()) return TC_ERR_INVAL;
    const u64 t = S->now();
    for (u32 i = 0; i < n; ++i) {
        Req q;
        q.kind = kinds[i];
        q.handle = handles[i];
        if (q.kind == TC_REQ_BATCH) {
            q.h_edges = h_edges[i];
            q.h_dev = dev[i];
            q.w = w[i];
        }
        q.ticket = S->next_ticket++;
        q.t_submit = t;
        tickets[i] = q.ticket;
        S->inbox.push_back(std::move(q));
    }
    S->submitted += n;
    S->cv_in.notify_one();
    return TC_OK;
}

int tc_server_close(tc_server *S, uint32_t handle, uint64_t *ticket) {
    if (!S) return TC_ERR_INVAL;
    if (!handle_open(S, handle, true)) return TC_ERR_INVAL;
    Req q;
    q.kind = TC_REQ_CLOSE;
    q.handle = handle;
    return submit(S, std::move(q), ticket);
}

int tc_server_poll(tc_server *S, tc_completion_t *out, uint32_t max_n, uint32_t wait_us,
                   uint32_t *n_out) {
    if (!S || !n_out || (max_n && !out)) return TC_ERR_INVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_us)
        S->cv_out.wait_for(lk, std::chrono::microseconds(wait_us),
                           [&] { return !S->done.empty(); });
    u32 n = 0;
    while (n < max_n && !S->done.empty()) {
        out[n++] = S->done.front();
        S->done.pop_front();
    }
    *n_out = n;
    return TC_OK;
}

int tc_server_drain(tc_server *S, uint32_t timeout_ms) {
    if (!S) return TC_ERR_INVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    const bool ok = S->cv_out.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        return S->completed == S->submitted;
    });
    if (!ok) return TC_ERR_TIMEOUT;
    return S->fatal;
}

int tc_server_stats(tc_server *S, tc_server_stats_t *out) {
    if (!S || !out) return TC_ERR_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    out->bytes_budget = S->cfg.budget_bytes;
    out->bytes_fixed = S->fixed;
    unsigned long long v = 0;  // the runtime reports these attributes as 64-bit values
    if (cudaMemPoolGetAttribute(S->pool, cudaMemPoolAttrReservedMemHigh, &v) == cudaSuccess)
        out->pool_reserved_high = (uint64_t)v;
    if (cudaMemPoolGetAttribute(S->pool, cudaMemPoolAttrUsedMemHigh, &v) == cudaSuccess)
        out->pool_used_high = (uint64_t)v;
    return TC_OK;
}

void tc_server_destroy(tc_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_in.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    server_free(S);
}

}  // extern "C"
