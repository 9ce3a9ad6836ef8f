// Host side of the C ABI declared in include/tc.h: context lifetime, the
// per-batch launch sequence of bulkUpdateAll (Sec. 4), the estimate of
// Lemma 3.1, stage timing and the standalone rankAll (Lemma 4.3).
#include <algorithm>
#include <chrono>
#include <random>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "tc_kernels.cuh"
#include "tc_nvtx.h"

using namespace tc;

static cudaError_t &last_cuda_error() {
    static thread_local cudaError_t e = cudaSuccess;
    return e;
}

#define TC_CUDA(call)                \
    do {                             \
        cudaError_t e_ = (call);     \
        if (e_ != cudaSuccess) {     \
            last_cuda_error() = e_;  \
            return TC_ERR_CUDA;      \
        }                            \
    } while (0)

namespace {

constexpr u64 kMaxBatch = 1ull << 28;
constexpr u64 kDefaultWMax = 1ull << 22;
constexpr size_t kEventPool = 8192;

enum Stage { kStart = -1, kPrep = 0, kArcSort, kEdgeSort, kDups, kSweep, kFinish, kEstimate,
             kStages };

using PassFn = void (*)(u64 *, u64 *, u32 *, u32 *, u32, u32, u32, int, SortPlan *, u32 *, u32 *,
                        Control *);

struct PassKernel {
    PassFn fn;
    size_t smem;
    int threads;
};

template <int kBits, bool kValues, int kRank>
void pass_variant(PassKernel &k) {
    k.fn = onesweep_pass_kernel<kBits, kValues, kRank>;
    k.smem = sizeof(OnesweepSmem<kBits, kValues, kRank>);
    k.threads = OnesweepShape<kBits>::kThreads;
}

// The onesweep instantiation for a digit width, value payload and ranking.
// Atomic-or ranking keeps a mask word per (warp, digit) twice over, which
// only fits shared memory for 8-bit digits; wider digits use match.any.
PassKernel select_pass(u32 bits, bool values, int rank) {
    PassKernel k{};
#define TC_PASS_RANK(B, V)                                                   \
    if (rank == kRankBallot) pass_variant<B, V, kRankBallot>(k);             \
    else if (rank == kRankMatch || B > 8) pass_variant<B, V, kRankMatch>(k); \
    else pass_variant<B, V, (B > 8 ? kRankMatch : kRankAtomicOr)>(k);
#define TC_PASS_CASE(B)           \
    case B:                       \
        if (values) {             \
            TC_PASS_RANK(B, true)  \
        } else {                  \
            TC_PASS_RANK(B, false) \
        }                         \
        return k;
    switch (bits) {
        TC_PASS_CASE(8)
        TC_PASS_CASE(9)
        TC_PASS_CASE(10)
        default:
        TC_PASS_CASE(11)
    }
#undef TC_PASS_CASE
#undef TC_PASS_RANK
}

constexpr u32 kDigitChoices[4] = {8, 9, 10, 11};

int configure_kernels() {
    static bool done[64] = {false};
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && done[dev]) return TC_OK;
    for (u32 bits : kDigitChoices)
        for (int v = 0; v < 2; ++v)
            for (int mt = 0; mt < 3; ++mt) {
                const PassKernel k = select_pass(bits, v, mt);
                TC_CUDA(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)k.smem));
            }
    TC_CUDA(cudaFuncSetAttribute(prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
    if (dev < 64) done[dev] = true;
    return TC_OK;
}

}  // namespace

// A fresh key for the Step-3 edge hash, from the OS's entropy source (with a
// clock-based fallback where none is available).  Results never depend on it.
u64 tc::random_hash_key() {
    u64 k = 0;
    try {
        std::random_device rd;
        k = ((u64)rd() << 32) ^ (u64)rd();
    } catch (...) {
    }
    if (!k) k = (u64)std::chrono::steady_clock::now().time_since_epoch().count() *
                0x9E3779B97F4A7C15ull;
    return k;
}

namespace {

// Digit width and pass count for `live` key bits: 8-bit digits unless
// tc_tune forced another width.  On GB300 the 8-bit passes measured fastest:
// a wider digit saves passes but each pass costs more than it saves (at
// 25-bit ids three 9-bit arc passes took 1.05 ms per batch against 0.95 ms
// for four 8-bit ones, the last of which ranks one live bit; 10- and 11-bit
// passes run at 2 or 3 blocks per SM for their shared-memory counters).
u32 pick_digits(u32 live, u32 forced, int &passes) {
    const u32 bits = forced ? forced : 8;
    passes = (int)((live + bits - 1) / bits);
    if (passes < 1) passes = 1;
    return bits;
}

// Bits of the Step-3 hash-bucket directory for batches of w edges: about
// w/4 buckets, so a bucket holds a handful of keys.
u32 hash_bucket_bits(u64 w) {
    const u32 bw = bits_for(w - 1);
    return bw > 3 ? bw - 2 : 1;
}

BatchShape make_shape(u64 w, u32 B, u32 force_a = 0, u32 force_e = 0, u64 hkey = 0) {
    BatchShape s{};
    s.hkey = hkey;
    s.w = (u32)w;
    s.bw = bits_for(w - 1);
    s.B = B;
    s.sha = s.bw + 1;
    s.hb = hash_bucket_bits(w);
    s.bits_a = pick_digits(B, force_a, s.npa);
    // the Step-3 keys sort on whole digits covering the bucket bits, at
    // most the 32 hash bits
    s.bits_e = pick_digits(s.hb, force_e, s.npe);
    s.hs = std::min(32u, (u32)s.npe * s.bits_e);
    s.she = s.bw + 32 - s.hs;
    return s;
}

u64 tiles_of(u64 n) { return (n + kSortTile - 1) / kSortTile; }

// Look-back words of one digit pass over n keys with `bits`-bit digits.
u64 pass_lookback_words(u64 n, u32 bits) {
    return (u64)lookback_stride((u32)tiles_of(n)) << bits;
}

// Words of look-back status for one batch of w edges.
u64 lookback_words(const BatchShape &s, bool edges) {
    u64 words = (u64)s.npa * pass_lookback_words(2ull * s.w, s.bits_a);
    if (edges) words += (u64)s.npe * pass_lookback_words(s.w, s.bits_e);
    return words;
}

// Largest look-back need over every digit width a context may use.
u64 lookback_words_max(u64 w, u32 B) {
    u64 best = lookback_words(make_shape(w, B), true);
    for (u32 ba : kDigitChoices)
        for (u32 be : kDigitChoices)
            best = std::max(best, lookback_words(make_shape(w, B, ba, be), true));
    return best;
}

// Digit bits of pass p that can be nonzero when the sort's live key bits
// are `total` and digits are `bits` wide.
u32 live_bits(u32 total, u32 bits, int p) {
    const u32 lo = (u32)p * bits;
    return lo >= total ? 0u : std::min(bits, total - lo);
}

size_t prep_smem(const BatchShape &s, bool edges) {
    return (((size_t)s.npa << s.bits_a) + (edges ? ((size_t)s.npe << s.bits_e) : 0)) *
           sizeof(u32);
}

// Per-batch zeroed scratch: BatchAcc, the batch's error word (256 bytes
// reserved), then SortPlan[2], then look-back words.
constexpr u64 kOffErr = sizeof(BatchAcc);
constexpr u64 kOffPlans = kOffErr + 256;
constexpr u64 kOffLookback = kOffPlans + 2 * sizeof(SortPlan);

}  // namespace

struct tc_ctx {
    int device = 0;
    int sm_count = 1;
    u64 r = 0, seed = 0;
    u32 stream_id = 0, vertex_bits = 32;
    u64 cap_w = 0;                           // scratch capacity in edges
    u32 force_bits_a = 0, force_bits_e = 0;  // tc_tune digit widths (0 = automatic)
    int rank_method = kRankBallot;           // tc_tune warp ranking method
    u32 sweep_bps = kSweepBlocksPerSM;       // tc_tune_sweep: sweep blocks per SM
    u64 hash_key = 0;                        // Step-3 edge hash key (random per context)
    cudaStream_t own = nullptr;
    // the edge sort runs on `side`, concurrently with the arc sort
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // pipelined host input: two device staging buffers filled on `copy`
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_copied[2] = {}, ev_used[2] = {};
    u64 *staging2 = nullptr;
    int stage_next = 0;
    // estimator state (structure of arrays)
    u64 *f1 = nullptr, *f2 = nullptr, *chi = nullptr;
    u32 *flags = nullptr;
    Control *ctl = nullptr;
    // per-batch scratch: one set, or two once a batch is pipelined (batch k+1
    // sorts into the set that batch k's sweep is not reading)
    struct Set {
        u64 *arcs[2] = {nullptr, nullptr};
        u64 *ekeys[2] = {nullptr, nullptr};
        unsigned char *zeroed = nullptr;  // BatchAcc, error word, SortPlan[2], look-back
        DirEntry *adir = nullptr;         // tagged arc directory (ids < 2^kDirMaxBits; made
                                          // by the first batch that needs it)
        u32 *aoff = nullptr;              // dense arc offsets, 2^B + 1 (ids < 2^kDirMaxBits)
        uint4 *pdir = nullptr;            // the same packed, packed_groups(2^B)
        uint2 *bdir = nullptr;            // Step-3 buckets {first index, filter mask}, 2^hb + 1
    };
    Set set[2];
    int nsets = 1;
    u32 seq = 0;                      // batches enqueued: directory tag, set parity
    cudaStream_t sa = nullptr;        // a pipelined batch's sort phase (with `side`)
    cudaEvent_t ev_sorted[2] = {}, ev_swept[2] = {};
    u64 *staging = nullptr;
    Control *h_ctl = nullptr;         // pinned host copy of the control block
    // launch accounting and stage timing
    u64 launches = 0;
    bool prof = false;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    struct Stamp {
        cudaEvent_t ev;
        int stage;  // stage that ends here; kStart opens a sequence
    };
    std::vector<Stamp> stamps;
    // per batch: sorts begin (main), arc passes end (main), edge passes end (side)
    struct SortSpan {
        cudaEvent_t begin, arc_end, edge_end;
    };
    std::vector<SortSpan> spans;
    u64 prof_launch0 = 0, prof_batches = 0, prof_sort_launches = 0, prof_sort_bytes = 0;
    u64 prof_skip0 = 0, prof_skipbytes0 = 0;
    bool prof_overflow = false;
};

// A profiling event recorded on `st` (nullptr when not profiling or out of events).
static cudaEvent_t mark(tc_ctx *c, cudaStream_t st) {
    if (!c->prof) return nullptr;
    if (c->pool_used >= c->pool.size()) {
        c->prof_overflow = true;
        return nullptr;
    }
    cudaEvent_t ev = c->pool[c->pool_used++];
    cudaEventRecord(ev, st);
    return ev;
}

static void stamp(tc_ctx *c, cudaStream_t st, int stage) {
    if (!c->prof) return;
    if (c->pool_used >= c->pool.size()) {
        c->prof_overflow = true;
        return;
    }
    cudaEvent_t ev = c->pool[c->pool_used++];
    cudaEventRecord(ev, st);
    c->stamps.push_back({ev, stage});
}

static void free_set(tc_ctx::Set &z, bool with_dir) {
    for (int k = 0; k < 2; ++k) {
        cudaFree(z.arcs[k]);
        cudaFree(z.ekeys[k]);
        z.arcs[k] = z.ekeys[k] = nullptr;
    }
    cudaFree(z.bdir);
    cudaFree(z.zeroed);
    z.bdir = nullptr;
    z.zeroed = nullptr;
    if (with_dir) {
        cudaFree(z.adir);
        cudaFree(z.aoff);
        cudaFree(z.pdir);
        z.adir = nullptr;
        z.aoff = nullptr;
        z.pdir = nullptr;
    }
}

static void free_scratch(tc_ctx *c) {
    for (int k = 0; k < 2; ++k) free_set(c->set[k], false);
    cudaFree(c->staging);
    cudaFree(c->staging2);
    c->staging = nullptr;
    c->staging2 = nullptr;
    c->cap_w = 0;
}

// Batch-size-dependent buffers of one scratch set (and its vertex directory
// the first time), for batches of up to w edges.
static bool alloc_set(tc_ctx *c, tc_ctx::Set &z, u64 w) {
    const u64 zb = kOffLookback + lookback_words_max(w, c->vertex_bits) * sizeof(u32);
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        ok &= cudaMalloc(&z.arcs[k], 2 * w * sizeof(u64)) == cudaSuccess;
        ok &= ok && cudaMalloc(&z.ekeys[k], w * sizeof(u64)) == cudaSuccess;
    }
    const u64 nb = 1ull << hash_bucket_bits(w);
    ok &= ok && cudaMalloc(&z.bdir, (nb + 1) * sizeof(uint2)) == cudaSuccess;
    ok &= ok && cudaMalloc(&z.zeroed, zb) == cudaSuccess;
    if (ok && !z.aoff && c->vertex_bits <= kDirMaxBits) {
        const u64 nverts = 1ull << c->vertex_bits;
        ok &= cudaMalloc(&z.aoff, (nverts + 1) * sizeof(u32)) == cudaSuccess;
        ok &= ok && cudaMalloc(&z.pdir, packed_groups(nverts) * sizeof(uint4)) == cudaSuccess;
    }
    return ok;
}

// How a batch of w edges finds its arc runs: the dense offsets when writing
// all 2^B + 1 of them costs no more than one arc pass moves (2^B <= 8w), the
// tagged directory for smaller batches, binary search beyond 2^kDirMaxBits ids.
static int arc_dir_mode(u32 B, u64 w) {
    if (B > kDirMaxBits) return kArcSearch;
    return ((1ull << B) <= 8 * w) ? kArcDense : kArcTagged;
}

// The tagged directory of a set, made on first need (all tags 0: no entry
// is valid for a batch, whose tags start at 1).
static int ensure_tagged_dir(tc_ctx *c, tc_ctx::Set &z, cudaStream_t st) {
    if (z.adir) return TC_OK;
    const u64 nverts = 1ull << c->vertex_bits;
    if (cudaMalloc(&z.adir, nverts * sizeof(DirEntry)) != cudaSuccess) {
        cudaGetLastError();
        return TC_ERR_NOMEM;
    }
    TC_CUDA(cudaMemsetAsync(z.adir, 0, nverts * sizeof(DirEntry), st));
    return TC_OK;
}

static int ensure_scratch(tc_ctx *c, u64 w) {
    if (w <= c->cap_w) return TC_OK;
    TC_CUDA(cudaDeviceSynchronize());
    free_scratch(c);
    bool ok = cudaMalloc(&c->staging, w * sizeof(u64)) == cudaSuccess;
    for (int k = 0; k < c->nsets && ok; ++k) ok &= alloc_set(c, c->set[k], w);
    if (!ok) {
        cudaGetLastError();
        free_scratch(c);
        return TC_ERR_NOMEM;
    }
    c->cap_w = w;
    return TC_OK;
}

// The second scratch set, for pipelined batches.
static int ensure_two_sets(tc_ctx *c) {
    if (c->nsets == 2) return TC_OK;
    if (!alloc_set(c, c->set[1], c->cap_w)) {
        cudaGetLastError();
        free_set(c->set[1], true);
        return TC_ERR_NOMEM;
    }
    c->nsets = 2;
    return TC_OK;
}

static int map_device_error(u32 e) {
    if (e == kErrInput) return TC_ERR_INPUT;
    if (e == kErrTimeout) return TC_ERR_TIMEOUT;
    return e ? TC_ERR_CUDA : TC_OK;
}

// Enqueue one batch whose update lands on `st`.  W is a device pointer; w in
// [1, cap_w].  Stream-ordered: every step runs behind earlier work on st.
// Pipelined (two scratch sets): the sort phase -- key build, both sorts and
// their directories -- runs on the library's own streams as soon as W is
// ready (at the call, or at w_ready) and the set it sorts into is free, so it
// overlaps the sweep of the previous batch; only the sweep and the
// bookkeeping are ordered on st.
static int enqueue_batch(tc_ctx *c, const u64 *W, u64 w, cudaStream_t st, bool pipelined = false,
                         cudaEvent_t w_ready = nullptr) {
    const NvtxRange range("tc batch");
    const BatchShape s =
        make_shape(w, c->vertex_bits, c->force_bits_a, c->force_bits_e, c->hash_key);
    const int b = c->nsets == 2 ? (int)(c->seq & 1) : 0;
    u32 tag = ++c->seq;
    if (tag == 0) {
        // the directory tags wrapped (after 2^32 batches): clear every tagged
        // entry so that no stale entry can carry a reused tag, and skip tag 0
        TC_CUDA(cudaDeviceSynchronize());
        for (int k = 0; k < c->nsets; ++k)
            if (c->set[k].adir)
                TC_CUDA(cudaMemset(c->set[k].adir, 0,
                                   (sizeof(DirEntry) << c->vertex_bits)));
        tag = ++c->seq;
    }
    tc_ctx::Set &z = c->set[b];
    BatchAcc *acc = reinterpret_cast<BatchAcc *>(z.zeroed);
    u32 *berr = reinterpret_cast<u32 *>(z.zeroed + kOffErr);
    SortPlan *plans = reinterpret_cast<SortPlan *>(z.zeroed + kOffPlans);
    u32 *lb = reinterpret_cast<u32 *>(z.zeroed + kOffLookback);
    const u64 used = kOffLookback + lookback_words(s, true) * sizeof(u32);
    // the sort phase's stream, and whether stage stamps go on one timeline
    cudaStream_t ms = pipelined ? c->sa : st;
    // the set's previous batch may have been swept on another stream
    TC_CUDA(cudaStreamWaitEvent(ms, c->ev_swept[b], 0));
    if (w_ready) TC_CUDA(cudaStreamWaitEvent(ms, w_ready, 0));
    const int dmode = arc_dir_mode(c->vertex_bits, w);
    if (dmode == kArcTagged) {
        const int rc = ensure_tagged_dir(c, z, ms);
        if (rc) return rc;
    }
    const bool stages = !pipelined;
    if (stages) stamp(c, ms, kStart);
    TC_CUDA(cudaMemsetAsync(z.zeroed, 0, used, ms));

    const u64 prep_blocks = std::min<u64>((w + kPrepThreads * 8 - 1) / (kPrepThreads * 8), 1216);
    prep_kernel<<<(unsigned)prep_blocks, kPrepThreads, prep_smem(s, true), ms>>>(
        W, s, z.arcs[0], z.ekeys[0], plans, berr, 1);
    sort_plan_kernel<<<dim3((unsigned)std::max(s.npa, s.npe), 2), 256, 0, ms>>>(
        plans, s.npa, (u32)(2 * w), s.bits_a, s.npe, (u32)w, s.bits_e);
    if (stages) stamp(c, ms, kPrep);
    const u64 ta = tiles_of(2 * w), te = tiles_of(w);
    const u64 la = pass_lookback_words(2 * w, s.bits_a), le = pass_lookback_words(w, s.bits_e);
    const PassKernel ka = select_pass(s.bits_a, false, c->rank_method);
    const PassKernel ke = select_pass(s.bits_e, false, c->rank_method);
    // The two sorts are independent: the edge sort and its index fork onto
    // the side stream and join before the sweep, so the kernels of one fill
    // the SMs the other leaves idle (tails of its waves, look-back waits).
    TC_CUDA(cudaEventRecord(c->ev_fork, ms));
    TC_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    const cudaEvent_t sort_begin = mark(c, ms);
    u32 *lbe = lb + (u64)s.npa * la;
    for (int p = 0; p < s.npe; ++p)
        ke.fn<<<(unsigned)te, ke.threads, ke.smem, c->side>>>(
            z.ekeys[0], z.ekeys[1], nullptr, nullptr, (u32)w, s.she + p * s.bits_e,
            live_bits(s.hs, s.bits_e, p), p, &plans[1], lbe + (u64)p * le, berr, c->ctl);
    const cudaEvent_t edge_end = mark(c, c->side);
    step3_index_kernel<<<index_blocks(w), kIdxThreads, 0, c->side>>>(
        z.ekeys[0], z.ekeys[1], &plans[1], s, z.bdir, W, berr);
    TC_CUDA(cudaEventRecord(c->ev_join, c->side));
    for (int p = 0; p < s.npa; ++p)
        ka.fn<<<(unsigned)ta, ka.threads, ka.smem, ms>>>(
            z.arcs[0], z.arcs[1], nullptr, nullptr, (u32)(2 * w), s.sha + p * s.bits_a,
            live_bits(s.B, s.bits_a, p), p, &plans[0], lb + (u64)p * la, berr, c->ctl);
    const cudaEvent_t arc_end = mark(c, ms);
    if (sort_begin && edge_end && arc_end) c->spans.push_back({sort_begin, arc_end, edge_end});
    if (stages) stamp(c, ms, kArcSort);  // arc passes, with the edge passes beside them
    if (dmode == kArcDense) {
        offsets_kernel<<<index_blocks(2 * w), kIdxThreads, 0, ms>>>(z.arcs[0], z.arcs[1],
                                                                     &plans[0], s, z.aoff);
        pack_offsets_kernel<<<pack_blocks(c->vertex_bits, c->sm_count), kIdxThreads, 0, ms>>>(
            z.aoff, 1u << c->vertex_bits, z.pdir);
    } else if (dmode == kArcTagged)
        index_kernel<<<index_blocks(2 * w), kIdxThreads, 0, ms>>>(z.arcs[0], z.arcs[1],
                                                                   &plans[0], s, z.adir, tag);
    if (stages) stamp(c, ms, kDups);  // the arc index, beside the rest of the edge branch
    TC_CUDA(cudaStreamWaitEvent(ms, c->ev_join, 0));
    if (stages) stamp(c, ms, kEdgeSort);  // what is left of the edge passes and their index
    if (pipelined) {
        TC_CUDA(cudaEventRecord(c->ev_sorted[b], ms));
        TC_CUDA(cudaStreamWaitEvent(st, c->ev_sorted[b], 0));
        stamp(c, st, kStart);  // the sweep's own timeline starts when its sorts are done
    }
    SweepArgs a{};
    a.W = W;
    a.f1 = c->f1;
    a.f2 = c->f2;
    a.chi = c->chi;
    a.flags = c->flags;
    a.r = c->r;
    a.arcs0 = z.arcs[0];
    a.arcs1 = z.arcs[1];
    a.ekeys0 = z.ekeys[0];
    a.ekeys1 = z.ekeys[1];
    a.plans = plans;
    a.adir = z.adir;
    a.aoff = z.aoff;
    a.pdir = z.pdir;
    a.bdir = z.bdir;
    a.ctl = c->ctl;
    a.acc = acc;
    a.berr = berr;
    a.epoch = tag;
    a.s = s;
    a.key = make_uint2((u32)(c->seed & 0xFFFFFFFFu), (u32)(c->seed >> 32));
    a.stream = c->stream_id;
    const unsigned sb = sweep_blocks(c->r, c->sm_count, c->sweep_bps);
    if (dmode == kArcDense)
        sweep_kernel<kArcDense><<<sb, kSweepThreads, 0, st>>>(a);
    else if (dmode == kArcTagged)
        sweep_kernel<kArcTagged><<<sb, kSweepThreads, 0, st>>>(a);
    else
        sweep_kernel<kArcSearch><<<sb, kSweepThreads, 0, st>>>(a);
    stamp(c, st, kSweep);
    finish_kernel<<<1, 1, 0, st>>>(c->ctl, acc, berr, w);
    stamp(c, st, kFinish);
    // this set is free again once the sweep and bookkeeping have read it
    TC_CUDA(cudaEventRecord(c->ev_swept[b], st));
    TC_CUDA(cudaGetLastError());
    c->launches += (dmode == kArcDense ? 7 : dmode == kArcTagged ? 6 : 5) + (u64)s.npa + (u64)s.npe;
    if (c->prof) {
        c->prof_batches += 1;
        c->prof_sort_launches += (u64)s.npa + (u64)s.npe;
        c->prof_sort_bytes +=
            (u64)s.npa * 2 * w * 16 + (u64)s.npe * w * 16;
    }
    return TC_OK;
}

// Wait for the device, copy the control block to the host.
static int read_control(tc_ctx *c) {
    TC_CUDA(cudaDeviceSynchronize());
    TC_CUDA(cudaMemcpy(c->h_ctl, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost));
    return TC_OK;
}

// After read_control: report and clear the first device-side error.
static int collect_error(tc_ctx *c) {
    const u32 e = c->h_ctl->sticky;
    if (e) {
        TC_CUDA(cudaMemsetAsync(&c->ctl->sticky, 0, sizeof(u32), c->own));
        TC_CUDA(cudaStreamSynchronize(c->own));
        c->h_ctl->sticky = 0;
    }
    return map_device_error(e);
}

extern "C" {

const char *tc_strerror(int code) {
    switch (code) {
        case TC_OK: return "ok";
        case TC_ERR_INVAL: return "invalid argument";
        case TC_ERR_NOMEM: return "out of memory";
        case TC_ERR_INPUT:
            return "batch breaks the stream model (self-loop, bad key, id range or repeated edge)";
        case TC_ERR_CUDA: return "CUDA runtime error";
        case TC_ERR_TIMEOUT: return "bounded device wait timed out";
        case TC_ERR_RANGE: return "size exceeds the fixed maximum of this entry point";
        default: return "unknown error";
    }
}

int tc_create_ex(uint64_t r, uint64_t seed, uint32_t stream_id, uint64_t w_max,
                 uint32_t vertex_bits, tc_ctx **out) {
    if (!out || r == 0 || r > 0xFFFFFFFFull || w_max == 0 || w_max > kMaxBatch ||
        vertex_bits < 1 || vertex_bits > 32)
        return TC_ERR_INVAL;
    *out = nullptr;
    int rc = configure_kernels();
    if (rc) return rc;
    tc_ctx *c = new (std::nothrow) tc_ctx();
    if (!c) return TC_ERR_NOMEM;
    c->r = r;
    c->seed = seed;
    c->stream_id = stream_id;
    c->vertex_bits = vertex_bits;
    c->hash_key = random_hash_key();
    bool ok = cudaGetDevice(&c->device) == cudaSuccess;
    ok &= ok && cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) ==
                    cudaSuccess;
    ok &= ok && cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) == cudaSuccess;
    ok &= ok && cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess;
    ok &= ok && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok &= ok && cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
    ok &= ok && cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 2; ++k) {
        ok &= ok && cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming) == cudaSuccess;
        ok &= ok && cudaEventCreateWithFlags(&c->ev_used[k], cudaEventDisableTiming) == cudaSuccess;
    }
    ok &= ok && cudaMalloc(&c->f1, r * sizeof(u64)) == cudaSuccess;
    ok &= ok && cudaMalloc(&c->f2, r * sizeof(u64)) == cudaSuccess;
    ok &= ok && cudaMalloc(&c->chi, r * sizeof(u64)) == cudaSuccess;
    ok &= ok && cudaMalloc(&c->flags, r * sizeof(u32)) == cudaSuccess;
    ok &= ok && cudaMalloc(&c->ctl, sizeof(Control)) == cudaSuccess;
    ok &= ok && cudaHostAlloc(&c->h_ctl, sizeof(Control), cudaHostAllocDefault) == cudaSuccess;
    ok &= ok && cudaStreamCreateWithFlags(&c->sa, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 2; ++k) {
        ok &= ok && cudaEventCreateWithFlags(&c->ev_sorted[k], cudaEventDisableTiming) == cudaSuccess;
        ok &= ok && cudaEventCreateWithFlags(&c->ev_swept[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (ok) {
        std::memset(c->h_ctl, 0, sizeof(Control));
        ok &= cudaMemsetAsync(c->f1, 0xFF, r * sizeof(u64), c->own) == cudaSuccess;
        ok &= cudaMemsetAsync(c->f2, 0xFF, r * sizeof(u64), c->own) == cudaSuccess;
        ok &= cudaMemsetAsync(c->chi, 0, r * sizeof(u64), c->own) == cudaSuccess;
        ok &= cudaMemsetAsync(c->flags, 0, r * sizeof(u32), c->own) == cudaSuccess;
        ok &= cudaMemsetAsync(c->ctl, 0, sizeof(Control), c->own) == cudaSuccess;
    }
    if (ok) {
        int rc2 = ensure_scratch(c, w_max);
        if (rc2) {
            tc_destroy(c);
            return rc2;
        }
        ok &= cudaStreamSynchronize(c->own) == cudaSuccess;
    }
    if (!ok) {
        cudaError_t e = cudaGetLastError();
        tc_destroy(c);
        return e == cudaErrorMemoryAllocation ? TC_ERR_NOMEM : TC_ERR_CUDA;
    }
    *out = c;
    return TC_OK;
}

int tc_create(uint64_t r, uint64_t seed, tc_ctx **out) {
    return tc_create_ex(r, seed, 0, kDefaultWMax, 32, out);
}

void tc_destroy(tc_ctx *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    free_scratch(c);
    cudaFree(c->f1);
    cudaFree(c->f2);
    cudaFree(c->chi);
    cudaFree(c->flags);
    cudaFree(c->ctl);
    for (int k = 0; k < 2; ++k) free_set(c->set[k], true);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    for (cudaEvent_t ev : c->pool) cudaEventDestroy(ev);
    if (c->own) cudaStreamDestroy(c->own);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->copy) cudaStreamDestroy(c->copy);
    if (c->sa) cudaStreamDestroy(c->sa);
    for (int k = 0; k < 2; ++k) {
        if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
        if (c->ev_used[k]) cudaEventDestroy(c->ev_used[k]);
        if (c->ev_sorted[k]) cudaEventDestroy(c->ev_sorted[k]);
        if (c->ev_swept[k]) cudaEventDestroy(c->ev_swept[k]);
    }
    delete c;
}

int tc_process_batch_async(tc_ctx *c, const uint64_t *d_edges, uint64_t w, void *cuda_stream) {
    if (!c || (w && !d_edges) || w > kMaxBatch) return TC_ERR_INVAL;
    if (w == 0) return TC_OK;
    if (w > c->cap_w) return TC_ERR_INVAL;
    return enqueue_batch(c, d_edges, w, (cudaStream_t)cuda_stream);
}

int tc_process_batches_async(tc_ctx *const *ctxs, const uint64_t *const *d_edges,
                             const uint64_t *w, uint32_t n, void *cuda_stream) {
    if (n && (!ctxs || !d_edges || !w)) return TC_ERR_INVAL;
    for (uint32_t k = 0; k < n; ++k) {
        const int rc = tc_process_batch_async(ctxs[k], d_edges[k], w[k], cuda_stream);
        if (rc) return rc;
    }
    return TC_OK;
}

int tc_process_batch(tc_ctx *c, const uint64_t *edges, uint64_t w) {
    if (!c || (w && !edges) || w > kMaxBatch) return TC_ERR_INVAL;
    if (w == 0) return TC_OK;
    int rc = ensure_scratch(c, w);
    if (rc) return rc;
    cudaPointerAttributes attr{};
    TC_CUDA(cudaPointerGetAttributes(&attr, edges));
    const u64 *W = edges;
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) {
        // staging may still feed a pipelined batch (tc_process_batch_host_async)
        TC_CUDA(cudaStreamWaitEvent(c->own, c->ev_used[0], 0));
        TC_CUDA(cudaMemcpyAsync(c->staging, edges, w * sizeof(u64), cudaMemcpyHostToDevice,
                                c->own));
        W = c->staging;
    }
    rc = enqueue_batch(c, W, w, c->own);
    if (rc) return rc;
    TC_CUDA(cudaStreamSynchronize(c->own));
    TC_CUDA(cudaMemcpy(c->h_ctl, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost));
    return collect_error(c);
}

int tc_process_batch_host_async(tc_ctx *c, const uint64_t *h_edges, uint64_t w,
                                void *cuda_stream) {
    if (!c || (w && !h_edges) || w > kMaxBatch) return TC_ERR_INVAL;
    if (w == 0) return TC_OK;
    if (w > c->cap_w) return TC_ERR_INVAL;
    if (!c->staging2 && cudaMalloc(&c->staging2, c->cap_w * sizeof(u64)) != cudaSuccess) {
        cudaGetLastError();
        return TC_ERR_NOMEM;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int b = c->stage_next;
    c->stage_next ^= 1;
    u64 *buf = b ? c->staging2 : c->staging;
    // the copy of this batch overlaps the update of the previous one; it only
    // waits for the batch before that to have finished reading this buffer
    TC_CUDA(cudaStreamWaitEvent(c->copy, c->ev_used[b], 0));
    TC_CUDA(cudaMemcpyAsync(buf, h_edges, w * sizeof(u64), cudaMemcpyHostToDevice, c->copy));
    TC_CUDA(cudaEventRecord(c->ev_copied[b], c->copy));
    int rc = ensure_two_sets(c);
    if (rc) return rc;
    // the batch is sorted as soon as its copy lands, beside the previous sweep
    rc = enqueue_batch(c, buf, w, st, true, c->ev_copied[b]);
    if (rc) return rc;
    TC_CUDA(cudaEventRecord(c->ev_used[b], st));
    return TC_OK;
}

int tc_process_batch_ready_async(tc_ctx *c, const uint64_t *d_edges, uint64_t w,
                                 void *cuda_stream) {
    if (!c || (w && !d_edges) || w > kMaxBatch) return TC_ERR_INVAL;
    if (w == 0) return TC_OK;
    if (w > c->cap_w) return TC_ERR_INVAL;
    const int rc = ensure_two_sets(c);
    if (rc) return rc;
    return enqueue_batch(c, d_edges, w, (cudaStream_t)cuda_stream, true);
}

int tc_sync(tc_ctx *c) {
    if (!c) return TC_ERR_INVAL;
    int rc = read_control(c);
    if (rc) return rc;
    return collect_error(c);
}

int tc_get_counters(tc_ctx *c, uint64_t *r, uint64_t *m, uint64_t *batches) {
    if (!c) return TC_ERR_INVAL;
    int rc = read_control(c);
    if (rc) return rc;
    if (r) *r = c->r;
    if (m) *m = c->h_ctl->m;
    if (batches) *batches = c->h_ctl->batches;
    return TC_OK;
}

int tc_estimate_async(tc_ctx *c, tc_estimate_t *d_out, void *cuda_stream) {
    if (!c || !d_out || (reinterpret_cast<uintptr_t>(d_out) & 7)) return TC_ERR_INVAL;
    // The sweep reduced S and the closed count of the new state, and the
    // batch's finish step committed them with |E|: form the record from them.
    cudaStream_t st = (cudaStream_t)cuda_stream;
    stamp(c, st, kStart);
    estimate_record_kernel<<<1, 1, 0, st>>>(c->ctl, c->r, d_out);
    TC_CUDA(cudaGetLastError());
    c->launches += 1;
    stamp(c, st, kEstimate);
    return TC_OK;
}

int tc_estimate(tc_ctx *c, tc_estimate_t *out) {
    if (!c || !out) return TC_ERR_INVAL;
    int rc = tc_sync(c);
    if (rc) return rc;
    const Control &h = *c->h_ctl;
    finish_estimate(h.est[0], h.est[1], h.est[2], h.est[3], c->r, h.batches, out);
    return TC_OK;
}

int tc_estimate_mom(tc_ctx *c, uint32_t g, uint64_t *num_lo, uint64_t *num_hi, uint64_t *den,
                    double *value) {
    if (!c || g == 0 || g > c->r) return TC_ERR_INVAL;
    int rc = tc_sync(c);
    if (rc) return rc;
    u64 *d_out = nullptr;
    TC_CUDA(cudaMallocAsync(&d_out, 2ull * g * sizeof(u64), c->own));
    group_sum_kernel<<<g, kReduceThreads, 0, c->own>>>(c->chi, c->flags, c->r, g, d_out);
    c->launches += 1;
    std::vector<u64> h(2ull * g);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 =
        cudaMemcpyAsync(h.data(), d_out, 2ull * g * sizeof(u64), cudaMemcpyDeviceToHost, c->own);
    cudaError_t e3 = cudaFreeAsync(d_out, c->own);
    cudaError_t e4 = cudaStreamSynchronize(c->own);
    if (e1 || e2 || e3 || e4) return TC_ERR_CUDA;
    using u128 = unsigned __int128;
    struct G {
        u128 s;
        u64 size;
    };
    std::vector<G> gs(g);
    for (u32 k = 0; k < g; ++k) {
        const u64 lo = (u64)(((u128)k * c->r) / g), hi = (u64)(((u128)(k + 1) * c->r) / g);
        gs[k].s = ((u128)h[2 * k + 1] << 64) | h[2 * k];
        gs[k].size = hi - lo;
    }
    // order the means S_k / size_k exactly (the common factor m drops out)
    std::sort(gs.begin(), gs.end(),
              [](const G &a, const G &b) { return a.s * (u128)b.size < b.s * (u128)a.size; });
    const G &med = gs[(g - 1) / 2];
    const u128 num = med.s * (u128)c->h_ctl->m;
    if (num_lo) *num_lo = (u64)num;
    if (num_hi) *num_hi = (u64)(num >> 64);
    if (den) *den = med.size;
    if (value) *value = (double)(num / med.size) + (double)(num % med.size) / (double)med.size;
    return TC_OK;
}

int tc_get_state(tc_ctx *c, uint64_t *f1, uint64_t *f2, uint64_t *chi, uint32_t *flags) {
    if (!c) return TC_ERR_INVAL;
    TC_CUDA(cudaDeviceSynchronize());
    if (f1) TC_CUDA(cudaMemcpy(f1, c->f1, c->r * sizeof(u64), cudaMemcpyDeviceToHost));
    if (f2) TC_CUDA(cudaMemcpy(f2, c->f2, c->r * sizeof(u64), cudaMemcpyDeviceToHost));
    if (chi) TC_CUDA(cudaMemcpy(chi, c->chi, c->r * sizeof(u64), cudaMemcpyDeviceToHost));
    if (flags) TC_CUDA(cudaMemcpy(flags, c->flags, c->r * sizeof(u32), cudaMemcpyDeviceToHost));
    return TC_OK;
}

int tc_tune_sweep(tc_ctx *c, uint32_t blocks_per_sm) {
    if (!c || blocks_per_sm > kSweepBlocksPerSM) return TC_ERR_INVAL;
    c->sweep_bps = blocks_per_sm ? blocks_per_sm : kSweepBlocksPerSM;
    return TC_OK;
}

int tc_set_hash_key(tc_ctx *c, uint64_t key) {
    if (!c) return TC_ERR_INVAL;
    c->hash_key = key;
    return TC_OK;
}

int tc_tune(tc_ctx *c, uint32_t arc_digit_bits, uint32_t edge_digit_bits, uint32_t ranking) {
    auto ok_bits = [](uint32_t b) { return b == 0 || (b >= 8 && b <= 11); };
    if (!c || !ok_bits(arc_digit_bits) || !ok_bits(edge_digit_bits) || ranking > 3)
        return TC_ERR_INVAL;
    c->force_bits_a = arc_digit_bits;
    c->force_bits_e = edge_digit_bits;
    c->rank_method = ranking == 1 ? kRankMatch : ranking == 3 ? kRankAtomicOr : kRankBallot;
    return TC_OK;
}

int tc_profile_begin(tc_ctx *c) {
    if (!c) return TC_ERR_INVAL;
    while (c->pool.size() < kEventPool) {
        cudaEvent_t ev;
        TC_CUDA(cudaEventCreate(&ev));
        c->pool.push_back(ev);
    }
    int rc = read_control(c);
    if (rc) return rc;
    c->prof_skip0 = c->h_ctl->skipped_passes;
    c->prof_skipbytes0 = c->h_ctl->skipped_bytes;
    c->pool_used = 0;
    c->stamps.clear();
    c->spans.clear();
    c->prof = true;
    c->prof_overflow = false;
    c->prof_launch0 = c->launches;
    c->prof_batches = c->prof_sort_launches = c->prof_sort_bytes = 0;
    return TC_OK;
}

int tc_profile_end(tc_ctx *c, tc_profile_t *out) {
    if (!c || !out) return TC_ERR_INVAL;
    int rc = read_control(c);
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    double ms[kStages] = {0};
    for (size_t k = 1; k < c->stamps.size(); ++k) {
        const int stg = c->stamps[k].stage;
        if (stg < 0) continue;
        float t = 0.f;
        TC_CUDA(cudaEventElapsedTime(&t, c->stamps[k - 1].ev, c->stamps[k].ev));
        ms[stg] += t;
    }
    double wall = 0;
    for (const tc_ctx::SortSpan &sp : c->spans) {
        float ta = 0.f, te = 0.f;
        TC_CUDA(cudaEventElapsedTime(&ta, sp.begin, sp.arc_end));
        TC_CUDA(cudaEventElapsedTime(&te, sp.begin, sp.edge_end));
        wall += ta > te ? ta : te;
    }
    out->ms_sort_wall = wall;
    out->batches = c->prof_batches;
    out->launches = c->launches - c->prof_launch0;
    out->sort_pass_launches = c->prof_sort_launches;
    out->sort_pass_skipped = c->h_ctl->skipped_passes - c->prof_skip0;
    out->sort_pass_bytes =
        c->prof_sort_bytes - (c->h_ctl->skipped_bytes - c->prof_skipbytes0);
    out->overflow = c->prof_overflow ? 1 : 0;
    out->ms_prep = ms[kPrep];
    out->ms_arc_sort = ms[kArcSort];
    out->ms_edge_sort = ms[kEdgeSort];
    out->ms_dups = ms[kDups];
    out->ms_sweep = ms[kSweep];
    out->ms_finish = ms[kFinish];
    out->ms_estimate = ms[kEstimate];
    c->prof = false;
    c->stamps.clear();
    c->spans.clear();
    c->pool_used = 0;
    return TC_OK;
}

int tc_rank_all(const uint64_t *d_edges, uint64_t w, uint32_t vertex_bits, uint32_t *d_src,
                uint32_t *d_dst, uint32_t *d_pos, uint32_t *d_rank, void *cuda_stream) {
    if (w > kMaxBatch || vertex_bits < 1 || vertex_bits > 32) return TC_ERR_INVAL;
    if (w == 0) return TC_OK;
    if (!d_edges || !d_src || !d_dst || !d_pos || !d_rank) return TC_ERR_INVAL;
    int rc = configure_kernels();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const BatchShape s = make_shape(w, vertex_bits);
    const u64 ta = tiles_of(2 * w);
    const u64 la = pass_lookback_words(2 * w, s.bits_a);
    const PassKernel ka = select_pass(s.bits_a, false, kRankBallot);
    const u64 zb = sizeof(SortPlan) * 2 + lookback_words(s, false) * sizeof(u32) + 16;
    unsigned char *z = nullptr;
    u64 *a0 = nullptr, *a1 = nullptr;
    if (cudaMallocAsync(&z, zb, st) != cudaSuccess ||
        cudaMallocAsync(&a0, 2 * w * sizeof(u64), st) != cudaSuccess ||
        cudaMallocAsync(&a1, 2 * w * sizeof(u64), st) != cudaSuccess) {
        cudaGetLastError();
        if (z) cudaFreeAsync(z, st);
        if (a0) cudaFreeAsync(a0, st);
        cudaStreamSynchronize(st);
        return TC_ERR_NOMEM;
    }
    SortPlan *plans = reinterpret_cast<SortPlan *>(z);
    u32 *lb = reinterpret_cast<u32 *>(z + 2 * sizeof(SortPlan));
    u32 *err = reinterpret_cast<u32 *>(z + zb - 16);
    cudaMemsetAsync(z, 0, zb, st);
    const u64 prep_blocks = std::min<u64>((w + kPrepThreads * 8 - 1) / (kPrepThreads * 8), 1216);
    prep_kernel<<<(unsigned)prep_blocks, kPrepThreads, prep_smem(s, false), st>>>(
        d_edges, s, a0, nullptr, plans, err, 0);
    sort_plan_kernel<<<dim3((unsigned)s.npa, 1), 256, 0, st>>>(plans, s.npa, (u32)(2 * w),
                                                               s.bits_a, 0, 0, 8);
    for (int p = 0; p < s.npa; ++p)
        ka.fn<<<(unsigned)ta, ka.threads, ka.smem, st>>>(a0, a1, nullptr, nullptr, (u32)(2 * w),
                                                         s.sha + p * s.bits_a, live_bits(s.B, s.bits_a, p), p, &plans[0],
                                                         lb + (u64)p * la, err, nullptr);
    const u64 rb = (2 * w + kRankTile - 1) / kRankTile;
    rank_out_kernel<<<(unsigned)rb, kRankThreads, 0, st>>>(d_edges, a0, a1, &plans[0], s, d_src,
                                                           d_dst, d_pos, d_rank);
    u32 h_err = 0;
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaMemcpyAsync(&h_err, err, sizeof(u32), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(a1, st);
    cudaFreeAsync(a0, st);
    cudaFreeAsync(z, st);
    cudaError_t e3 = cudaStreamSynchronize(st);
    if (e1 || e2 || e3) {
        last_cuda_error() = e1 ? e1 : (e2 ? e2 : e3);
        return TC_ERR_CUDA;
    }
    return map_device_error(h_err & kErrTimeout);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// rankAll without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// rankAll: a process whose HBM is already handed out to another allocator
// (a framework's caching allocator that reserved nearly all of it), a
// latency-critical loop where cudaMalloc / cudaFree would synchronise the
// device or fail with out-of-memory halfway through, or code that must not
// fail for lack of memory once it has started.  tc_rank_all_noalloc serves
// them with scratch that lives in a fixed array in the library's own device
// image: every GPU that loads libtc.so holds these kNoAllocScratchBytes
// (about 12.3 MB) from module load until the process exits, and batches are
// limited to TC_NOALLOC_MAX_EDGES edges.
// ---------------------------------------------------------------------------
namespace {

constexpr u64 kNoAllocArcs = 2ull * TC_NOALLOC_MAX_EDGES;
constexpr u64 kNoAllocPlanBytes = 2 * sizeof(SortPlan);
// Look-back words for any vertex width: at most 4 passes (8-bit digits over
// 32 vertex bits), each reserved for the widest (11-bit) digits.
constexpr u64 kNoAllocLookbackWords =
    4ull * ((kNoAllocArcs / kSortTile + kLookWin - 1) / kLookWin * kLookWin) * kMaxRadix;
constexpr u64 align256(u64 x) { return (x + 255) / 256 * 256; }
constexpr u64 kNoAllocOffLookback = align256(kNoAllocPlanBytes);
constexpr u64 kNoAllocOffErr = kNoAllocOffLookback + align256(kNoAllocLookbackWords * sizeof(u32));
constexpr u64 kNoAllocOffArcs0 = kNoAllocOffErr + 256;
constexpr u64 kNoAllocOffArcs1 = kNoAllocOffArcs0 + align256(kNoAllocArcs * sizeof(u64));
constexpr u64 kNoAllocScratchBytes = kNoAllocOffArcs1 + align256(kNoAllocArcs * sizeof(u64));

// The scratch itself.  In host code this name is only a stand-in for the
// device array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
// Per-device cache of the scratch's device address.  Host threads may make
// their first calls at the same time: every one of them stores the same
// value, through an atomic so that the race is well defined.
std::atomic<unsigned char *> g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per
// device, on that device's first call, with that device current).
int noalloc_scratch(unsigned char **out) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return TC_ERR_INVAL;
    unsigned char *addr = g_noalloc_addr[dev].load(std::memory_order_relaxed);
    if (!addr) {
        void *p = nullptr;
        TC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        addr = static_cast<unsigned char *>(p);
        g_noalloc_addr[dev].store(addr, std::memory_order_relaxed);
    }
    *out = addr;
    return TC_OK;
}

}  // namespace

extern "C" int tc_rank_all_noalloc(const uint64_t *d_edges, uint64_t w, uint32_t vertex_bits,
                                   uint32_t *d_src, uint32_t *d_dst, uint32_t *d_pos,
                                   uint32_t *d_rank, void *cuda_stream) {
    if (vertex_bits < 1 || vertex_bits > 32) return TC_ERR_INVAL;
    if (w > TC_NOALLOC_MAX_EDGES) return TC_ERR_RANGE;
    if (w == 0) return TC_OK;
    if (!d_edges || !d_src || !d_dst || !d_pos || !d_rank) return TC_ERR_INVAL;
    int rc = configure_kernels();
    if (rc) return rc;
    unsigned char *z = nullptr;
    rc = noalloc_scratch(&z);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const BatchShape s = make_shape(w, vertex_bits);
    const u64 ta = tiles_of(2 * w);
    const u64 la = pass_lookback_words(2 * w, s.bits_a);
    if ((u64)s.npa * la > kNoAllocLookbackWords) return TC_ERR_RANGE;
    const PassKernel ka = select_pass(s.bits_a, false, kRankBallot);
    SortPlan *plans = reinterpret_cast<SortPlan *>(z);
    u32 *lb = reinterpret_cast<u32 *>(z + kNoAllocOffLookback);
    u32 *err = reinterpret_cast<u32 *>(z + kNoAllocOffErr);
    u64 *a0 = reinterpret_cast<u64 *>(z + kNoAllocOffArcs0);
    u64 *a1 = reinterpret_cast<u64 *>(z + kNoAllocOffArcs1);
    // The array keeps the previous call's contents: clear the histograms,
    // tile counters, this call's look-back words and the error word.  On a
    // failure part-way, the stream is still drained before returning, so
    // that no work of this call is left running on the shared array when
    // the caller issues the next one.
    cudaError_t e = cudaMemsetAsync(z, 0, kNoAllocPlanBytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(lb, 0, (u64)s.npa * la * sizeof(u32), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(u32), st);
    u32 h_err = 0;
    if (e == cudaSuccess) {
        const u64 prep_blocks =
            std::min<u64>((w + kPrepThreads * 8 - 1) / (kPrepThreads * 8), 1216);
        prep_kernel<<<(unsigned)prep_blocks, kPrepThreads, prep_smem(s, false), st>>>(
            d_edges, s, a0, nullptr, plans, err, 0);
        sort_plan_kernel<<<dim3((unsigned)s.npa, 1), 256, 0, st>>>(plans, s.npa, (u32)(2 * w),
                                                                   s.bits_a, 0, 0, 8);
        for (int p = 0; p < s.npa; ++p)
            ka.fn<<<(unsigned)ta, ka.threads, ka.smem, st>>>(
                a0, a1, nullptr, nullptr, (u32)(2 * w), s.sha + p * s.bits_a,
                live_bits(s.B, s.bits_a, p), p, &plans[0], lb + (u64)p * la, err, nullptr);
        const u64 rb = (2 * w + kRankTile - 1) / kRankTile;
        rank_out_kernel<<<(unsigned)rb, kRankThreads, 0, st>>>(d_edges, a0, a1, &plans[0], s,
                                                               d_src, d_dst, d_pos, d_rank);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&h_err, err, sizeof(u32), cudaMemcpyDeviceToHost, st);
    }
    const cudaError_t e_sync = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e_sync;
    if (e != cudaSuccess) {
        last_cuda_error() = e;
        return TC_ERR_CUDA;
    }
    return map_device_error(h_err & kErrTimeout);
}

// ---- self-test of the bounded device-side waits -----------------------------
// One keys-only 8-bit digit pass over two tiles with a single CTA whose tile
// counter starts at 1: it takes tile 1, and tile 0 -- the predecessor its
// look-back waits for -- is never processed, so the wait must give up after
// kSpinLimit idle rounds and record kErrTimeout.  Every key has digit 0, so
// the scatter after the timeout stays inside the output buffer.
extern "C" int tc_selftest_wait_timeout(void) {
    int rc = configure_kernels();
    if (rc) return rc;
    constexpr u32 n = 2 * kSortTile;
    const u64 lb_words = (u64)lookback_stride(2) << 8;
    u64 *k0 = nullptr, *k1 = nullptr;
    SortPlan *plan = nullptr;
    u32 *lb = nullptr, *err = nullptr;
    bool ok = cudaMalloc(&k0, n * sizeof(u64)) == cudaSuccess;
    ok &= ok && cudaMalloc(&k1, n * sizeof(u64)) == cudaSuccess;
    ok &= ok && cudaMalloc(&plan, sizeof(SortPlan)) == cudaSuccess;
    ok &= ok && cudaMalloc(&lb, lb_words * sizeof(u32)) == cudaSuccess;
    ok &= ok && cudaMalloc(&err, sizeof(u32)) == cudaSuccess;
    u32 h_err = 0;
    if (ok) {
        const u32 one = 1;
        ok &= cudaMemset(k0, 0, n * sizeof(u64)) == cudaSuccess;
        ok &= cudaMemset(plan, 0, sizeof(SortPlan)) == cudaSuccess;
        ok &= cudaMemcpy(&plan->tile_counter[0], &one, sizeof(u32), cudaMemcpyHostToDevice) ==
              cudaSuccess;
        ok &= cudaMemset(lb, 0, lb_words * sizeof(u32)) == cudaSuccess;
        ok &= cudaMemset(err, 0, sizeof(u32)) == cudaSuccess;
        const PassKernel k = select_pass(8, false, kRankBallot);
        if (ok) {
            k.fn<<<1, k.threads, k.smem>>>(k0, k1, nullptr, nullptr, n, 0, 8, 0, plan, lb, err,
                                           nullptr);
            ok &= cudaGetLastError() == cudaSuccess;
            ok &= cudaDeviceSynchronize() == cudaSuccess;
            ok &= ok && cudaMemcpy(&h_err, err, sizeof(u32), cudaMemcpyDeviceToHost) == cudaSuccess;
        }
    }
    cudaFree(k0);
    cudaFree(k1);
    cudaFree(plan);
    cudaFree(lb);
    cudaFree(err);
    if (!ok) return TC_ERR_CUDA;
    return h_err == kErrTimeout ? TC_ERR_TIMEOUT : h_err ? TC_ERR_CUDA : TC_OK;
}

// ---- checkpoint / resume -------------------------------------------------------
// Blob: a 128-byte header of little-endian uint64 words, then f1[r], f2[r],
// chi[r] (uint64) and flags[r] (uint32).  Restoring the estimator tuples,
// |E| and the batch counter (with seed and stream id, the whole Philox
// counter context) resumes a stream bit for bit.
namespace {

constexpr u64 kSaveMagic = 0x3145544154534354ull;  // "TCSTATE1"
constexpr u64 kSaveVersion = 1;

struct SaveHeader {
    u64 magic, version, r, seed, stream_id, vertex_bits, m, batches;
    u64 s_lo, s_hi, closed;
    u64 pad[5];
};
static_assert(sizeof(SaveHeader) == 128, "header is 16 words");

u64 save_bytes(u64 r) { return sizeof(SaveHeader) + 28 * r; }

}  // namespace

extern "C" uint64_t tc_save_size(tc_ctx *c) { return c ? save_bytes(c->r) : 0; }

extern "C" int tc_save(tc_ctx *c, void *buf, uint64_t size) {
    if (!c || !buf || size < save_bytes(c->r)) return TC_ERR_INVAL;
    int rc = read_control(c);
    if (rc) return rc;
    SaveHeader h{};
    h.magic = kSaveMagic;
    h.version = kSaveVersion;
    h.r = c->r;
    h.seed = c->seed;
    h.stream_id = c->stream_id;
    h.vertex_bits = c->vertex_bits;
    h.m = c->h_ctl->m;
    h.batches = c->h_ctl->batches;
    h.s_lo = c->h_ctl->est[0];
    h.s_hi = c->h_ctl->est[1];
    h.closed = c->h_ctl->est[2];
    unsigned char *p = static_cast<unsigned char *>(buf);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const u64 r = c->r;
    TC_CUDA(cudaMemcpy(p, c->f1, r * 8, cudaMemcpyDeviceToHost));
    TC_CUDA(cudaMemcpy(p + 8 * r, c->f2, r * 8, cudaMemcpyDeviceToHost));
    TC_CUDA(cudaMemcpy(p + 16 * r, c->chi, r * 8, cudaMemcpyDeviceToHost));
    TC_CUDA(cudaMemcpy(p + 24 * r, c->flags, r * 4, cudaMemcpyDeviceToHost));
    return TC_OK;
}

extern "C" int tc_load(const void *buf, uint64_t size, uint64_t w_max, tc_ctx **out) {
    if (!buf || !out || size < sizeof(SaveHeader)) return TC_ERR_INVAL;
    *out = nullptr;
    SaveHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kSaveMagic || h.version != kSaveVersion || h.r == 0 ||
        h.r > 0xFFFFFFFFull || h.vertex_bits < 1 || h.vertex_bits > 32 ||
        h.stream_id > 0xFFFFFFFFull || size < save_bytes(h.r))
        return TC_ERR_INVAL;
    const u64 r = h.r;
    const unsigned char *p = static_cast<const unsigned char *>(buf) + sizeof(h);
    // Every tuple must be one the update can reach (Sec. 3): before the first
    // edge all are empty; after it, f1 is an edge of the stream model (u < v,
    // ids below 2^B), f2 is empty or another such edge sharing an endpoint
    // with f1, with chi >= 1, and only a tuple with f2 can be closed.  The
    // sweep indexes the vertex directories by f1's endpoints, so a blob
    // outside these is refused here rather than read out of bounds there.
    // The committed estimate must also be the one the state gives (Lemma
    // 3.1's S over the closed estimators).
    const u64 id_lim = h.vertex_bits >= 32 ? (1ull << 32) : (1ull << h.vertex_bits);
    auto edge_ok = [id_lim](u64 e) {
        const u64 u = e >> 32, v = e & 0xFFFFFFFFull;
        return u < v && v < id_lim;
    };
    using u128 = unsigned __int128;
    u128 S = 0;
    u64 closed = 0;
    for (u64 i = 0; i < r; ++i) {
        u64 f1, f2, chi;
        u32 fl;
        std::memcpy(&f1, p + 8 * i, 8);
        std::memcpy(&f2, p + 8 * r + 8 * i, 8);
        std::memcpy(&chi, p + 16 * r + 8 * i, 8);
        std::memcpy(&fl, p + 24 * r + 4 * i, 4);
        if (fl & ~TC_FLAG_CLOSED) return TC_ERR_INVAL;
        if (h.m == 0) {
            if (f1 != kEmpty || f2 != kEmpty || chi != 0 || fl != 0) return TC_ERR_INVAL;
            continue;
        }
        if (!edge_ok(f1)) return TC_ERR_INVAL;
        if (f2 == kEmpty) {
            // chi turns positive exactly when the first f2 is drawn
            if ((fl & TC_FLAG_CLOSED) || chi != 0) return TC_ERR_INVAL;
        } else {
            const u64 a1 = f1 >> 32, b1 = f1 & 0xFFFFFFFFull;
            const u64 a2 = f2 >> 32, b2 = f2 & 0xFFFFFFFFull;
            const bool adjacent = a1 == a2 || a1 == b2 || b1 == a2 || b1 == b2;
            if (!edge_ok(f2) || f2 == f1 || !adjacent || chi == 0) return TC_ERR_INVAL;
        }
        if (fl & TC_FLAG_CLOSED) {
            S += chi;
            ++closed;
        }
    }
    if ((u64)S != h.s_lo || (u64)(S >> 64) != h.s_hi || closed != h.closed) return TC_ERR_INVAL;
    tc_ctx *c = nullptr;
    int rc = tc_create_ex(r, h.seed, (u32)h.stream_id, w_max, (u32)h.vertex_bits, &c);
    if (rc) return rc;
    bool ok = cudaMemcpy(c->f1, p, r * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(c->f2, p + 8 * r, r * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(c->chi, p + 16 * r, r * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(c->flags, p + 24 * r, r * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= read_control(c) == TC_OK;
    if (ok) {
        c->h_ctl->m = h.m;
        c->h_ctl->batches = h.batches;
        c->h_ctl->est[0] = h.s_lo;
        c->h_ctl->est[1] = h.s_hi;
        c->h_ctl->est[2] = h.closed;
        c->h_ctl->est[3] = h.m;
        ok &= cudaMemcpy(c->ctl, c->h_ctl, sizeof(Control), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) {
        tc_destroy(c);
        return TC_ERR_CUDA;
    }
    *out = c;
    return TC_OK;
}
