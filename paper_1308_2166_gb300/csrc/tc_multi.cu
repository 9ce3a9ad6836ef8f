// Many independent streams advanced together: one round folds one batch per
// stream (any stream may sit a round out) into every stream's estimators
// with a single segmented launch sequence -- one key build, one pair of
// radix sorts over all streams' keys, one repeat check, one estimator sweep
// and one bookkeeping launch -- instead of a full launch sequence per
// stream.  Each stream is the bulkUpdateAll of Sec. 4 on its own stream of
// edges; results are bit-identical to processing each stream alone with the
// same seed, stream id and batch boundaries.
//
// Layout per round (S streams, round edges D[0..Wt) = the streams' batches
// concatenated in stream order, stream s at [eoff_s, eoff_s + w_s)):
//   arc keys   s << (B+bw+1) | src << (bw+1) | (w_s-1-j) << 1 | side, written
//              stream-major in decreasing local position j and sorted on the
//              (s, src) bits: every stream's arcs end up in its own range
//              [2 eoff_s, 2 eoff_s + 2 w_s), in Lemma 4.3's order;
//   edge keys  s << 2B | u << B | v with value j: stream s's keys end up in
//              [eoff_s, eoff_s + w_s) sorted by (u, v).
//   bw = bits of (max_s w_s) - 1, sb = bits of S-1, B = vertex id bits.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include "tc_kernels.cuh"

using namespace tc;

namespace {

#define TCM_CUDA(call)                        \
    do {                                      \
        if ((call) != cudaSuccess) return TC_ERR_CUDA; \
    } while (0)

// Per-stream device record.
struct MStream {
    u64 est_off;  // first global estimator index
    u64 r;        // estimators
    u64 m;        // |E| of this stream
    u64 batches;
    uint2 key;    // Philox key (seed lo, seed hi)
    u32 stream_id;
    u32 err;      // error of the round in flight
    u32 sticky;   // first error since the host last looked
    u32 pad;
    u64 est[4];   // committed estimate: S lo, S hi, closed, m
    u64 acc[3];   // this round's S lo, S hi, closed
    u64 pad2;
};

struct RoundShape {
    u32 S;      // streams
    u32 sb;     // stream id bits
    u32 B;      // vertex id bits
    u32 bw;     // bits of max w_s - 1
    u32 sha;    // arc key: src shift = bw + 1
    u64 Wt;     // edges this round
    int npa, npe;
    u32 bits_a, bits_e;
};

__device__ __forceinline__ u32 stream_of(const u64 *__restrict__ off, u32 S, u64 x) {
    // last s with off[s] <= x (off has S+1 entries, off[0] = 0)
    u32 lo = 0, hi = S;
    while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

constexpr int kMThreads = 256;

__global__ void __launch_bounds__(kMThreads) mprep_kernel(const u64 *__restrict__ D,
                                                           const u64 *__restrict__ eoff,
                                                           RoundShape rs, MStream *ms,
                                                           u64 *__restrict__ arcs0,
                                                           u64 *__restrict__ ekeys0,
                                                           u32 *__restrict__ evals0,
                                                           SortPlan *plans) {
    extern __shared__ u32 h[];
    const u32 ra = 1u << rs.bits_a, re = 1u << rs.bits_e;
    const u32 na = (u32)rs.npa * ra, nh = na + (u32)rs.npe * re;
    u32 *he = h + na;
    for (u32 k = threadIdx.x; k < nh; k += kMThreads) h[k] = 0;
    __syncthreads();
    const u64 id_lim = (rs.B >= 32) ? (1ull << 32) : (1ull << rs.B);
    for (u64 j = (u64)blockIdx.x * kMThreads + threadIdx.x; j < rs.Wt;
         j += (u64)gridDim.x * kMThreads) {
        const u32 s = stream_of(eoff, rs.S, j);
        const u64 e0 = __ldg(eoff + s), ws = __ldg(eoff + s + 1) - e0;
        const u64 jl = j - e0;
        const u64 e = D[j];
        const u64 u = e >> 32, v = e & kMask32;
        if (!(u < v) || v >= id_lim) atomicOr(&ms[s].err, kErrInput);
        const u64 sp = (u64)s << (rs.B + rs.sha);
        const u64 rpos = (ws - 1 - jl) << 1;
        const u64 au = sp | (u << rs.sha) | rpos;
        const u64 av = sp | (v << rs.sha) | rpos | 1ull;
        reinterpret_cast<ulonglong2 *>(arcs0)[e0 + ws - 1 - jl] = make_ulonglong2(au, av);
        for (int p = 0; p < rs.npa; ++p) {
            atomicAdd(&h[p * ra + digit_bits(au, rs.sha + p * rs.bits_a, ra - 1)], 1u);
            atomicAdd(&h[p * ra + digit_bits(av, rs.sha + p * rs.bits_a, ra - 1)], 1u);
        }
        const u64 ek = ((u64)s << (2 * rs.B)) | (u << rs.B) | v;
        ekeys0[j] = ek;
        evals0[j] = (u32)jl;
        for (int p = 0; p < rs.npe; ++p)
            atomicAdd(&he[p * re + digit_bits(ek, p * rs.bits_e, re - 1)], 1u);
    }
    __syncthreads();
    for (u32 k = threadIdx.x; k < nh; k += kMThreads) {
        const u32 c = h[k];
        if (!c) continue;
        if (k < na) atomicAdd(&plans[0].counts[k / ra][k % ra], c);
        else atomicAdd(&plans[1].counts[(k - na) / re][(k - na) % re], c);
    }
}

// Repeats inside one stream's batch are adjacent after the edge sort.
__global__ void mdups_kernel(const u64 *ekeys0, const u64 *ekeys1, const SortPlan *plans,
                             RoundShape rs, MStream *ms) {
    const u64 *E = plan_final_sel(&plans[1]) ? ekeys1 : ekeys0;
    for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x + 1; k < rs.Wt;
         k += (u64)gridDim.x * blockDim.x) {
        const u64 a = E[k];
        if (a == E[k - 1]) atomicOr(&ms[a >> (2 * rs.B)].err, kErrInput);
    }
}

struct MSweepArgs {
    const u64 *D;
    const u64 *eoff;     // round edge offsets, S+1
    const u64 *est_off;  // estimator offsets, S+1
    u64 *f1, *f2, *chi;
    u32 *flags;
    u64 R;
    const u64 *arcs0, *arcs1, *ekeys0, *ekeys1;
    const u32 *evals0, *evals1;
    const SortPlan *plans;
    MStream *ms;
    const u32 *gerr;     // round-wide error (a timed-out sort)
    RoundShape rs;
};

// Sum of (lo, hi, cnt) over the lanes of this warp whose `key` equals this
// lane's; the lowest such lane gets the sum and returns true.
__device__ __forceinline__ bool warp_segment_sum(u32 key, u64 &lo, u64 &hi, u64 &cnt) {
    const u32 grp = __match_any_sync(0xFFFFFFFFu, key);
    const int lane = threadIdx.x & 31;
    u64 slo = 0, shi = 0, sc = 0;
    for (u32 g = grp; g; g &= g - 1) {
        const int src = __ffs(g) - 1;
        const u64 l = __shfl_sync(grp, lo, src), hh = __shfl_sync(grp, hi, src),
                  cc = __shfl_sync(grp, cnt, src);
        const u64 t = slo + l;
        shi += hh + (t < slo ? 1 : 0);
        slo = t;
        sc += cc;
    }
    lo = slo;
    hi = shi;
    cnt = sc;
    return lane == __ffs(grp) - 1;
}

__global__ void __launch_bounds__(kMThreads) msweep_kernel(MSweepArgs a) {
    if (ld_relaxed(a.gerr)) return;
    const u64 g = (u64)blockIdx.x * kMThreads + threadIdx.x;
    const RoundShape &rs = a.rs;
    u32 s = 0xFFFFFFFFu;
    u64 add = 0, closed = 0;
    if (g < a.R) {
        s = stream_of(a.est_off, rs.S, g);
        const u64 e0 = __ldg(a.eoff + s), ws = __ldg(a.eoff + s + 1) - e0;
        MStream &st = a.ms[s];
        if (ws > 0 && !ld_relaxed(&st.err)) {
            const u64 i = g - __ldg(a.est_off + s);
            const u64 m = st.m;
            const DrawKey dk{st.key, (u32)st.batches, st.stream_id};
            const u64 *arcs = plan_final_sel(&a.plans[0]) ? a.arcs1 : a.arcs0;
            const bool es = plan_final_sel(&a.plans[1]) != 0;
            const u64 *E = es ? a.ekeys1 : a.ekeys0;
            const u32 *EV = es ? a.evals1 : a.evals0;
            const u64 a_lo = 2 * e0, a_hi = 2 * (e0 + ws);
            const u64 sp = (u64)s << (rs.B + rs.sha);
            const u64 wmask = (1ull << rs.bw) - 1;
            u64 f1 = a.f1[g], f2 = a.f2[g], chi = a.chi[g];
            u32 fl = a.flags[g];
            // ---- Step 1 (Sec. 4.2)
            const u64 x = draw_bounded(dk, (u32)i, kStep1, m + ws);
            const bool new1 = x >= m;
            u64 p1 = 0;
            if (new1) {
                p1 = x - m;
                f1 = __ldg(a.D + e0 + p1);
                chi = 0;
                f2 = kEmpty;
                fl = 0;
            }
            // ---- Step 2 (Sec. 4.3)
            const u64 u = f1 >> 32, v = f1 & kMask32;
            // (x + 1) << sha may carry into the stream bits: add, do not OR
            const u64 su = lower_bound_range(arcs, a_lo, a_hi, sp + (u << rs.sha));
            const u64 eu = lower_bound_range(arcs, su, a_hi, sp + ((u + 1) << rs.sha));
            const u64 sv = lower_bound_range(arcs, a_lo, a_hi, sp + (v << rs.sha));
            const u64 ev = lower_bound_range(arcs, sv, a_hi, sp + ((v + 1) << rs.sha));
            u64 ld, rd;
            if (new1) {
                const u64 rp = (ws - 1 - p1) << 1;
                ld = lower_bound_range(arcs, su, eu, sp | (u << rs.sha) | rp) - su;
                rd = lower_bound_range(arcs, sv, ev, sp | (v << rs.sha) | rp) - sv;
            } else {
                ld = eu - su;
                rd = ev - sv;
            }
            const u64 chi_plus = ld + rd;
            bool new2 = false;
            u64 p2 = 0;
            if (chi_plus > 0) {
                const u64 y = draw_bounded(dk, (u32)i, kStep2, chi + chi_plus);
                if (y >= chi) {
                    const u64 phi = y - chi;
                    const u64 k = (phi < ld) ? su + phi : sv + (phi - ld);
                    p2 = ws - 1 - ((__ldg(arcs + k) >> 1) & wmask);
                    f2 = __ldg(a.D + e0 + p2);
                    fl &= ~TC_FLAG_CLOSED;
                    new2 = true;
                }
            }
            chi += chi_plus;
            // ---- Step 3 (Sec. 4.4)
            if (f2 != kEmpty && !(fl & TC_FLAG_CLOSED)) {
                const u64 a1 = f1 >> 32, b1 = f1 & kMask32, a2 = f2 >> 32, b2 = f2 & kMask32;
                const u64 x1 = (a1 == a2 || a1 == b2) ? b1 : a1;
                const u64 x2 = (a2 == a1 || a2 == b1) ? b2 : a2;
                const u64 gu = x1 < x2 ? x1 : x2, gv = x1 < x2 ? x2 : x1;
                const u64 probe = ((u64)s << (2 * rs.B)) | (gu << rs.B) | gv;
                const u64 k = lower_bound_range(E, e0, e0 + ws, probe);
                if (k < e0 + ws && __ldg(E + k) == probe) {
                    const u64 q = __ldg(EV + k);
                    if (!new2 || q > p2) fl |= TC_FLAG_CLOSED;
                }
            }
            a.f1[g] = f1;
            a.f2[g] = f2;
            a.chi[g] = chi;
            a.flags[g] = fl;
            if (fl & TC_FLAG_CLOSED) {
                add = chi;
                closed = 1;
            }
        } else {
            s = 0xFFFFFFFFu;  // untouched stream: contributes nothing
        }
    }
    u64 hi = 0;
    if (warp_segment_sum(s, add, hi, closed) && s != 0xFFFFFFFFu) {
        MStream &st = a.ms[s];
        if (add | hi) add_u128(st.acc, add, hi);
        if (closed) atomicAdd((unsigned long long *)&st.acc[2], (unsigned long long)closed);
    }
}

// Close the round for every stream that had a batch.
__global__ void mfinish_kernel(MStream *ms, const u64 *eoff, u32 S, u32 *gerr) {
    const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    MStream &st = ms[s];
    const u64 ws = eoff[s + 1] - eoff[s];
    if (ws > 0) {
        const u32 e = st.err ? st.err : *gerr;
        if (e) {
            if (!st.sticky) st.sticky = e;
        } else {
            st.m += ws;
            st.batches += 1;
            st.est[0] = st.acc[0];
            st.est[1] = st.acc[1];
            st.est[2] = st.acc[2];
            st.est[3] = st.m;
        }
    }
    st.err = 0;
    st.acc[0] = st.acc[1] = st.acc[2] = 0;
}

using PassFn = void (*)(u64 *, u64 *, u32 *, u32 *, u32, u32, u32, int, SortPlan *, u32 *, u32 *,
                        Control *);

struct PassK {
    PassFn fn;
    size_t smem;
    int threads;
};

template <int kBits>
PassK pass_kv(int rank) {
    PassK k{};
    if (rank == kRankMatch)
        k.fn = onesweep_pass_kernel<kBits, true, kRankMatch>,
        k.smem = sizeof(OnesweepSmem<kBits, true, kRankMatch>);
    else
        k.fn = onesweep_pass_kernel<kBits, true, kRankBallot>,
        k.smem = sizeof(OnesweepSmem<kBits, true, kRankBallot>);
    k.threads = OnesweepShape<kBits>::kThreads;
    return k;
}

template <int kBits>
PassK pass_keys(int rank) {
    PassK k{};
    if (rank == kRankMatch)
        k.fn = onesweep_pass_kernel<kBits, false, kRankMatch>,
        k.smem = sizeof(OnesweepSmem<kBits, false, kRankMatch>);
    else
        k.fn = onesweep_pass_kernel<kBits, false, kRankBallot>,
        k.smem = sizeof(OnesweepSmem<kBits, false, kRankBallot>);
    k.threads = OnesweepShape<kBits>::kThreads;
    return k;
}

PassK mselect(u32 bits, bool values, int rank) {
    if (bits == 8) return values ? pass_kv<8>(rank) : pass_keys<8>(rank);
    if (bits == 10) return values ? pass_kv<10>(rank) : pass_keys<10>(rank);
    return values ? pass_kv<11>(rank) : pass_keys<11>(rank);
}

int mconfigure() {
    static bool done[64] = {false};
    int dev = 0;
    TCM_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && done[dev]) return TC_OK;
    for (u32 bits : {8u, 10u, 11u})
        for (int v = 0; v < 2; ++v)
            for (int rk : {kRankBallot, kRankMatch}) {
                const PassK k = mselect(bits, v, rk);
                TCM_CUDA(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)k.smem));
            }
    TCM_CUDA(cudaFuncSetAttribute(mprep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024));
    if (dev < 64) done[dev] = true;
    return TC_OK;
}

u32 mbits_for(u64 x) {
    u32 b = 1;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

u32 mpick(u32 live, u32 forced, int &passes) {
    const u32 bits = forced ? forced : 8;
    passes = (int)((live + bits - 1) / bits);
    if (passes < 1) passes = 1;
    return bits;
}

u64 mtiles(u64 n) { return (n + kSortTile - 1) / kSortTile; }
u64 mlookback(u64 n, u32 bits) { return (u64)lookback_stride((u32)mtiles(n)) << bits; }

u32 mlive(u32 total, u32 bits, int p) {
    const u32 lo = (u32)p * bits;
    return lo >= total ? 0u : std::min(bits, total - lo);
}

constexpr int kRing = 8;

}  // namespace

struct tc_multi {
    u32 S = 0, B = 32, sb = 1;
    u64 R = 0, w_max = 0;
    u32 force_a = 0, force_e = 0;
    int rank = kRankBallot;
    u64 *f1 = nullptr, *f2 = nullptr, *chi = nullptr;
    u32 *flags = nullptr;
    MStream *ms = nullptr;
    u64 *est_off = nullptr;
    std::vector<u64> h_est_off;
    // round scratch
    u64 *arcs[2] = {nullptr, nullptr};
    u64 *ekeys[2] = {nullptr, nullptr};
    u32 *evals[2] = {nullptr, nullptr};
    unsigned char *zeroed = nullptr;  // SortPlan[2], look-back, global error
    u64 zeroed_bytes = 0;
    u64 *eoff[kRing] = {};            // device copies of round offsets
    u64 *h_eoff[kRing] = {};          // pinned staging
    cudaEvent_t ring_ev[kRing] = {};
    int ring = 0;
    u64 launches = 0;
    MStream *h_ms = nullptr;          // pinned host copy for reads
    cudaGraphExec_t gexec = nullptr;  // captured round (tc_multi_capture)
    u64 *g_eoff = nullptr;            // its fixed device offsets
    u64 graph_launches = 0;           // kernels in the captured round
};

static void multi_free(tc_multi *M) {
    cudaDeviceSynchronize();
    cudaFree(M->f1);
    cudaFree(M->f2);
    cudaFree(M->chi);
    cudaFree(M->flags);
    cudaFree(M->ms);
    cudaFree(M->est_off);
    for (int k = 0; k < 2; ++k) {
        cudaFree(M->arcs[k]);
        cudaFree(M->ekeys[k]);
        cudaFree(M->evals[k]);
    }
    cudaFree(M->zeroed);
    for (int k = 0; k < kRing; ++k) {
        cudaFree(M->eoff[k]);
        if (M->h_eoff[k]) cudaFreeHost(M->h_eoff[k]);
        if (M->ring_ev[k]) cudaEventDestroy(M->ring_ev[k]);
    }
    if (M->h_ms) cudaFreeHost(M->h_ms);
    if (M->gexec) cudaGraphExecDestroy(M->gexec);
    cudaFree(M->g_eoff);
    delete M;
}

extern "C" {

int tc_multi_create(uint32_t n_streams, const uint64_t *r, const uint64_t *seeds,
                    const uint32_t *stream_ids, uint64_t w_max_round, uint32_t vertex_bits,
                    tc_multi **out) {
    if (!out || n_streams == 0 || !r || !seeds || !stream_ids || w_max_round == 0 ||
        w_max_round > (1ull << 28) || vertex_bits < 1 || vertex_bits > 32)
        return TC_ERR_INVAL;
    *out = nullptr;
    const u32 sb = mbits_for(n_streams - 1);
    const u32 bwmax = mbits_for(w_max_round - 1);
    if (sb + vertex_bits + bwmax + 1 > 64 || sb + 2 * vertex_bits > 64) return TC_ERR_INVAL;
    u64 R = 0;
    for (u32 s = 0; s < n_streams; ++s) {
        if (r[s] == 0 || r[s] > 0xFFFFFFFFull) return TC_ERR_INVAL;
        R += r[s];
    }
    int rc = mconfigure();
    if (rc) return rc;
    tc_multi *M = new (std::nothrow) tc_multi();
    if (!M) return TC_ERR_NOMEM;
    M->S = n_streams;
    M->B = vertex_bits;
    M->sb = sb;
    M->R = R;
    M->w_max = w_max_round;
    std::vector<MStream> h(n_streams);
    M->h_est_off.assign(n_streams + 1, 0);
    for (u32 s = 0; s < n_streams; ++s) {
        std::memset(&h[s], 0, sizeof(MStream));
        h[s].est_off = M->h_est_off[s];
        h[s].r = r[s];
        h[s].key = make_uint2((u32)(seeds[s] & 0xFFFFFFFFu), (u32)(seeds[s] >> 32));
        h[s].stream_id = stream_ids[s];
        M->h_est_off[s + 1] = M->h_est_off[s] + r[s];
    }
    // worst-case look-back: any digit width for both sorts
    u64 lb = 0;
    for (u32 ba : {8u, 10u, 11u})
        for (u32 be : {8u, 10u, 11u}) {
            int pa, pe;
            mpick(vertex_bits + sb, ba, pa);
            mpick(2 * vertex_bits + sb, be, pe);
            lb = std::max(lb, (u64)pa * mlookback(2 * w_max_round, ba) +
                                  (u64)pe * mlookback(w_max_round, be));
        }
    M->zeroed_bytes = 2 * sizeof(SortPlan) + lb * sizeof(u32) + 256;
    bool ok = cudaMalloc(&M->f1, R * sizeof(u64)) == cudaSuccess;
    ok &= ok && cudaMalloc(&M->f2, R * sizeof(u64)) == cudaSuccess;
    ok &= ok && cudaMalloc(&M->chi, R * sizeof(u64)) == cudaSuccess;
    ok &= ok && cudaMalloc(&M->flags, R * sizeof(u32)) == cudaSuccess;
    ok &= ok && cudaMalloc(&M->ms, n_streams * sizeof(MStream)) == cudaSuccess;
    ok &= ok && cudaMalloc(&M->est_off, (n_streams + 1) * sizeof(u64)) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k) {
        ok &= cudaMalloc(&M->arcs[k], 2 * w_max_round * sizeof(u64)) == cudaSuccess;
        ok &= ok && cudaMalloc(&M->ekeys[k], w_max_round * sizeof(u64)) == cudaSuccess;
        ok &= ok && cudaMalloc(&M->evals[k], w_max_round * sizeof(u32)) == cudaSuccess;
    }
    ok &= ok && cudaMalloc(&M->zeroed, M->zeroed_bytes) == cudaSuccess;
    for (int k = 0; k < kRing && ok; ++k) {
        ok &= cudaMalloc(&M->eoff[k], (n_streams + 1) * sizeof(u64)) == cudaSuccess;
        ok &= ok && cudaHostAlloc(&M->h_eoff[k], (n_streams + 1) * sizeof(u64),
                                  cudaHostAllocDefault) == cudaSuccess;
        ok &= ok && cudaEventCreateWithFlags(&M->ring_ev[k], cudaEventDisableTiming) == cudaSuccess;
    }
    ok &= ok && cudaHostAlloc(&M->h_ms, n_streams * sizeof(MStream), cudaHostAllocDefault) ==
                    cudaSuccess;
    if (ok) {
        ok &= cudaMemset(M->f1, 0xFF, R * sizeof(u64)) == cudaSuccess;
        ok &= cudaMemset(M->f2, 0xFF, R * sizeof(u64)) == cudaSuccess;
        ok &= cudaMemset(M->chi, 0, R * sizeof(u64)) == cudaSuccess;
        ok &= cudaMemset(M->flags, 0, R * sizeof(u32)) == cudaSuccess;
        ok &= cudaMemset(M->zeroed, 0, M->zeroed_bytes) == cudaSuccess;
        ok &= cudaMemcpy(M->ms, h.data(), n_streams * sizeof(MStream), cudaMemcpyHostToDevice) ==
              cudaSuccess;
        ok &= cudaMemcpy(M->est_off, M->h_est_off.data(), (n_streams + 1) * sizeof(u64),
                         cudaMemcpyHostToDevice) == cudaSuccess;
        ok &= cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        const cudaError_t e = cudaGetLastError();
        multi_free(M);
        return e == cudaErrorMemoryAllocation ? TC_ERR_NOMEM : TC_ERR_CUDA;
    }
    *out = M;
    return TC_OK;
}

void tc_multi_destroy(tc_multi *M) {
    if (M) multi_free(M);
}

int tc_multi_tune(tc_multi *M, uint32_t arc_digit_bits, uint32_t edge_digit_bits,
                  uint32_t ranking) {
    auto ok_bits = [](uint32_t b) { return b == 0 || b == 8 || b == 10 || b == 11; };
    if (!M || !ok_bits(arc_digit_bits) || !ok_bits(edge_digit_bits) || ranking > 3)
        return TC_ERR_INVAL;
    M->force_a = arc_digit_bits;
    M->force_e = edge_digit_bits;
    M->rank = ranking == 1 ? kRankMatch : kRankBallot;
    return TC_OK;
}

// Check a round's offsets; returns the largest batch through *wmax.
static int check_round(const tc_multi *M, const uint64_t *offsets, u64 *wmax) {
    if (!offsets || offsets[0] != 0) return TC_ERR_INVAL;
    u64 w = 0;
    for (u32 s = 0; s < M->S; ++s) {
        if (offsets[s + 1] < offsets[s]) return TC_ERR_INVAL;
        w = std::max<u64>(w, offsets[s + 1] - offsets[s]);
    }
    if (offsets[M->S] > M->w_max) return TC_ERR_INVAL;
    *wmax = w;
    return TC_OK;
}

static int enqueue_round(tc_multi *M, const u64 *d_edges, const u64 *offsets, u64 wmax,
                         const u64 *eoff, cudaStream_t st);

int tc_multi_process_async(tc_multi *M, const uint64_t *d_edges, const uint64_t *offsets,
                           void *cuda_stream) {
    if (!M) return TC_ERR_INVAL;
    u64 wmax = 0;
    int rc = check_round(M, offsets, &wmax);
    if (rc) return rc;
    if (offsets[M->S] == 0) return TC_OK;
    if (!d_edges) return TC_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // round offsets through a ring of pinned buffers
    const int slot = M->ring;
    M->ring = (M->ring + 1) % kRing;
    TCM_CUDA(cudaEventSynchronize(M->ring_ev[slot]));
    std::memcpy(M->h_eoff[slot], offsets, (M->S + 1) * sizeof(u64));
    TCM_CUDA(cudaMemcpyAsync(M->eoff[slot], M->h_eoff[slot], (M->S + 1) * sizeof(u64),
                             cudaMemcpyHostToDevice, st));
    TCM_CUDA(cudaEventRecord(M->ring_ev[slot], st));
    return enqueue_round(M, d_edges, offsets, wmax, M->eoff[slot], st);
}

int tc_multi_capture(tc_multi *M, const uint64_t *d_edges, const uint64_t *offsets,
                     void *cuda_stream) {
    if (!M || !d_edges) return TC_ERR_INVAL;
    u64 wmax = 0;
    int rc = check_round(M, offsets, &wmax);
    if (rc) return rc;
    if (offsets[M->S] == 0) return TC_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (M->gexec) {
        cudaGraphExecDestroy(M->gexec);
        M->gexec = nullptr;
    }
    if (!M->g_eoff) TCM_CUDA(cudaMalloc(&M->g_eoff, (M->S + 1) * sizeof(u64)));
    TCM_CUDA(cudaMemcpy(M->g_eoff, offsets, (M->S + 1) * sizeof(u64), cudaMemcpyHostToDevice));
    TCM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const u64 before = M->launches;
    rc = enqueue_round(M, d_edges, offsets, wmax, M->g_eoff, st);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &graph);
    if (rc || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return rc ? rc : TC_ERR_CUDA;
    }
    M->graph_launches = M->launches - before;
    M->launches = before;
    const cudaError_t ei = cudaGraphInstantiate(&M->gexec, graph, 0);
    cudaGraphDestroy(graph);
    return ei == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

int tc_multi_replay(tc_multi *M, void *cuda_stream) {
    if (!M || !M->gexec) return TC_ERR_INVAL;
    TCM_CUDA(cudaGraphLaunch(M->gexec, (cudaStream_t)cuda_stream));
    M->launches += M->graph_launches;
    return TC_OK;
}

}  // extern "C"

static int enqueue_round(tc_multi *M, const u64 *d_edges, const u64 *offsets, u64 wmax,
                         const u64 *eoff, cudaStream_t st) {
    const u64 Wt = offsets[M->S];

    RoundShape rs{};
    rs.S = M->S;
    rs.sb = M->sb;
    rs.B = M->B;
    rs.bw = mbits_for(wmax - 1);
    rs.sha = rs.bw + 1;
    rs.Wt = Wt;
    rs.bits_a = mpick(M->B + M->sb, M->force_a, rs.npa);
    rs.bits_e = mpick(2 * M->B + M->sb, M->force_e, rs.npe);
    SortPlan *plans = reinterpret_cast<SortPlan *>(M->zeroed);
    u32 *lb = reinterpret_cast<u32 *>(M->zeroed + 2 * sizeof(SortPlan));
    const u64 la = mlookback(2 * Wt, rs.bits_a), le = mlookback(Wt, rs.bits_e);
    const u64 lwords = (u64)rs.npa * la + (u64)rs.npe * le;
    u32 *gerr = reinterpret_cast<u32 *>(M->zeroed + M->zeroed_bytes - 256);
    TCM_CUDA(cudaMemsetAsync(M->zeroed, 0, 2 * sizeof(SortPlan) + lwords * sizeof(u32), st));
    TCM_CUDA(cudaMemsetAsync(gerr, 0, sizeof(u32), st));

    const size_t hsm = (((size_t)rs.npa << rs.bits_a) + ((size_t)rs.npe << rs.bits_e)) * 4;
    const u64 pb = std::min<u64>((Wt + kMThreads * 8 - 1) / (kMThreads * 8), 1216);
    mprep_kernel<<<(unsigned)pb, kMThreads, hsm, st>>>(d_edges, eoff, rs, M->ms, M->arcs[0],
                                                       M->ekeys[0], M->evals[0], plans);
    sort_plan_kernel<<<dim3((unsigned)std::max(rs.npa, rs.npe), 2), 256, 0, st>>>(
        plans, rs.npa, (u32)(2 * Wt), rs.bits_a, rs.npe, (u32)Wt, rs.bits_e);
    const PassK ka = mselect(rs.bits_a, false, M->rank);
    const PassK ke = mselect(rs.bits_e, true, M->rank);
    const u64 ta = mtiles(2 * Wt), te = mtiles(Wt);
    for (int p = 0; p < rs.npa; ++p)
        ka.fn<<<(unsigned)ta, ka.threads, ka.smem, st>>>(
            M->arcs[0], M->arcs[1], nullptr, nullptr, (u32)(2 * Wt), rs.sha + p * rs.bits_a,
            mlive(M->B + M->sb, rs.bits_a, p), p, &plans[0], lb + (u64)p * la, gerr, nullptr);
    u32 *lbe = lb + (u64)rs.npa * la;
    for (int p = 0; p < rs.npe; ++p)
        ke.fn<<<(unsigned)te, ke.threads, ke.smem, st>>>(
            M->ekeys[0], M->ekeys[1], M->evals[0], M->evals[1], (u32)Wt, p * rs.bits_e,
            mlive(2 * M->B + M->sb, rs.bits_e, p), p, &plans[1], lbe + (u64)p * le, gerr,
            nullptr);
    const u64 db = std::min<u64>((Wt + 255) / 256, 1216);
    mdups_kernel<<<(unsigned)db, 256, 0, st>>>(M->ekeys[0], M->ekeys[1], plans, rs, M->ms);
    MSweepArgs a{};
    a.D = d_edges;
    a.eoff = eoff;
    a.est_off = M->est_off;
    a.f1 = M->f1;
    a.f2 = M->f2;
    a.chi = M->chi;
    a.flags = M->flags;
    a.R = M->R;
    a.arcs0 = M->arcs[0];
    a.arcs1 = M->arcs[1];
    a.ekeys0 = M->ekeys[0];
    a.ekeys1 = M->ekeys[1];
    a.evals0 = M->evals[0];
    a.evals1 = M->evals[1];
    a.plans = plans;
    a.ms = M->ms;
    a.gerr = gerr;
    a.rs = rs;
    msweep_kernel<<<(unsigned)((M->R + kMThreads - 1) / kMThreads), kMThreads, 0, st>>>(a);
    mfinish_kernel<<<(M->S + 255) / 256, 256, 0, st>>>(M->ms, eoff, M->S, gerr);
    TCM_CUDA(cudaGetLastError());
    M->launches += 5 + (u64)rs.npa + (u64)rs.npe;
    return TC_OK;
}

extern "C" {

int tc_multi_sync(tc_multi *M, int32_t *stream_errors) {
    if (!M) return TC_ERR_INVAL;
    TCM_CUDA(cudaDeviceSynchronize());
    TCM_CUDA(cudaMemcpy(M->h_ms, M->ms, M->S * sizeof(MStream), cudaMemcpyDeviceToHost));
    int first = TC_OK;
    bool any = false;
    for (u32 s = 0; s < M->S; ++s) {
        const u32 e = M->h_ms[s].sticky;
        const int code = e == kErrInput ? TC_ERR_INPUT : e == kErrTimeout ? TC_ERR_TIMEOUT
                                                                           : e ? TC_ERR_CUDA : TC_OK;
        if (stream_errors) stream_errors[s] = code;
        if (code && first == TC_OK) first = code;
        if (e) {
            any = true;
            M->h_ms[s].sticky = 0;
        }
    }
    if (any) {
        TCM_CUDA(cudaMemcpy(M->ms, M->h_ms, M->S * sizeof(MStream), cudaMemcpyHostToDevice));
    }
    return first;
}

int tc_multi_estimate(tc_multi *M, uint32_t s, tc_estimate_t *out) {
    if (!M || !out || s >= M->S) return TC_ERR_INVAL;
    TCM_CUDA(cudaDeviceSynchronize());
    MStream h{};
    TCM_CUDA(cudaMemcpy(&h, M->ms + s, sizeof(MStream), cudaMemcpyDeviceToHost));
    using u128 = unsigned __int128;
    const u128 S = ((u128)h.est[1] << 64) | h.est[0];
    const u128 N = S * (u128)h.m;
    out->sum_lo = (u64)S;
    out->sum_hi = (u64)(S >> 64);
    out->num_lo = (u64)N;
    out->num_hi = (u64)(N >> 64);
    out->r = h.r;
    out->m = h.m;
    out->n_closed = h.est[2];
    out->batches = h.batches;
    const u128 q = N / h.r, rem = N % h.r;
    out->tau_hat = (double)q + (double)rem / (double)h.r;
    return TC_OK;
}

int tc_multi_estimates_async(tc_multi *M, uint64_t *d_out, void *cuda_stream) {
    if (!M || !d_out) return TC_ERR_INVAL;
    const unsigned char *est0 =
        reinterpret_cast<const unsigned char *>(M->ms) + offsetof(MStream, est);
    TCM_CUDA(cudaMemcpy2DAsync(d_out, 4 * sizeof(u64), est0, sizeof(MStream),
                               4 * sizeof(u64), M->S, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)cuda_stream));
    return TC_OK;
}

int tc_multi_get_state(tc_multi *M, uint32_t s, uint64_t *f1, uint64_t *f2, uint64_t *chi,
                       uint32_t *flags) {
    if (!M || s >= M->S) return TC_ERR_INVAL;
    TCM_CUDA(cudaDeviceSynchronize());
    const u64 o = M->h_est_off[s], n = M->h_est_off[s + 1] - o;
    if (f1) TCM_CUDA(cudaMemcpy(f1, M->f1 + o, n * sizeof(u64), cudaMemcpyDeviceToHost));
    if (f2) TCM_CUDA(cudaMemcpy(f2, M->f2 + o, n * sizeof(u64), cudaMemcpyDeviceToHost));
    if (chi) TCM_CUDA(cudaMemcpy(chi, M->chi + o, n * sizeof(u64), cudaMemcpyDeviceToHost));
    if (flags) TCM_CUDA(cudaMemcpy(flags, M->flags + o, n * sizeof(u32), cudaMemcpyDeviceToHost));
    return TC_OK;
}

int tc_multi_get_counters(tc_multi *M, uint32_t s, uint64_t *r, uint64_t *m,
                          uint64_t *batches) {
    if (!M || s >= M->S) return TC_ERR_INVAL;
    TCM_CUDA(cudaDeviceSynchronize());
    MStream h{};
    TCM_CUDA(cudaMemcpy(&h, M->ms + s, sizeof(MStream), cudaMemcpyDeviceToHost));
    if (r) *r = h.r;
    if (m) *m = h.m;
    if (batches) *batches = h.batches;
    return TC_OK;
}

int tc_multi_launches(tc_multi *M, uint64_t *launches) {
    if (!M || !launches) return TC_ERR_INVAL;
    *launches = M->launches;
    return TC_OK;
}

}  // extern "C"
