// Many independent streams advanced together: one round folds one batch into
// each of K participating streams with a single segmented launch sequence --
// one key build, one pair of radix sorts over all participants' keys, one
// repeat check, one estimator sweep and one bookkeeping launch -- instead of
// a full launch sequence per stream.  Each stream is the bulkUpdateAll of
// Sec. 4 on its own stream of edges; results are bit-identical to processing
// each stream alone with the same seed, stream id and batch boundaries.
//
// Layout per round (K participants k = 0..K-1, participant k folds batch
// D_k[0..w_k) into slot slot_k; eoff = exclusive prefix sums of w_k, roff =
// exclusive prefix sums of the participants' estimator counts r_k):
//   descriptor  u64 words: eoff[K+1], D_k pointers[K], roff[K+1], slot_k[K]
//   arc keys    k << (B+bw+1) | pi(src) << (bw+1) | (w_k-1-j) << 1 | side,
//               pi a bijection of [0, 2^B) (multiplication by an odd
//               Fibonacci-hashing constant mod 2^B) that spreads any set of
//               ids evenly over the range; written participant-major in
//               decreasing local position j and sorted on the (k, pi(src))
//               bits: every participant's arcs end up in its own range
//               [2 eoff_k, 2 eoff_k + 2 w_k), each vertex's arcs contiguous
//               in Lemma 4.3's order;
//   edge keys   k << (32+bw) | h << bw | j, h = edge_hash(u, v) (or k << 32 | h
//               with value j when kb + 32 + bw > 64), sorted on k and the top
//               hs bits of h (whole digits, hs >= bw + 1 where they fit):
//               participant k's keys end up in [eoff_k, eoff_k + w_k), and
//               a lookup scans the short run sharing the probe's sorted bits,
//               checking each candidate with its whole hash against D_k;
//   directories bucket directories over the two sorted arrays, like the
//               single-stream Step-3 directory: arcs by the top hA bits of
//               (k, pi(src)), Step-3 keys by the top hE bits of their sorted
//               (k, hash) bits; a lookup reads its bucket's [start, end) and
//               searches only there.  Entries carry the round set's tag, a
//               device word that each round's bookkeeping advances (so a
//               replayed CUDA graph gets a fresh tag every time);
//   sweep       one thread per estimator of the participants only (roff).
//   bw = bits of (max_k w_k) - 1, kb = bits of K-1, B = vertex id bits.
#include <algorithm>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include "tc_kernels.cuh"
#include "tc_nvtx.h"
#include "tc_multi_impl.cuh"

using namespace tc;

namespace {

#define TCM_CUDA(call)                        \
    do {                                      \
        if ((call) != cudaSuccess) return TC_ERR_CUDA; \
    } while (0)

struct RoundShape {
    u32 K;      // participants
    u32 kb;     // participant index bits
    u32 B;      // vertex id bits
    u32 bw;     // bits of max w_k - 1
    u32 sha;    // arc key: src shift = bw + 1
    u64 Wt;     // edges this round
    int npa, npe;
    u32 bits_a, bits_e;
    u32 eko;    // 1: Step-3 keys carry j in their low bw bits (else as a value)
    u32 hs;     // Step-3 hash bits sorted (the top of h)
    u32 she;    // Step-3 key: first sorted bit ((bw or 0) + 32 - hs)
    u32 ha_sh;  // arc bucket: (k, pi(src)) >> ha_sh, 2^hA buckets
    u32 he_sh;  // Step-3 bucket: sorted bits >> he_sh, 2^hE buckets
    u64 nba, nbe;   // 2^hA, 2^hE
    u64 pmul;   // pi: x -> x * pmul mod 2^B (pmul odd)
    u64 hkey;   // key of the Step-3 edge hash
};

// pi(x): the vertex id bijection of the arc keys.
__device__ __forceinline__ u64 vperm(const RoundShape &rs, u64 x) {
    return (x * rs.pmul) & ((rs.B >= 64) ? ~0ull : ((1ull << rs.B) - 1));
}

// Step-3 key of participant k's edge at local position j with hash h.
__device__ __forceinline__ u64 mkey(const RoundShape &rs, u64 k, u64 h, u64 j) {
    return rs.eko ? (k << (32 + rs.bw)) | (h << rs.bw) | j : (k << 32) | h;
}

// (participant, hash) part of a Step-3 key.
__device__ __forceinline__ u64 mkey_prefix(const RoundShape &rs, u64 key) {
    return rs.eko ? key >> rs.bw : key;
}

// The sorted part of a Step-3 key: participant and the top hs hash bits.
__device__ __forceinline__ u64 mkey_sorted(const RoundShape &rs, u64 key) {
    return key >> rs.she;
}

// Views of a round descriptor.
struct Desc {
    const u64 *eoff;              // K+1
    const u64 *const *ebase;      // K
    const u64 *roff;              // K+1
    const u64 *slot;              // K
};

__device__ __forceinline__ Desc desc_view(const u64 *d, u32 K) {
    Desc v;
    v.eoff = d;
    v.ebase = reinterpret_cast<const u64 *const *>(d + K + 1);
    v.roff = d + 2 * K + 1;
    v.slot = d + 3 * K + 2;
    return v;
}

__device__ __forceinline__ u32 segment_of(const u64 *__restrict__ off, u32 K, u64 x) {
    // last k with off[k] <= x (off has K+1 entries, off[0] = 0)
    u32 lo = 0, hi = K;
    while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

constexpr int kMThreads = 256;

__global__ void __launch_bounds__(kMThreads) mprep_kernel(const u64 *__restrict__ desc,
                                                           RoundShape rs, u32 *perr,
                                                           u64 *__restrict__ arcs0,
                                                           u64 *__restrict__ ekeys0,
                                                           u32 *__restrict__ evals0,
                                                           SortPlan *plans) {
    extern __shared__ u32 h[];
    const Desc d = desc_view(desc, rs.K);
    const u32 ra = 1u << rs.bits_a, re = 1u << rs.bits_e;
    const u32 na = (u32)rs.npa * ra, nh = na + (u32)rs.npe * re;
    u32 *he = h + na;
    for (u32 k = threadIdx.x; k < nh; k += kMThreads) h[k] = 0;
    __syncthreads();
    const u64 id_lim = (rs.B >= 32) ? (1ull << 32) : (1ull << rs.B);
    for (u64 j = (u64)blockIdx.x * kMThreads + threadIdx.x; j < rs.Wt;
         j += (u64)gridDim.x * kMThreads) {
        const u32 k = segment_of(d.eoff, rs.K, j);
        const u64 e0 = __ldg(d.eoff + k), ws = __ldg(d.eoff + k + 1) - e0;
        const u64 jl = j - e0;
        const u64 e = d.ebase[k][jl];
        const u64 u = e >> 32, v = e & kMask32;
        if (!(u < v) || v >= id_lim) atomicOr(&perr[k], kErrInput);
        const u64 sp = (u64)k << (rs.B + rs.sha);
        const u64 rpos = (ws - 1 - jl) << 1;
        const u64 au = sp | (vperm(rs, u) << rs.sha) | rpos;
        const u64 av = sp | (vperm(rs, v) << rs.sha) | rpos | 1ull;
        reinterpret_cast<ulonglong2 *>(arcs0)[e0 + ws - 1 - jl] = make_ulonglong2(au, av);
        for (int p = 0; p < rs.npa; ++p) {
            atomicAdd(&h[p * ra + digit_bits(au, rs.sha + p * rs.bits_a, ra - 1)], 1u);
            atomicAdd(&h[p * ra + digit_bits(av, rs.sha + p * rs.bits_a, ra - 1)], 1u);
        }
        const u64 ek = mkey(rs, k, edge_hash(e, rs.hkey), jl);
        ekeys0[j] = ek;
        if (!rs.eko) evals0[j] = (u32)jl;
        for (int p = 0; p < rs.npe; ++p)
            atomicAdd(&he[p * re + digit_bits(ek, rs.she + p * rs.bits_e, re - 1)], 1u);
    }
    __syncthreads();
    for (u32 k = threadIdx.x; k < nh; k += kMThreads) {
        const u32 c = h[k];
        if (!c) continue;
        if (k < na) atomicAdd(&plans[0].counts[k / ra][k % ra], c);
        else atomicAdd(&plans[1].counts[(k - na) / re][(k - na) % re], c);
    }
}

// Repeats inside one participant's batch share participant and hash, so
// they lie in one run of equal (participant, hash) after the edge sort: each
// key compares its edge with those of the rest of its run (almost always
// empty).
// Bucket directory over a sorted array: the first key of bucket x writes
// (tag, start), the last one writes end; x = key >> shift.  prev / next: the
// neighbouring keys (ignored at the array's ends).
__device__ __forceinline__ void dir_mark(DirEntry *dir, u64 nb, u32 tag, u64 n, u64 i, u64 key,
                                         u64 prev_key, u64 next_key, u32 shift) {
    const u64 x = key >> shift;
    if (x >= nb) return;  // only keys of a rejected batch; never looked up
    const u64 prev = i ? prev_key >> shift : ~0ull;
    const u64 next = i + 1 < n ? next_key >> shift : ~0ull;
    if (x != prev) *reinterpret_cast<u64 *>(&dir[x].epoch) = (i << 32) | tag;
    if (x != next) dir[x].end = (u32)(i + 1);
}

// Stage keys [t0 - 1, t0 + kIdxTile] of K (n keys) into st[0 .. kIdxTile + 1]
// with coalesced loads; keys outside the array read as 0.
__device__ __forceinline__ void stage_tile(u64 *st, const u64 *K, u64 n, u64 t0) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int j = 0; j < kIdxItems; ++j) {
        const u64 k = t0 + (u64)(j * kIdxThreads + tid);
        st[1 + j * kIdxThreads + tid] = k < n ? __ldg(K + k) : 0ull;
    }
    if (tid == 0) st[0] = t0 ? __ldg(K + t0 - 1) : 0ull;
    if (tid == 1) st[kIdxTile + 1] = t0 + kIdxTile < n ? __ldg(K + t0 + kIdxTile) : 0ull;
}

// Arc bucket directory (after the arc sort).
__global__ void __launch_bounds__(kIdxThreads) marc_index_kernel(const u64 *arcs0,
                                                                 const u64 *arcs1,
                                                                 const SortPlan *plans,
                                                                 RoundShape rs, DirEntry *adir,
                                                                 const u32 *tagp) {
    __shared__ u64 st[kIdxTile + 2];
    const u64 *A = plan_final_sel(&plans[0]) ? arcs1 : arcs0;
    const u32 tag = *tagp;
    const u64 n = 2 * rs.Wt;
    for (u64 t0 = (u64)blockIdx.x * kIdxTile; t0 < n; t0 += (u64)gridDim.x * kIdxTile) {
        stage_tile(st, A, n, t0);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kIdxItems; ++j) {
            const int i = j * kIdxThreads + threadIdx.x;
            if (t0 + i >= n) break;
            dir_mark(adir, rs.nba, tag, n, t0 + i, st[1 + i], st[i], st[i + 2],
                     rs.sha + rs.ha_sh);
        }
        __syncthreads();  // the tile is restaged next
    }
}

// Step-3 bucket directory and the in-round repeat check (after the Step-3
// sort).
__global__ void __launch_bounds__(kIdxThreads) mdups_kernel(
    const u64 *ekeys0, const u64 *ekeys1, const u32 *evals0, const u32 *evals1,
    const SortPlan *plans, const u64 *__restrict__ desc, RoundShape rs, u32 *perr,
    DirEntry *edir, const u32 *tagp) {
    __shared__ u64 st[kIdxTile + 2];
    const Desc d = desc_view(desc, rs.K);
    const bool sel = plan_final_sel(&plans[1]) != 0;
    const u64 *E = sel ? ekeys1 : ekeys0;
    const u32 *EV = sel ? evals1 : evals0;
    const u64 jmask = (1ull << rs.bw) - 1;
    const u32 tag = *tagp;
    const u64 n = rs.Wt;
    for (u64 t0 = (u64)blockIdx.x * kIdxTile; t0 < n; t0 += (u64)gridDim.x * kIdxTile) {
        stage_tile(st, E, n, t0);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kIdxItems; ++j) {
            const int ti = j * kIdxThreads + threadIdx.x;
            const u64 i = t0 + ti;
            if (i >= n) break;
            const u64 a = st[1 + ti];
            dir_mark(edir, rs.nbe, tag, n, i, a, st[ti], st[ti + 2], rs.she + rs.he_sh);
            const u64 sa = mkey_sorted(rs, a), pa = mkey_prefix(rs, a);
            if (i + 1 >= n || mkey_sorted(rs, st[ti + 2]) != sa) continue;
            // a repeat shares the whole hash, so it lies in the run of equal
            // sorted bits that follows (almost always empty)
            const u64 k = rs.eko ? a >> (32 + rs.bw) : a >> 32;
            const u64 *D = d.ebase[k];
            u64 ea = 0;
            bool have = false;
            for (u64 q = i + 1; q < n; ++q) {
                const u64 b = __ldg(E + q);
                if (mkey_sorted(rs, b) != sa) break;
                if (mkey_prefix(rs, b) != pa) continue;
                if (!have) {
                    ea = __ldg(D + (rs.eko ? (a & jmask) : __ldg(EV + i)));
                    have = true;
                }
                if (__ldg(D + (rs.eko ? (b & jmask) : __ldg(EV + q))) == ea) {
                    atomicOr(&perr[k], kErrInput);
                    break;
                }
            }
        }
        __syncthreads();  // the tile is restaged next
    }
}

struct MSweepArgs {
    const u64 *desc;
    u64 R;               // estimators of the participants
    const u64 *arcs0, *arcs1, *ekeys0, *ekeys1;
    const u32 *evals0, *evals1;
    const SortPlan *plans;
    MStream *ms;
    const u32 *gerr;     // round-wide error (a timed-out sort)
    const u32 *perr;     // each participant's error this round
    const DirEntry *adir, *edir;
    const u32 *tag;      // the round set's directory tag
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

// The arcs [start, end) of vertex prefix x = (k, pi(src)): its bucket's
// range from the directory, then the run of keys with that prefix in it.
// First index in [lo, hi) of the sorted array a with a[idx] >= key (hi if
// none).  Indices are 32-bit: a round holds fewer than 2^29 arcs.
__device__ __forceinline__ u32 lower_bound32(const u64 *__restrict__ a, u32 lo, u32 hi,
                                             u64 key) {
    u32 n = hi - lo;
    while (n > 0) {
        const u32 half = n >> 1;
        if (__ldg(a + lo + half) < key) {
            lo += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    return lo;
}

// The arcs [start, end) of vertex prefix x = (k, pi(src)): its bucket's
// range from the directory, then the run of keys with that prefix in it.
__device__ __forceinline__ void vertex_arcs(const DirEntry *adir, u32 tag, const u64 *arcs,
                                            const RoundShape &rs, u64 x, u32 &start, u32 &end) {
    const uint4 e = __ldg(reinterpret_cast<const uint4 *>(adir + (x >> rs.ha_sh)));
    const u32 n_arcs = (u32)(2 * rs.Wt);
    const bool hit = e.x == tag;
    // (clamped to start <= end <= n, as dir_segment)
    const u32 hi = hit ? min(e.z, n_arcs) : 0u, lo = hit ? min(e.y, hi) : 0u;
    if (lo < hi) {
        // the bucket's first and last keys: usually the bucket holds one
        // vertex (or x is outside it), which settles the run at once
        const u64 p0 = __ldg(arcs + lo) >> rs.sha, p1 = __ldg(arcs + hi - 1) >> rs.sha;
        if (p0 == x && p1 == x) {
            start = lo;
            end = hi;
            return;
        }
        if (x < p0 || x > p1) {
            start = end = lo;
            return;
        }
    }
    start = lower_bound32(arcs, lo, hi, x << rs.sha);
    // first key past the prefix: compare prefixes (x + 1 << sha may not fit)
    u32 b = start, n = hi - start;
    while (n > 0) {
        const u32 half = n >> 1;
        if ((__ldg(arcs + b + half) >> rs.sha) <= x) {
            b += half + 1;
            n -= half + 1;
        } else {
            n = half;
        }
    }
    end = b;
}

// Positions and indices are 32-bit (a round holds fewer than 2^29 arcs and a
// stream fewer than 2^32 estimators), which keeps the live registers down;
// at 7 blocks per SM (32 registers, some spills to local memory) rounds were
// 3% faster than at 6 and 5.
__global__ void __launch_bounds__(kMThreads, 7) msweep_kernel(MSweepArgs a) {
    __shared__ u32 s_k[2];
    if (ld_relaxed(a.gerr)) return;
    const u64 g0 = (u64)blockIdx.x * kMThreads;
    const u64 g = g0 + threadIdx.x;
    const RoundShape &rs = a.rs;
    const Desc d = desc_view(a.desc, rs.K);
    // participants of the block's first and last estimators: usually the
    // same, else every thread searches only between them
    if (threadIdx.x == 0) s_k[0] = segment_of(d.roff, rs.K, g0);
    if (threadIdx.x == 32) s_k[1] = segment_of(d.roff, rs.K, min(g0 + kMThreads, a.R) - 1);
    __syncthreads();
    u32 k = 0xFFFFFFFFu;
    u64 add = 0, closed = 0;
    if (g < a.R) {
        u32 lo = s_k[0], hi = s_k[1] + 1;  // last k in [lo, hi) with roff[k] <= g
        while (hi - lo > 1) {
            const u32 mid = (lo + hi) >> 1;
            if (__ldg(d.roff + mid) <= g) lo = mid;
            else hi = mid;
        }
        k = lo;
        const u32 ws = (u32)(__ldg(d.eoff + k + 1) - __ldg(d.eoff + k));
        MStream &st = a.ms[__ldg(d.slot + k)];
        if (ws > 0 && !ld_relaxed(a.perr + k)) {
            const u32 i = (u32)(g - __ldg(d.roff + k));
            const u64 m = st.m;
            const DrawKey dk{st.key, (u32)st.batches, st.stream_id};
            const u64 *D = d.ebase[k];
            u64 *const F1 = st.f1, *const F2 = st.f2, *const CHI = st.chi;
            u32 *const FL = st.flags;
            const u64 *arcs = plan_final_sel(&a.plans[0]) ? a.arcs1 : a.arcs0;
            const u32 wmask = (u32)((1ull << rs.bw) - 1);
            const u32 tag = *a.tag;
            // the state streams through once: evict-first, so that L2 keeps
            // the directories and sorted arrays the searches hit at random
            u64 f1 = __ldcs(F1 + i), f2 = __ldcs(F2 + i), chi = __ldcs(CHI + i);
            u32 fl = __ldcs(FL + i);
            // ---- Step 1 (Sec. 4.2)
            const u64 x = draw_bounded(dk, i, kStep1, m + ws);
            const bool new1 = x >= m;
            u32 p1 = 0;
            if (new1) {
                p1 = (u32)(x - m);
                f1 = __ldg(D + p1);
                chi = 0;
                f2 = kEmpty;
                fl = 0;
            }
            // ---- Step 2 (Sec. 4.3): each endpoint's arcs, from its bucket
            const u64 xu = ((u64)k << rs.B) | vperm(rs, f1 >> 32);
            const u64 xv = ((u64)k << rs.B) | vperm(rs, f1 & kMask32);
            u32 su, eu, sv, ev;
            vertex_arcs(a.adir, tag, arcs, rs, xu, su, eu);
            vertex_arcs(a.adir, tag, arcs, rs, xv, sv, ev);
            u32 ld, rd;
            if (new1) {
                const u64 rp = (u64)(ws - 1 - p1) << 1;
                ld = lower_bound32(arcs, su, eu, (xu << rs.sha) | rp) - su;
                rd = lower_bound32(arcs, sv, ev, (xv << rs.sha) | rp) - sv;
            } else {
                ld = eu - su;
                rd = ev - sv;
            }
            const u64 chi_plus = (u64)ld + rd;
            bool new2 = false;
            u32 p2 = 0;
            if (chi_plus > 0) {
                const u64 y = draw_bounded(dk, i, kStep2, chi + chi_plus);
                if (y >= chi) {
                    const u32 phi = (u32)(y - chi);
                    const u32 q = (phi < ld) ? su + phi : sv + (phi - ld);
                    p2 = ws - 1 - ((u32)(__ldg(arcs + q) >> 1) & wmask);
                    f2 = __ldg(D + p2);
                    fl &= ~TC_FLAG_CLOSED;
                    new2 = true;
                }
            }
            chi += chi_plus;
            // ---- Step 3 (Sec. 4.4): by the closing edge's hash, each
            // candidate checked against the batch itself
            if (f2 != kEmpty && !(fl & TC_FLAG_CLOSED)) {
                const u64 a1 = f1 >> 32, b1 = f1 & kMask32, a2 = f2 >> 32, b2 = f2 & kMask32;
                const u64 x1 = (a1 == a2 || a1 == b2) ? b1 : a1;
                const u64 x2 = (a2 == a1 || a2 == b1) ? b2 : a2;
                const u64 gu = x1 < x2 ? x1 : x2, gv = x1 < x2 ? x2 : x1;
                const u64 gkey = (gu << 32) | gv;
                const u64 probe = mkey(rs, k, edge_hash(gkey, rs.hkey), 0);
                const u64 pp = mkey_prefix(rs, probe), ps = mkey_sorted(rs, probe);
                const bool es = plan_final_sel(&a.plans[1]) != 0;
                const u64 *E = es ? a.ekeys1 : a.ekeys0;
                const u32 *EV = es ? a.evals1 : a.evals0;
                u64 lo64, hi64;
                dir_segment(a.edir, tag, ps >> rs.he_sh, rs.Wt, lo64, hi64);
                const u32 qhi = (u32)hi64;
                for (u32 q = lower_bound32(E, (u32)lo64, qhi, ps << rs.she); q < qhi; ++q) {
                    const u64 ek = __ldg(E + q);
                    if (mkey_sorted(rs, ek) != ps) break;
                    if (mkey_prefix(rs, ek) != pp) continue;
                    const u32 pq = rs.eko ? ((u32)ek & wmask) : __ldg(EV + q);
                    if (__ldg(D + pq) == gkey) {
                        if (!new2 || pq > p2) fl |= TC_FLAG_CLOSED;
                        break;
                    }
                }
            }
            __stcs(F1 + i, f1);
            __stcs(F2 + i, f2);
            __stcs(CHI + i, chi);
            __stcs(FL + i, fl);
            if (fl & TC_FLAG_CLOSED) {
                add = chi;
                closed = 1;
            }
        } else {
            k = 0xFFFFFFFFu;  // rejected batch: contributes nothing
        }
    }
    u64 hi = 0;
    if (warp_segment_sum(k, add, hi, closed) && k != 0xFFFFFFFFu) {
        MStream &st = a.ms[__ldg(d.slot + k)];
        if (add | hi) add_u128(st.acc, add, hi);
        if (closed) atomicAdd((unsigned long long *)&st.acc[2], (unsigned long long)closed);
    }
}

__device__ __forceinline__ void write_record(u64 *o, u32 status, const MStream &st) {
    o[0] = status;
    o[1] = st.batches;
    o[2] = st.est[0];
    o[3] = st.est[1];
    o[4] = st.est[2];
    o[5] = st.est[3];
}

// Close the round for every participant.
__global__ void mfinish_kernel(MStream *ms, const u64 *__restrict__ desc, u32 K, u32 *gerr,
                               const u32 *perr, u64 *out, u32 *tag) {
    const u32 k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    if (k == 0) {  // the set's next round writes its directories under a new tag
        const u32 t = *tag + 1;
        *tag = t ? t : 1;
    }
    const Desc d = desc_view(desc, K);
    MStream &st = ms[d.slot[k]];
    const u64 ws = d.eoff[k + 1] - d.eoff[k];
    const u32 e = perr[k] ? perr[k] : *gerr;
    if (e) {
        if (!st.sticky) st.sticky = e;
    } else if (ws > 0) {
        st.m += ws;
        st.batches += 1;
        st.est[0] = st.acc[0];
        st.est[1] = st.acc[1];
        st.est[2] = st.acc[2];
        st.est[3] = st.m;
    }
    if (out) write_record(out + (u64)k * kRecordWords, e, st);
    st.acc[0] = st.acc[1] = st.acc[2] = 0;
}

// tc_multi_estimates_async: every slot's estimate record (zero for an empty
// slot), formed as tc_multi_estimate forms it on the host.
__global__ void mestimate_kernel(const MStream *ms, u32 S, tc_estimate_t *out) {
    const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const MStream &st = ms[s];
    if (st.r == 0) {
        out[s] = tc_estimate_t{};
        return;
    }
    finish_estimate(st.est[0], st.est[1], st.est[2], st.m, st.r, st.batches, out + s);
}

__global__ void mgather_kernel(const MStream *ms, const u32 *slots, u32 Q, u64 *out) {
    const u32 q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < Q) write_record(out + (u64)q * kRecordWords, 0, ms[slots[q]]);
}

// Reset one slot: its record, and its r estimators to the empty state.
__global__ void mopen_kernel(MStream *ms, u32 slot, MStream rec) {
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) ms[slot] = rec;
    if (i < rec.r) {
        rec.f1[i] = kEmpty;
        rec.f2[i] = kEmpty;
        rec.chi[i] = 0;
        rec.flags[i] = 0;
    }
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

// Bytes of the zero-initialised scratch block: SortPlan[2], the worst-case
// look-back of both sorts for any digit width, 256 bytes for the error word.
u64 zeroed_bytes_for(u32 sb, u64 w_max_round, u32 vertex_bits) {
    u64 lb = 0;
    for (u32 ba : {8u, 10u, 11u})
        for (u32 be : {8u, 10u, 11u}) {
            int pa, pe;
            mpick(vertex_bits + sb, ba, pa);
            mpick(32 + sb, be, pe);
            lb = std::max(lb, (u64)pa * mlookback(2 * w_max_round, ba) +
                                  (u64)pe * mlookback(w_max_round, be));
        }
    return 2 * sizeof(SortPlan) + lb * sizeof(u32) + 256;
}

// Bucket bits of the two round directories for Wt edges (at most, before
// the clamp to the sorted bits): between 2 Wt and 4 Wt arc buckets (a
// bucket then mostly holds one vertex's arcs; 3% faster rounds at 512
// streams than 2 Wt / 4) and about Wt / 4 Step-3 buckets.
u32 arc_dir_bits(u64 Wt) {
    return mbits_for(2 * Wt - 1);
}
u32 edge_dir_bits(u64 Wt) {
    const u32 b = mbits_for(Wt - 1);
    return b > 3 ? b - 2 : 1;
}

// pi's multiplier for B-bit ids: the odd integer next to 2^B / phi
// (Fibonacci hashing, Knuth TAOCP vol. 3, 6.4).
u64 fib_multiplier(u32 B) {
    return (u64)(0.6180339887498949 * (double)(1ull << B)) | 1ull;
}

// Bytes of one round set's directories and tag word.
u64 dir_bytes(u64 w_max_round) {
    return ((1ull << arc_dir_bits(w_max_round)) + (1ull << edge_dir_bits(w_max_round))) *
               sizeof(DirEntry) + 256;
}

// Participant error words at the end of the zeroed block, one per slot at most.
u64 perr_bytes(u32 S) { return ((u64)S * 4 + 255) & ~255ull; }

// Rounds a set's directory tags may serve before the set is cleared: each
// round advances the 32-bit tag (skipping 0), so well before it could come
// back to a value still held by a stale entry, every entry is reset to tag 0
// and the tag restarts at 1.
constexpr u64 kTagRoundsMax = 0xFFFFFF00ull;

// Per-stream state block bytes (f1, f2, chi, flags), padded to 256 bytes.
u64 state_bytes(u64 r) { return (28 * r + 255) & ~255ull; }

}  // namespace

namespace tc {

u64 multi_scratch_bytes(u32 S, u64 w_max_round, u32 vertex_bits, int sets) {
    const u32 sb = mbits_for(S - 1);
    const u64 per_set = 2 * (2 * w_max_round * 8 + w_max_round * 8 + w_max_round * 4) +
                        zeroed_bytes_for(sb, w_max_round, vertex_bits) + perr_bytes(S) +
                        dir_bytes(w_max_round);
    return (u64)S * sizeof(MStream) + (u64)sets * per_set + kRing * desc_words(S) * 8;
}

static void free_round_set(tc_multi::RoundSet &z) {
    for (int k = 0; k < 2; ++k) {
        cudaFree(z.arcs[k]);
        cudaFree(z.ekeys[k]);
        cudaFree(z.evals[k]);
    }
    cudaFree(z.zeroed);
    cudaFree(z.adir);
    cudaFree(z.edir);
    cudaFree(z.tag);
    z = tc_multi::RoundSet{};
}

// Allocate one set of round scratch: the sort buffers, the zeroed block,
// the two directories (tag 0 everywhere) and the tag word (1: the first
// round's tag).  On failure the set is freed and false returned.
// Before a set's tag could wrap: wait for the device, reset every directory
// entry of the set to tag 0 and its tag word to 1.
static int clear_tags_if_due(tc_multi *M, int b) {
    if (M->set_rounds[b] < kTagRoundsMax) return TC_OK;
    tc_multi::RoundSet &z = M->rset[b];
    const u64 na = 1ull << arc_dir_bits(M->w_max), ne = 1ull << edge_dir_bits(M->w_max);
    const u32 one = 1;
    TCM_CUDA(cudaDeviceSynchronize());
    TCM_CUDA(cudaMemset(z.adir, 0, na * sizeof(DirEntry)));
    TCM_CUDA(cudaMemset(z.edir, 0, ne * sizeof(DirEntry)));
    TCM_CUDA(cudaMemcpy(z.tag, &one, sizeof(one), cudaMemcpyHostToDevice));
    M->set_rounds[b] = 0;
    return TC_OK;
}

static bool alloc_round_set(tc_multi::RoundSet &z, u64 w_max, u64 zeroed_bytes) {
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        ok &= cudaMalloc(&z.arcs[k], 2 * w_max * sizeof(u64)) == cudaSuccess;
        ok &= ok && cudaMalloc(&z.ekeys[k], w_max * sizeof(u64)) == cudaSuccess;
        ok &= ok && cudaMalloc(&z.evals[k], w_max * sizeof(u32)) == cudaSuccess;
    }
    ok &= ok && cudaMalloc(&z.zeroed, zeroed_bytes) == cudaSuccess;
    ok &= ok && cudaMemset(z.zeroed, 0, zeroed_bytes) == cudaSuccess;
    const u64 na = 1ull << arc_dir_bits(w_max), ne = 1ull << edge_dir_bits(w_max);
    ok &= ok && cudaMalloc(&z.adir, na * sizeof(DirEntry)) == cudaSuccess;
    ok &= ok && cudaMemset(z.adir, 0, na * sizeof(DirEntry)) == cudaSuccess;
    ok &= ok && cudaMalloc(&z.edir, ne * sizeof(DirEntry)) == cudaSuccess;
    ok &= ok && cudaMemset(z.edir, 0, ne * sizeof(DirEntry)) == cudaSuccess;
    const u32 one = 1;
    ok &= ok && cudaMalloc(&z.tag, 256) == cudaSuccess;
    ok &= ok && cudaMemcpy(z.tag, &one, sizeof(one), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) free_round_set(z);
    return ok;
}

void multi_free(tc_multi *M) {
    cudaDeviceSynchronize();
    cudaFree(M->state);
    cudaFree(M->ms);
    for (tc_multi::RoundSet &z : M->rset) free_round_set(z);
    if (M->sa) cudaStreamDestroy(M->sa);
    for (int k = 0; k < 2; ++k) {
        if (M->ev_sorted[k]) cudaEventDestroy(M->ev_sorted[k]);
        if (M->ev_swept[k]) cudaEventDestroy(M->ev_swept[k]);
    }
    for (int k = 0; k < kRing; ++k) {
        cudaFree(M->desc[k]);
        if (M->h_desc[k]) cudaFreeHost(M->h_desc[k]);
        if (M->ring_ev[k]) cudaEventDestroy(M->ring_ev[k]);
    }
    if (M->h_ms) cudaFreeHost(M->h_ms);
    if (M->gexec) cudaGraphExecDestroy(M->gexec);
    cudaFree(M->g_desc);
    if (M->side) cudaStreamDestroy(M->side);
    if (M->ev_fork) cudaEventDestroy(M->ev_fork);
    if (M->ev_join) cudaEventDestroy(M->ev_join);
    delete M;
}

int multi_alloc(u32 S, u64 w_max_round, u32 vertex_bits, tc_multi **out, int sets) {
    *out = nullptr;
    if (S == 0 || w_max_round == 0 || w_max_round > (1ull << 28) || vertex_bits < 1 ||
        vertex_bits > 32)
        return TC_ERR_INVAL;
    const u32 sb = mbits_for(S - 1);
    const u32 bwmax = mbits_for(w_max_round - 1);
    if (sb + vertex_bits + bwmax + 1 > 64) return TC_ERR_INVAL;
    int rc = mconfigure();
    if (rc) return rc;
    tc_multi *M = new (std::nothrow) tc_multi();
    if (!M) return TC_ERR_NOMEM;
    M->S = S;
    M->hash_key = random_hash_key();
    M->B = vertex_bits;
    M->sb = sb;
    M->w_max = w_max_round;
    M->rank = kRankBallot;
    M->h_rec.assign(S, MStream{});
    M->zeroed_bytes = zeroed_bytes_for(sb, w_max_round, vertex_bits) + perr_bytes(S);
    M->nsets = sets == 2 ? 2 : 1;
    bool ok = cudaMalloc(&M->ms, S * sizeof(MStream)) == cudaSuccess;
    for (int z = 0; z < M->nsets && ok; ++z)
        ok &= alloc_round_set(M->rset[z], w_max_round, M->zeroed_bytes);
    ok &= ok && cudaStreamCreateWithFlags(&M->sa, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k) {
        ok &= cudaEventCreateWithFlags(&M->ev_sorted[k], cudaEventDisableTiming) == cudaSuccess;
        ok &= ok && cudaEventCreateWithFlags(&M->ev_swept[k], cudaEventDisableTiming) == cudaSuccess;
    }
    for (int k = 0; k < kRing && ok; ++k) {
        ok &= cudaMalloc(&M->desc[k], desc_words(S) * sizeof(u64)) == cudaSuccess;
        ok &= ok && cudaHostAlloc(&M->h_desc[k], desc_words(S) * sizeof(u64),
                                  cudaHostAllocMapped) == cudaSuccess;
        M->h_desc_dev[k] = ok ? static_cast<u64 *>(mapped_device_ptr(M->h_desc[k])) : nullptr;
        ok &= M->h_desc_dev[k] != nullptr;
        ok &= ok && cudaEventCreateWithFlags(&M->ring_ev[k], cudaEventDisableTiming) == cudaSuccess;
    }
    ok &= ok && cudaHostAlloc(&M->h_ms, S * sizeof(MStream), cudaHostAllocDefault) == cudaSuccess;
    ok &= ok && cudaStreamCreateWithFlags(&M->side, cudaStreamNonBlocking) == cudaSuccess;
    ok &= ok && cudaEventCreateWithFlags(&M->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok &= ok && cudaEventCreateWithFlags(&M->ev_join, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        ok &= cudaMemset(M->ms, 0, S * sizeof(MStream)) == cudaSuccess;
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

int multi_open_slot(tc_multi *M, u32 slot, u64 r, u64 seed, u32 stream_id, void *state,
                    cudaStream_t st) {
    if (slot >= M->S || r == 0 || r > 0xFFFFFFFFull || !state) return TC_ERR_INVAL;
    MStream rec{};
    u64 *base = static_cast<u64 *>(state);
    rec.f1 = base;
    rec.f2 = base + r;
    rec.chi = base + 2 * r;
    rec.flags = reinterpret_cast<u32 *>(base + 3 * r);
    rec.r = r;
    rec.key = make_uint2((u32)(seed & 0xFFFFFFFFu), (u32)(seed >> 32));
    rec.stream_id = stream_id;
    const u64 blocks = (r + 255) / 256;
    mopen_kernel<<<(unsigned)blocks, 256, 0, st>>>(M->ms, slot, rec);
    TCM_CUDA(cudaGetLastError());
    M->h_rec[slot] = rec;
    M->launches += 1;
    return TC_OK;
}

u64 write_descriptor(const tc_multi *M, const RoundItem *items, u32 K, u64 *h) {
    u64 *eoff = h, *ebase = h + K + 1, *roff = h + 2 * K + 1, *slot = h + 3 * K + 2;
    u64 wmax = 0;
    eoff[0] = 0;
    roff[0] = 0;
    for (u32 k = 0; k < K; ++k) {
        eoff[k + 1] = eoff[k] + items[k].w;
        ebase[k] = (u64)items[k].edges;
        roff[k + 1] = roff[k] + M->h_rec[items[k].slot].r;
        slot[k] = items[k].slot;
        wmax = std::max(wmax, items[k].w);
    }
    return wmax;
}

static __global__ void __launch_bounds__(256) copy_words_kernel(u64 *__restrict__ dst,
                                                                const u64 *__restrict__ src,
                                                                u64 n) {
    for (u64 i = (u64)blockIdx.x * 256 + threadIdx.x; i < n; i += (u64)gridDim.x * 256)
        dst[i] = src[i];
}

int copy_words_async(tc_multi *M, u64 *dst, const u64 *src, u64 n, cudaStream_t st) {
    if (n == 0) return TC_OK;
    const u64 blocks = std::min<u64>((n + 255) / 256, 64);
    copy_words_kernel<<<(unsigned)blocks, 256, 0, st>>>(dst, src, n);
    TCM_CUDA(cudaGetLastError());
    if (M) M->launches += 1;
    return TC_OK;
}

void *mapped_device_ptr(void *h) {
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return d;
}

int multi_gather(tc_multi *M, const u32 *d_slots, u32 Q, u64 *out, cudaStream_t st) {
    if (Q == 0) return TC_OK;
    mgather_kernel<<<(Q + 255) / 256, 256, 0, st>>>(M->ms, d_slots, Q, out);
    TCM_CUDA(cudaGetLastError());
    M->launches += 1;
    return TC_OK;
}

int multi_enqueue(tc_multi *M, const RoundItem *items, u32 K, u64 *desc, const u64 *h_desc,
                  u64 *out, cudaStream_t st, bool pipelined, cudaEvent_t wait_ev,
                  cudaEvent_t ev_sort0, cudaEvent_t ev_sort1) {
    const NvtxRange range("tc round");
    u64 Wt = 0, wmax = 0, R = 0;
    for (u32 k = 0; k < K; ++k) {
        Wt += items[k].w;
        wmax = std::max(wmax, items[k].w);
        R += M->h_rec[items[k].slot].r;
    }
    if (K == 0 || Wt == 0 || Wt > M->w_max) return TC_ERR_INVAL;
    if (pipelined && M->nsets != 2) return TC_ERR_INVAL;
    RoundShape rs{};
    rs.K = K;
    rs.kb = mbits_for(K - 1);
    rs.B = M->B;
    rs.bw = mbits_for(wmax - 1);
    rs.sha = rs.bw + 1;
    rs.Wt = Wt;
    rs.bits_a = mpick(M->B + rs.kb, M->force_a, rs.npa);
    // Step-3 keys: whole digits covering k and at least bw + 1 hash bits
    // (runs of equal sorted bits then hold half a key on average in the
    // largest batch), at most all 32
    rs.bits_e = mpick(rs.kb + std::min(32u, rs.bw + 1), M->force_e, rs.npe);
    rs.hs = std::min(32u, (u32)rs.npe * rs.bits_e - rs.kb);
    rs.eko = rs.kb + 32 + rs.bw <= 64 ? 1u : 0u;
    rs.she = (rs.eko ? rs.bw : 0u) + 32 - rs.hs;
    // bucket directories: at most the sorted bits
    const u32 ha = std::min(arc_dir_bits(Wt), rs.kb + rs.B);
    const u32 he = std::min(edge_dir_bits(Wt), rs.kb + rs.hs);
    rs.ha_sh = rs.kb + rs.B - ha;
    rs.he_sh = rs.kb + rs.hs - he;
    rs.nba = 1ull << ha;
    rs.nbe = 1ull << he;
    rs.pmul = fib_multiplier(rs.B);
    rs.hkey = M->hash_key;
    const int b = M->nsets == 2 ? (int)(M->rseq & 1) : 0;
    M->rseq++;
    tc_multi::RoundSet &z = M->rset[b];
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    TCM_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap == cudaStreamCaptureStatusNone) {
        const int rc = clear_tags_if_due(M, b);
        if (rc) return rc;
    } else {
        M->graph_set = b;
    }
    M->set_rounds[b]++;
    SortPlan *plans = reinterpret_cast<SortPlan *>(z.zeroed);
    u32 *lb = reinterpret_cast<u32 *>(z.zeroed + 2 * sizeof(SortPlan));
    const u64 la = mlookback(2 * Wt, rs.bits_a), le = mlookback(Wt, rs.bits_e);
    const u64 lwords = (u64)rs.npa * la + (u64)rs.npe * le;
    u32 *perr = reinterpret_cast<u32 *>(z.zeroed + M->zeroed_bytes - perr_bytes(M->S));
    u32 *gerr = reinterpret_cast<u32 *>(reinterpret_cast<unsigned char *>(perr) - 256);
    // the sort phase's stream: the caller's, or the engine's own when pipelined
    cudaStream_t ms = pipelined ? M->sa : st;
    // with two sets, the set's previous round may have been swept on another
    // stream (one set: every round runs in the order of its stream)
    if (M->nsets == 2) TCM_CUDA(cudaStreamWaitEvent(ms, M->ev_swept[b], 0));
    if (wait_ev) TCM_CUDA(cudaStreamWaitEvent(ms, wait_ev, 0));
    if (ev_sort0) TCM_CUDA(cudaEventRecord(ev_sort0, ms));
    if (h_desc) {
        const int rc = copy_words_async(M, desc, h_desc, desc_words(K), ms);
        if (rc) return rc;
    }
    TCM_CUDA(cudaMemsetAsync(z.zeroed, 0, 2 * sizeof(SortPlan) + lwords * sizeof(u32), ms));
    TCM_CUDA(cudaMemsetAsync(gerr, 0, 256 + (u64)K * 4, ms));

    const size_t hsm = (((size_t)rs.npa << rs.bits_a) + ((size_t)rs.npe << rs.bits_e)) * 4;
    const u64 pb = std::min<u64>((Wt + kMThreads * 8 - 1) / (kMThreads * 8), 1216);
    mprep_kernel<<<(unsigned)pb, kMThreads, hsm, ms>>>(desc, rs, perr, z.arcs[0], z.ekeys[0],
                                                       z.evals[0], plans);
    sort_plan_kernel<<<dim3((unsigned)std::max(rs.npa, rs.npe), 2), 256, 0, ms>>>(
        plans, rs.npa, (u32)(2 * Wt), rs.bits_a, rs.npe, (u32)Wt, rs.bits_e);
    const PassK ka = mselect(rs.bits_a, false, M->rank);
    const PassK ke = mselect(rs.bits_e, !rs.eko, M->rank);
    const u64 ta = mtiles(2 * Wt), te = mtiles(Wt);
    // the two sorts are independent: the edge sort forks onto the side stream
    TCM_CUDA(cudaEventRecord(M->ev_fork, ms));
    TCM_CUDA(cudaStreamWaitEvent(M->side, M->ev_fork, 0));
    u32 *lbe = lb + (u64)rs.npa * la;
    for (int p = 0; p < rs.npe; ++p)
        ke.fn<<<(unsigned)te, ke.threads, ke.smem, M->side>>>(
            z.ekeys[0], z.ekeys[1], rs.eko ? nullptr : z.evals[0], rs.eko ? nullptr : z.evals[1],
            (u32)Wt, rs.she + p * rs.bits_e, mlive(rs.hs + rs.kb, rs.bits_e, p), p, &plans[1],
            lbe + (u64)p * le, gerr, nullptr);
    mdups_kernel<<<index_blocks(Wt), kIdxThreads, 0, M->side>>>(
        z.ekeys[0], z.ekeys[1], z.evals[0], z.evals[1], plans, desc, rs, perr, z.edir, z.tag);
    TCM_CUDA(cudaEventRecord(M->ev_join, M->side));
    for (int p = 0; p < rs.npa; ++p)
        ka.fn<<<(unsigned)ta, ka.threads, ka.smem, ms>>>(
            z.arcs[0], z.arcs[1], nullptr, nullptr, (u32)(2 * Wt), rs.sha + p * rs.bits_a,
            mlive(M->B + rs.kb, rs.bits_a, p), p, &plans[0], lb + (u64)p * la, gerr, nullptr);
    marc_index_kernel<<<index_blocks(2 * Wt), kIdxThreads, 0, ms>>>(z.arcs[0], z.arcs[1], plans,
                                                                   rs, z.adir, z.tag);
    TCM_CUDA(cudaStreamWaitEvent(ms, M->ev_join, 0));
    if (ev_sort1) TCM_CUDA(cudaEventRecord(ev_sort1, ms));
    if (pipelined) {
        TCM_CUDA(cudaEventRecord(M->ev_sorted[b], ms));
        TCM_CUDA(cudaStreamWaitEvent(st, M->ev_sorted[b], 0));
    }
    MSweepArgs a{};
    a.desc = desc;
    a.R = R;
    a.arcs0 = z.arcs[0];
    a.arcs1 = z.arcs[1];
    a.ekeys0 = z.ekeys[0];
    a.ekeys1 = z.ekeys[1];
    a.evals0 = z.evals[0];
    a.evals1 = z.evals[1];
    a.plans = plans;
    a.ms = M->ms;
    a.gerr = gerr;
    a.perr = perr;
    a.adir = z.adir;
    a.edir = z.edir;
    a.tag = z.tag;
    a.rs = rs;
    msweep_kernel<<<(unsigned)((R + kMThreads - 1) / kMThreads), kMThreads, 0, st>>>(a);
    mfinish_kernel<<<(K + 255) / 256, 256, 0, st>>>(M->ms, desc, K, gerr, perr, out, z.tag);
    if (M->nsets == 2) TCM_CUDA(cudaEventRecord(M->ev_swept[b], st));  // the set is free again
    TCM_CUDA(cudaGetLastError());
    M->launches += 6 + (u64)rs.npa + (u64)rs.npe;
    return TC_OK;
}

}  // namespace tc

// ---- tc_multi_* entry points ----------------------------------------------

// Participants of a round given as offsets into one buffer (w_s > 0 only).
static int items_from_offsets(const tc_multi *M, const u64 *d_edges, const uint64_t *offsets,
                              std::vector<RoundItem> &items) {
    if (!offsets || offsets[0] != 0) return TC_ERR_INVAL;
    for (u32 s = 0; s < M->S; ++s) {
        if (offsets[s + 1] < offsets[s]) return TC_ERR_INVAL;
        const u64 w = offsets[s + 1] - offsets[s];
        if (w) items.push_back(RoundItem{s, d_edges + offsets[s], w});
    }
    if (offsets[M->S] > M->w_max) return TC_ERR_INVAL;
    if (offsets[M->S] && !d_edges) return TC_ERR_INVAL;
    return TC_OK;
}

// Write the descriptor through the ring of pinned buffers and enqueue.
static int upload_and_enqueue(tc_multi *M, const std::vector<RoundItem> &items,
                              cudaStream_t st) {
    const u32 K = (u32)items.size();
    const int slot = M->ring;
    M->ring = (M->ring + 1) % kRing;
    TCM_CUDA(cudaEventSynchronize(M->ring_ev[slot]));
    write_descriptor(M, items.data(), K, M->h_desc[slot]);
    const int rc = copy_words_async(M, M->desc[slot], M->h_desc_dev[slot], desc_words(K), st);
    if (rc) return rc;
    TCM_CUDA(cudaEventRecord(M->ring_ev[slot], st));
    return multi_enqueue(M, items.data(), K, M->desc[slot], nullptr, nullptr, st);
}

extern "C" {

int tc_multi_create(uint32_t n_streams, const uint64_t *r, const uint64_t *seeds,
                    const uint32_t *stream_ids, uint64_t w_max_round, uint32_t vertex_bits,
                    tc_multi **out) {
    if (!out || n_streams == 0 || !r || !seeds || !stream_ids) return TC_ERR_INVAL;
    *out = nullptr;
    u64 total = 0;
    for (u32 s = 0; s < n_streams; ++s) {
        if (r[s] == 0 || r[s] > 0xFFFFFFFFull) return TC_ERR_INVAL;
        total += state_bytes(r[s]);
    }
    tc_multi *M = nullptr;
    int rc = multi_alloc(n_streams, w_max_round, vertex_bits, &M);
    if (rc) return rc;
    if (cudaMalloc(&M->state, total) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        multi_free(M);
        return e == cudaErrorMemoryAllocation ? TC_ERR_NOMEM : TC_ERR_CUDA;
    }
    unsigned char *p = reinterpret_cast<unsigned char *>(M->state);
    for (u32 s = 0; s < n_streams && rc == TC_OK; ++s) {
        rc = multi_open_slot(M, s, r[s], seeds[s], stream_ids[s], p, 0);
        p += state_bytes(r[s]);
    }
    if (rc == TC_OK && cudaDeviceSynchronize() != cudaSuccess) rc = TC_ERR_CUDA;
    if (rc) {
        multi_free(M);
        return rc;
    }
    M->launches = 0;
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

int tc_multi_set_hash_key(tc_multi *M, uint64_t key) {
    if (!M) return TC_ERR_INVAL;
    M->hash_key = key;
    return TC_OK;
}

int tc_multi_process_async(tc_multi *M, const uint64_t *d_edges, const uint64_t *offsets,
                           void *cuda_stream) {
    if (!M) return TC_ERR_INVAL;
    std::vector<RoundItem> items;
    int rc = items_from_offsets(M, d_edges, offsets, items);
    if (rc || items.empty()) return rc;
    return upload_and_enqueue(M, items, (cudaStream_t)cuda_stream);
}

// The second round scratch set, for pipelined rounds.
static int ensure_two_round_sets(tc_multi *M) {
    if (M->nsets == 2) return TC_OK;
    if (!alloc_round_set(M->rset[1], M->w_max, M->zeroed_bytes)) {
        cudaGetLastError();
        return TC_ERR_NOMEM;
    }
    M->nsets = 2;
    return TC_OK;
}

int tc_multi_process_ready_async(tc_multi *M, const uint64_t *d_edges, const uint64_t *offsets,
                                 void *cuda_stream) {
    if (!M) return TC_ERR_INVAL;
    std::vector<RoundItem> items;
    int rc = items_from_offsets(M, d_edges, offsets, items);
    if (rc || items.empty()) return rc;
    rc = ensure_two_round_sets(M);
    if (rc) return rc;
    const int slot = M->ring;
    M->ring = (M->ring + 1) % kRing;
    TCM_CUDA(cudaEventSynchronize(M->ring_ev[slot]));
    write_descriptor(M, items.data(), (u32)items.size(), M->h_desc[slot]);
    rc = multi_enqueue(M, items.data(), (u32)items.size(), M->desc[slot], M->h_desc_dev[slot],
                       nullptr, (cudaStream_t)cuda_stream, true, nullptr);
    if (rc) return rc;
    TCM_CUDA(cudaEventRecord(M->ring_ev[slot], M->sa));  // after the descriptor's upload
    return TC_OK;
}

int tc_multi_process_ptrs_async(tc_multi *M, const uint64_t *const *d_batches,
                                const uint64_t *w, void *cuda_stream) {
    if (!M || !d_batches || !w) return TC_ERR_INVAL;
    std::vector<RoundItem> items;
    u64 total = 0;
    for (u32 s = 0; s < M->S; ++s) {
        if (!w[s]) continue;
        if (!d_batches[s]) return TC_ERR_INVAL;
        total += w[s];
        items.push_back(RoundItem{s, d_batches[s], w[s]});
    }
    if (total > M->w_max) return TC_ERR_INVAL;
    if (items.empty()) return TC_OK;
    return upload_and_enqueue(M, items, (cudaStream_t)cuda_stream);
}

int tc_multi_capture(tc_multi *M, const uint64_t *d_edges, const uint64_t *offsets,
                     void *cuda_stream) {
    if (!M || !d_edges) return TC_ERR_INVAL;
    std::vector<RoundItem> items;
    int rc = items_from_offsets(M, d_edges, offsets, items);
    if (rc) return rc;
    if (items.empty()) return TC_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (M->gexec) {
        cudaGraphExecDestroy(M->gexec);
        M->gexec = nullptr;
    }
    if (!M->g_desc) TCM_CUDA(cudaMalloc(&M->g_desc, desc_words(M->S) * sizeof(u64)));
    std::vector<u64> h(desc_words((u32)items.size()));
    write_descriptor(M, items.data(), (u32)items.size(), h.data());
    TCM_CUDA(cudaMemcpy(M->g_desc, h.data(), h.size() * sizeof(u64), cudaMemcpyHostToDevice));
    TCM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const u64 before = M->launches;
    rc = multi_enqueue(M, items.data(), (u32)items.size(), M->g_desc, nullptr, nullptr, st);
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
    const int rc = clear_tags_if_due(M, M->graph_set);
    if (rc) return rc;
    M->set_rounds[M->graph_set]++;
    TCM_CUDA(cudaGraphLaunch(M->gexec, (cudaStream_t)cuda_stream));
    M->launches += M->graph_launches;
    return TC_OK;
}

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
    if (!M || !out || s >= M->S || M->h_rec[s].r == 0) return TC_ERR_INVAL;
    TCM_CUDA(cudaDeviceSynchronize());
    MStream h{};
    TCM_CUDA(cudaMemcpy(&h, M->ms + s, sizeof(MStream), cudaMemcpyDeviceToHost));
    finish_estimate(h.est[0], h.est[1], h.est[2], h.m, h.r, h.batches, out);
    return TC_OK;
}

int tc_multi_estimates_async(tc_multi *M, tc_estimate_t *d_out, void *cuda_stream) {
    if (!M || !d_out || (reinterpret_cast<uintptr_t>(d_out) & 7)) return TC_ERR_INVAL;
    mestimate_kernel<<<(M->S + 127) / 128, 128, 0, (cudaStream_t)cuda_stream>>>(M->ms, M->S,
                                                                               d_out);
    TCM_CUDA(cudaGetLastError());
    M->launches += 1;
    return TC_OK;
}

int tc_multi_get_state(tc_multi *M, uint32_t s, uint64_t *f1, uint64_t *f2, uint64_t *chi,
                       uint32_t *flags) {
    if (!M || s >= M->S || M->h_rec[s].r == 0) return TC_ERR_INVAL;
    TCM_CUDA(cudaDeviceSynchronize());
    const MStream &h = M->h_rec[s];
    const u64 n = h.r;
    if (f1) TCM_CUDA(cudaMemcpy(f1, h.f1, n * sizeof(u64), cudaMemcpyDeviceToHost));
    if (f2) TCM_CUDA(cudaMemcpy(f2, h.f2, n * sizeof(u64), cudaMemcpyDeviceToHost));
    if (chi) TCM_CUDA(cudaMemcpy(chi, h.chi, n * sizeof(u64), cudaMemcpyDeviceToHost));
    if (flags) TCM_CUDA(cudaMemcpy(flags, h.flags, n * sizeof(u32), cudaMemcpyDeviceToHost));
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
