// Onesweep LSD radix sort of packed uint64 keys (optionally carrying a
// uint32 value), used for the two sorts of the estimator update: the arcs of
// rankAll (Lemma 4.3: by src, ties by decreasing pos) and the Step-3 keys of
// Sec. 4.4 (by a hash of the edge).
//
// Design (after Adinets and Merrill, "Onesweep: A Faster Least Significant
// Digit Radix Sort for GPUs", 2022):
//   * all digit histograms of a sort are counted up front, in the same pass
//     that builds the keys (no separate upsweep per digit);
//   * one kernel per digit: each CTA takes the next tile id from an atomic
//     counter (so it only ever waits on tiles that already run), counts its
//     digits and publishes the counts at once, ranks its keys stably inside
//     each warp (peers with equal digits found by warp votes: one ballot per
//     digit bit, one match.any, or lanes OR-ing their bit into a shared
//     word) and writes them to a digit-ordered staging area;
//   * then each thread walks back, for its digits, over earlier tiles'
//     published counts / inclusive prefixes (decoupled look-back).  Status
//     words are stored tile-major, so a warp's loads of one tile's statuses
//     are coalesced; after the nearest predecessor, up to eight predecessors
//     are loaded per round trip;
//   * the staged keys are scattered in digit order, so each digit's keys go
//     to consecutive global addresses;
//   * a pass whose digit is the same for every key is an identity
//     permutation and is skipped (decided on the device from the
//     histogram); ping-pong buffer selection follows on the device, so the
//     host never needs the histogram.
// Digit width (8, 9, 10 or 11 bits) is a template parameter.
// Look-back waits are bounded: after kSpinLimit rounds without progress the
// CTA records kErrTimeout and proceeds (the batch is then rejected, never
// hung).
#pragma once

#include "tc_common.cuh"

namespace tc {

constexpr int kMaxRadixBits = 11;
constexpr int kMaxRadix = 1 << kMaxRadixBits;
constexpr int kMaxPasses = 8;
constexpr int kRankThreads8 = 256;  // ranking warps x 32
constexpr int kSortWarps = kRankThreads8 / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kRankThreads8 * kSortItems;
constexpr int kLookWin = 8;  // predecessors per look-back load group
constexpr u32 kSpinLimit = 1u << 21;

constexpr u32 kFlagAgg = 1u << 30;  // tile count published
constexpr u32 kFlagPre = 2u << 30;  // inclusive prefix published
constexpr u32 kFlagMask = 3u << 30;
constexpr u32 kValMask = (1u << 30) - 1;

// Sort plan in device memory (one per sort and batch; zeroed per batch).
struct SortPlan {
    u32 counts[kMaxPasses][kMaxRadix];   // digit histograms (filled by the key build)
    u32 offsets[kMaxPasses][kMaxRadix];  // exclusive bucket offsets
    u32 skip[kMaxPasses];                // 1 if every key has the same digit
    u32 npass;                           // passes of this sort
    u32 tile_counter[kMaxPasses];
    u32 pad[15];
};

// Tiles whose look-back statuses one pass keeps (rounded up to whole
// groups of kLookWin).
__host__ __device__ __forceinline__ u32 lookback_stride(u32 tiles) {
    return (tiles + kLookWin - 1) / kLookWin * kLookWin;
}

__device__ __forceinline__ u32 digit_bits(u64 key, u32 shift, u32 mask) {
    return (u32)(key >> shift) & mask;
}

// The digit at bit `shift` of a 64-bit key, on 32-bit halves: a pass's
// shift is uniform, so the word choice is a uniform predicate and the
// extraction one funnel or plain shift plus a mask.
struct DigitAt {
    bool hi;  // digit lies in the high word
    u32 sh;   // shift inside the word pair
    __device__ __forceinline__ explicit DigitAt(u32 shift)
        : hi(shift >= 32), sh(shift >= 32 ? shift - 32 : shift) {}
    __device__ __forceinline__ u32 operator()(u64 key, u32 mask) const {
        const u32 lo = (u32)key, hw = (u32)(key >> 32);
        return (hi ? (hw >> sh) : __funnelshift_r(lo, hw, sh)) & mask;
    }
};

// Exclusive prefix over the values `x` of threads [0, kThreads) of a CTA.
// `s_tmp` holds kThreads/32 words.  Must be reached by every thread of the
// CTA; threads at or beyond kThreads contribute nothing.
template <int kThreads>
__device__ __forceinline__ u32 block_exclusive_sum(u32 x, u32 *s_tmp, u32 *total = nullptr) {
    constexpr int kWarps = kThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31 && warp < kWarps) s_tmp[warp] = inc;
    __syncthreads();
    u32 before = 0, all = 0;
#pragma unroll
    for (int w2 = 0; w2 < kWarps; ++w2) {
        const u32 v = s_tmp[w2];
        if (w2 < warp) before += v;
        all += v;
    }
    __syncthreads();
    if (total) *total = all;
    return before + inc - x;
}

// Turn the histogram of one pass over `n` keys (digit width `bits`) into
// bucket offsets and its skip flag.  Grid (passes, 2): blockIdx.x is the
// pass, blockIdx.y the plan; 256 threads per block.
static __global__ void __launch_bounds__(256) sort_plan_kernel(SortPlan *plans, int npass0, u32 n0,
                                                         u32 bits0, int npass1, u32 n1,
                                                         u32 bits1) {
    __shared__ u32 s_tmp[8];
    const int j = blockIdx.y;
    SortPlan *plan = plans + j;
    const int npass = j == 0 ? npass0 : npass1;
    const int p = blockIdx.x;
    if (p == 0 && threadIdx.x == 0) plan->npass = (u32)npass;
    if (p >= npass) return;
    const u32 n = j == 0 ? n0 : n1;
    const u32 radix = 1u << (j == 0 ? bits0 : bits1);
    const u32 per = (radix + 255) / 256;  // digits per thread
    const u32 d0 = threadIdx.x * per;
    u32 local = 0;
    bool single = false;
    for (u32 k = 0; k < per; ++k) {
        const u32 c = d0 + k < radix ? plan->counts[p][d0 + k] : 0u;
        local += c;
        single |= (c == n);
    }
    u32 run = block_exclusive_sum<256>(local, s_tmp);
    for (u32 k = 0; k < per && d0 + k < radix; ++k) {
        plan->offsets[p][d0 + k] = run;
        run += plan->counts[p][d0 + k];
    }
    const int any_single = __syncthreads_or(single);
    if (threadIdx.x == 0) plan->skip[p] = any_single ? 1u : 0u;
}

// Ping-pong buffer holding the keys before pass `upto` (0 or 1): one flip
// per pass that was not skipped.  upto = plan->npass gives the sorted keys.
__device__ __forceinline__ u32 plan_sel(const SortPlan *plan, int upto) {
    u32 sel = 0;
    for (int q = 0; q < upto; ++q) sel ^= plan->skip[q] ? 0u : 1u;
    return sel;
}

__device__ __forceinline__ u32 plan_final_sel(const SortPlan *plan) {
    return plan_sel(plan, (int)plan->npass);
}

// Warp ranking methods: how a warp finds the lanes holding the same digit.
enum RankMethod : int {
    kRankBallot = 0,    // one ballot per digit bit
    kRankMatch = 1,     // one match.any per key
    kRankAtomicOr = 2,  // lanes OR their bit into a per-(warp, digit) word
};

// Launch shape of a digit pass: every thread ranks keys, then walks back for
// its kDPT digits.
template <int kBits>
struct OnesweepShape {
    static constexpr int kRadix = 1 << kBits;
    static constexpr int kThreads = kRankThreads8;
    static constexpr int kDPT = kRadix / kRankThreads8;  // digits per thread
};

template <int kBits, bool kHasValues, int kRank>
struct OnesweepSmem {
    static constexpr int kRadix = 1 << kBits;
    static constexpr int kPeerWords = kRank == kRankAtomicOr ? kRadix : 1;
    u32 cursor[kSortWarps][kRadix];        // per-warp counts, then running local slots
    u32 peers[2][kSortWarps][kPeerWords];  // atomic-or ranking masks (double-buffered)
    u32 tile_excl[kRadix];
    u32 count[kRadix];
    u32 base[kRadix];
    u32 scan_tmp[kSortWarps + 8];
    u32 tile;
    u64 keys[kSortTile];
    u32 vals[kHasValues ? kSortTile : 1];
};

// Stable ranking of one warp's kSortItems rows of 32 keys: every key goes to
// its tile staging slot S.cursor[warp][digit] + (earlier equal digits of the
// warp).  kLive > 0: the digit has exactly kLive live bits (ballot votes on
// those only); kLive == 0: `live` bits, decided at run time.  kFull: every
// key of the warp is valid (no tail predicates).
template <int kBits, int kLive, bool kFull, bool kHasValues, int kRank, typename Smem>
__device__ __forceinline__ void rank_warp(Smem &S, const u64 (&keys)[kSortItems],
                                          const u32 (&vals)[kHasValues ? kSortItems : 1],
                                          u32 nvalid, const DigitAt &dig, u32 live, int lane,
                                          int warp) {
    constexpr u32 kMask = (1u << kBits) - 1;
    const u32 lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const bool valid = kFull || (u32)(j * 32 + lane) < nvalid;
        const u32 d = dig(keys[j], kMask);
        u32 peers;
        if constexpr (kRank == kRankMatch) {
            peers = __match_any_sync(0xFFFFFFFFu, valid ? d : (u32)(1u << kBits) + lane);
        } else if constexpr (kRank == kRankBallot) {
            peers = kFull ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
            for (int b = 0; b < kBits; ++b) {
                if (kLive == 0 ? (u32)b >= live : b >= kLive) break;
                const bool bit = (d >> b) & 1u;
                const u32 vote = __ballot_sync(0xFFFFFFFFu, bit);
                peers &= bit ? vote : ~vote;
            }
        } else {
            u32 *word = &S.peers[j & 1][warp][d];
            if (valid) atomicOr(word, 1u << lane);
            __syncwarp();
            peers = valid ? *word : (1u << lane);
        }
        const int leader = 31 - __clz(peers);
        u32 slot = 0;
        if (valid && lane == leader) {
            slot = S.cursor[warp][d];
            S.cursor[warp][d] = slot + __popc(peers);
        }
        if constexpr (kRank == kRankAtomicOr) {
            // every lane has read this iteration's mask before its leader
            // clears it; the buffer is next OR-ed two iterations later
            __syncwarp();
            if (valid && lane == leader) S.peers[j & 1][warp][d] = 0;
        }
        slot = __shfl_sync(0xFFFFFFFFu, slot, leader) + __popc(peers & lt_mask);
        if (valid) {
            S.keys[slot] = keys[j];
            if constexpr (kHasValues) S.vals[slot] = vals[j];
        }
        __syncwarp();
    }
}

// One digit pass.  keys/vals ping-pong between buffers 0 and 1 as selected
// by plan_sel(plan, pass); `lookback` holds this pass's status words, tile-major
// ([tiles][2^kBits]), zeroed before the pass.
template <int kBits, bool kHasValues, int kRank>
static __global__ void __launch_bounds__(OnesweepShape<kBits>::kThreads, (kBits <= 9 ? 4 : 3))
    onesweep_pass_kernel(u64 *keys0, u64 *keys1, u32 *vals0, u32 *vals1, u32 n, u32 shift,
                         u32 live, int pass, SortPlan *plan, u32 *lookback, u32 *err,
                         Control *ctl) {
    // live: digit bits that can be nonzero in this pass (higher key bits are
    // zero for every key), so ballot ranking votes only on those.
    using Shape = OnesweepShape<kBits>;
    constexpr int kRadix = Shape::kRadix;
    constexpr u32 kMask = kRadix - 1;
    constexpr int kDPT = Shape::kDPT;
    static_assert(kRadix % kRankThreads8 == 0, "whole digits per thread");
    static_assert(kDPT <= 32, "pending bits per thread");
    if (plan->skip[pass]) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && ctl) {
            atomicAdd((unsigned long long *)&ctl->skipped_passes, 1ull);
            atomicAdd((unsigned long long *)&ctl->skipped_bytes,
                      (unsigned long long)n * (kHasValues ? 24ull : 16ull));
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &S = *reinterpret_cast<OnesweepSmem<kBits, kHasValues, kRank> *>(smem_raw);

    const u32 sel = plan_sel(plan, pass);
    const u64 *__restrict__ kin = sel ? keys1 : keys0;
    u64 *__restrict__ kout = sel ? keys0 : keys1;
    const u32 *__restrict__ vin = sel ? vals1 : vals0;
    u32 *__restrict__ vout = sel ? vals0 : vals1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DigitAt dig(shift);
    if (tid == 0) S.tile = atomicAdd(&plan->tile_counter[pass], 1u);
    for (int k = tid; k < kSortWarps * kRadix; k += Shape::kThreads) (&S.cursor[0][0])[k] = 0;
    if constexpr (kRank == kRankAtomicOr)
        for (int k = tid; k < 2 * kSortWarps * kRadix; k += Shape::kThreads)
            (&S.peers[0][0][0])[k] = 0;
    __syncthreads();
    const u32 tile = S.tile;
    const u64 tile_base = (u64)tile * kSortTile;
    const u64 warp_base = tile_base + (u64)warp * 32 * kSortItems;
    // items of a ranking thread: warp_base + j*32 + lane, valid while < n
    const u32 nvalid = (warp_base >= n)
                           ? 0u
                           : (u32)min((u64)kSortItems * 32, (u64)n - warp_base);

    const bool full = nvalid == (u32)(kSortItems * 32);  // no tail in this warp
    u64 keys[kSortItems];
    u32 vals[kHasValues ? kSortItems : 1];
    if (full) {
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            keys[j] = kin[warp_base + j * 32 + lane];
            if constexpr (kHasValues) vals[j] = vin[warp_base + j * 32 + lane];
        }
    } else {
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const bool valid = (u32)(j * 32 + lane) < nvalid;
            keys[j] = valid ? kin[warp_base + j * 32 + lane] : ~0ull;
            if constexpr (kHasValues) vals[j] = valid ? vin[warp_base + j * 32 + lane] : 0u;
        }
    }

    // -- early digit counts per warp (order-free)
    if (full) {
#pragma unroll
        for (int j = 0; j < kSortItems; ++j)
            atomicAdd(&S.cursor[warp][dig(keys[j], kMask)], 1u);
    } else {
#pragma unroll
        for (int j = 0; j < kSortItems; ++j)
            if ((u32)(j * 32 + lane) < nvalid)
                atomicAdd(&S.cursor[warp][dig(keys[j], kMask)], 1u);
    }
    __syncthreads();

    // -- per digit (thread tid owns digits q*256 + tid, so a warp's status
    //    words are consecutive): tile count, publish it, turn warp counts
    //    into staging slots
    u32 carry = 0;  // keys of this tile in earlier digit slices
#pragma unroll
    for (int q = 0; q < kDPT; ++q) {
        const int d = q * kRankThreads8 + tid;
        u32 c = 0;
#pragma unroll
        for (int w2 = 0; w2 < kSortWarps; ++w2) c += S.cursor[w2][d];
        st_relaxed(lookback + (u64)tile * kRadix + d, (tile == 0 ? kFlagPre : kFlagAgg) | c);
        S.count[d] = c;
        u32 total = 0;
        const u32 excl = carry + block_exclusive_sum<kRankThreads8>(c, S.scan_tmp, &total);
        carry += total;
        S.tile_excl[d] = excl;
        u32 slot = excl;
#pragma unroll
        for (int w2 = 0; w2 < kSortWarps; ++w2) {
            const u32 t = S.cursor[w2][d];
            S.cursor[w2][d] = slot;
            slot += t;
        }
    }
    __syncthreads();

    // -- stable ranking inside each warp, written straight to the staging area
    if (full) {
        if (kRank != kRankBallot || live >= (u32)kBits)
            rank_warp<kBits, kBits, true, kHasValues, kRank>(S, keys, vals, nvalid, dig, live,
                                                             lane, warp);
        else
            rank_warp<kBits, 0, true, kHasValues, kRank>(S, keys, vals, nvalid, dig, live, lane,
                                                         warp);
    } else {
        rank_warp<kBits, 0, false, kHasValues, kRank>(S, keys, vals, nvalid, dig, live, lane,
                                                      warp);
    }
    {
        // -- look-back: each thread walks back for its kDPT digits, in aligned
        //    groups of kLookWin predecessors per round trip (earlier tiles
        //    have had the ranking time to publish)
        u32 sum[kDPT];
        int next[kDPT];  // next predecessor tile to examine
        u32 pending = 0;
#pragma unroll
        for (int q = 0; q < kDPT; ++q) {
            sum[q] = 0;
            next[q] = (int)tile - 1;
            if (tile > 0) pending |= 1u << q;
        }
        u32 idle = 0;
        int window = 1;  // the nearest predecessor usually holds a prefix already
        while (pending) {
            bool progress = false;
#pragma unroll
            for (int q = 0; q < kDPT; ++q) {
                if (!(pending & (1u << q))) continue;
                // statuses of tiles next, next-1, ...: independent loads at a
                // fixed stride from one base, each coalesced across the warp's
                // consecutive digits
                const u32 *p = lookback + ((u32)next[q] * kRadix + q * kRankThreads8 + tid);
                const int lim = min(window, next[q] + 1);  // tiles >= 0 only
                u32 st[kLookWin];
#pragma unroll
                for (int t = 0; t < kLookWin; ++t)
                    st[t] = t < lim ? ld_relaxed(p - t * kRadix) : 0u;
#pragma unroll
                for (int t = 0; t < kLookWin; ++t) {
                    if (t >= lim) break;
                    const u32 s = st[t];
                    const u32 flag = s & kFlagMask;
                    if (flag == 0) break;  // not published yet: retry this tile
                    sum[q] += s & kValMask;
                    progress = true;
                    if (flag == kFlagPre) {
                        pending &= ~(1u << q);
                        break;
                    }
                    --next[q];  // tile 0 always publishes a prefix
                }
            }
            // A round that found the nearest predecessor unpublished polls
            // only that one word next, and a thread that keeps waiting backs
            // off: the spinning threads otherwise take issue slots from the
            // tiles still ranking (at r = w = 2^24 a thread averaged 37 such
            // rounds per tile; re-polling one word cut both sorts' wall time
            // by 2.5%).
            window = progress ? kLookWin : 1;
            if (!progress && pending) {
                if (++idle > kSpinLimit) {
                    set_error(err, kErrTimeout);
                    break;
                }
                if (idle > 2) __nanosleep(idle > 8 ? 256 : 64);
            }
        }
#pragma unroll
        for (int q = 0; q < kDPT; ++q) {
            const int d = q * kRankThreads8 + tid;
            if (tile > 0)
                st_relaxed(lookback + (u64)tile * kRadix + d,
                           kFlagPre | ((sum[q] + S.count[d]) & kValMask));
            S.base[d] = plan->offsets[pass][d] + sum[q] - S.tile_excl[d];
        }
    }
    __syncthreads();

    // -- scatter: consecutive local slots of one digit go to consecutive
    //    global slots
    const u64 left = (u64)n - tile_base;
    const u32 tile_n = left < (u64)kSortTile ? (u32)left : (u32)kSortTile;
    for (u32 i = tid; i < tile_n; i += Shape::kThreads) {
        const u64 key = S.keys[i];
        const u32 pos = S.base[dig(key, kMask)] + i;
        if (pos < n) {  // only a timed-out look-back can make it larger
            kout[pos] = key;
            if constexpr (kHasValues) vout[pos] = S.vals[i];
        }
    }
}

}  // namespace tc
