// Onesweep LSD radix sort of packed uint64 keys (optionally carrying a
// uint32 value), used for the two sorts of the estimator update: the arcs of
// rankAll (Lemma 4.3: by src, ties by decreasing pos) and the `edges` array
// of Step 3 (Sec. 4.4: by (src, dst)).
//
// Design (after Adinets and Merrill, "Onesweep: A Faster Least Significant
// Digit Radix Sort for GPUs", 2022):
//   * all digit histograms of a sort are counted up front, in the same pass
//     that builds the keys (no separate upsweep per digit);
//   * one kernel per digit: each CTA takes the next tile id from an atomic
//     counter (so it only ever waits on tiles that already run), ranks its
//     keys per warp -- peers with equal digits found by warp votes, either
//     one ballot per digit bit or one match.any -- adds the warp histograms
//     up, publishes its per-digit tile counts and walks back over earlier
//     tiles' published counts / inclusive prefixes (decoupled look-back);
//   * keys are re-ordered by digit in shared memory first so that the scatter
//     to global memory writes runs of consecutive addresses;
//   * a pass whose digit is the same for every key is an identity
//     permutation and is skipped (decided on the device from the
//     histogram); ping-pong buffer selection follows on the device, so the
//     host never needs the histogram.
// Digit width (8, 10 or 11 bits) is a template parameter; the host picks the
// width that needs the fewest passes over the live key bits.
// Look-back waits are bounded: after kSpinLimit polls the CTA records
// kErrTimeout and proceeds (the batch is then rejected, never hung).
#pragma once

#include "tc_common.cuh"

namespace tc {

constexpr int kMaxRadixBits = 11;
constexpr int kMaxRadix = 1 << kMaxRadixBits;
constexpr int kMaxPasses = 8;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
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
    u32 sel[kMaxPasses + 1];             // ping-pong buffer holding keys before pass p
    u32 tile_counter[kMaxPasses];
    u32 pad[7];
};

__device__ __forceinline__ u32 digit_bits(u64 key, u32 shift, u32 mask) {
    return (u32)(key >> shift) & mask;
}

// Exclusive prefix over the values `x` of the kThreads threads of a CTA.
// `s_tmp` holds kThreads/32 words.  Must be called by all threads.
template <int kThreads>
__device__ __forceinline__ u32 block_exclusive_sum(u32 x, u32 *s_tmp) {
    constexpr int kWarps = kThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    u32 before = 0;
#pragma unroll
    for (int w2 = 0; w2 < kWarps; ++w2)
        if (w2 < warp) before += s_tmp[w2];
    __syncthreads();
    return before + inc - x;
}

// Turn the histograms of `npass` passes over `n` keys (digit width `bits`)
// into bucket offsets, skip flags and buffer selections.  One CTA of
// kSortThreads per plan; blockIdx.x selects the plan.
__global__ void __launch_bounds__(kSortThreads) sort_plan_kernel(SortPlan *plans, int npass0,
                                                                  u32 n0, u32 bits0, int npass1,
                                                                  u32 n1, u32 bits1) {
    __shared__ u32 s_tmp[kSortWarps];
    SortPlan *plan = plans + blockIdx.x;
    const int npass = blockIdx.x == 0 ? npass0 : npass1;
    const u32 n = blockIdx.x == 0 ? n0 : n1;
    const u32 radix = 1u << (blockIdx.x == 0 ? bits0 : bits1);
    const u32 per = (radix + kSortThreads - 1) / kSortThreads;  // digits per thread
    const u32 d0 = threadIdx.x * per;
    for (int p = 0; p < npass; ++p) {
        u32 local = 0;
        bool single = false;
        for (u32 k = 0; k < per; ++k) {
            const u32 c = d0 + k < radix ? plan->counts[p][d0 + k] : 0u;
            local += c;
            single |= (c == n);
        }
        u32 run = block_exclusive_sum<kSortThreads>(local, s_tmp);
        for (u32 k = 0; k < per && d0 + k < radix; ++k) {
            plan->offsets[p][d0 + k] = run;
            run += plan->counts[p][d0 + k];
        }
        const int any_single = __syncthreads_or(single);
        if (threadIdx.x == 0) plan->skip[p] = any_single ? 1u : 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 sel = 0;
        for (int p = 0; p < kMaxPasses; ++p) {
            plan->sel[p] = sel;
            if (p < npass && !plan->skip[p]) sel ^= 1u;
        }
        plan->sel[kMaxPasses] = sel;  // where the sorted keys end up
    }
}

template <int kBits, bool kHasValues>
struct OnesweepSmem {
    static constexpr int kRadix = 1 << kBits;
    u32 warp_hist[kSortWarps][kRadix];
    u32 tile_excl[kRadix];
    u32 base[kRadix];
    u32 scan_tmp[kSortWarps];
    u32 tile;
    u64 keys[kSortTile];
    u32 vals[kHasValues ? kSortTile : 1];
};

// One digit pass.  keys/vals ping-pong between buffers 0 and 1 as selected
// by plan->sel[pass]; `lookback` holds this pass's [tiles][2^kBits] status
// words, zeroed before the pass.  kMatch: peers found with one match.any
// per key; otherwise with one ballot per digit bit.
template <int kBits, bool kHasValues, bool kMatch>
__global__ void __launch_bounds__(kSortThreads, (kBits <= 10 ? 3 : 2)) onesweep_pass_kernel(
    u64 *keys0, u64 *keys1, u32 *vals0, u32 *vals1, u32 n, u32 shift, int pass,
    SortPlan *plan, u32 *lookback, u32 *err, Control *ctl) {
    constexpr int kRadix = 1 << kBits;
    constexpr u32 kMask = kRadix - 1;
    constexpr int kDPT = (kRadix + kSortThreads - 1) / kSortThreads;  // digits per thread
    if (plan->skip[pass]) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && ctl) {
            atomicAdd((unsigned long long *)&ctl->skipped_passes, 1ull);
            atomicAdd((unsigned long long *)&ctl->skipped_bytes,
                      (unsigned long long)n * (kHasValues ? 24ull : 16ull));
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &S = *reinterpret_cast<OnesweepSmem<kBits, kHasValues> *>(smem_raw);

    const u32 sel = plan->sel[pass];
    const u64 *__restrict__ kin = sel ? keys1 : keys0;
    u64 *__restrict__ kout = sel ? keys0 : keys1;
    const u32 *__restrict__ vin = sel ? vals1 : vals0;
    u32 *__restrict__ vout = sel ? vals0 : vals1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) S.tile = atomicAdd(&plan->tile_counter[pass], 1u);
    for (int k = tid; k < kSortWarps * kRadix; k += kSortThreads) (&S.warp_hist[0][0])[k] = 0;
    __syncthreads();
    const u32 tile = S.tile;
    const u64 tile_base = (u64)tile * kSortTile;
    const u64 warp_base = tile_base + (u64)warp * 32 * kSortItems;

    u64 keys[kSortItems];
    u32 vals[kHasValues ? kSortItems : 1];
    u32 ranks[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const u64 idx = warp_base + (u64)j * 32 + lane;
        keys[j] = idx < n ? kin[idx] : ~0ull;
        if constexpr (kHasValues) vals[j] = idx < n ? vin[idx] : 0u;
    }

    // -- warp-level ranking: peers = lanes of this warp holding the same digit
    const u32 lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const bool valid = warp_base + (u64)j * 32 + lane < n;
        const u32 d = digit_bits(keys[j], shift, kMask);
        u32 peers;
        if constexpr (kMatch) {
            peers = __match_any_sync(0xFFFFFFFFu, valid ? d : (u32)kRadix + lane);
        } else {
            peers = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
            for (int b = 0; b < kBits; ++b) {
                const bool bit = (d >> b) & 1u;
                const u32 vote = __ballot_sync(0xFFFFFFFFu, bit);
                peers &= bit ? vote : ~vote;
            }
        }
        const int leader = 31 - __clz(peers);
        u32 before = 0;
        if (valid && lane == leader) {
            before = S.warp_hist[warp][d];
            S.warp_hist[warp][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xFFFFFFFFu, before, leader);
        ranks[j] = before + __popc(peers & lt_mask);
        __syncwarp();
    }
    __syncthreads();

    // -- per digit: warp-exclusive offsets and the tile count; publish counts
    static_assert(kRadix % kSortThreads == 0, "whole digits per thread");
    u32 count[kDPT];
    u32 local = 0;
#pragma unroll
    for (int q = 0; q < kDPT; ++q) {
        const int d = tid * kDPT + q;
        u32 c = 0;
#pragma unroll
        for (int w2 = 0; w2 < kSortWarps; ++w2) {
            const u32 t = S.warp_hist[w2][d];
            S.warp_hist[w2][d] = c;
            c += t;
        }
        st_relaxed(lookback + (u64)tile * kRadix + d, (tile == 0 ? kFlagPre : kFlagAgg) | c);
        count[q] = c;
        local += c;
    }
    u32 run = block_exclusive_sum<kSortThreads>(local, S.scan_tmp);

    // -- decoupled look-back over earlier tiles; the thread's digits walk back
    //    in lockstep so their status loads overlap
    u32 excl[kDPT];
    if (tile > 0) {
        long k[kDPT];
        u32 pending = 0;
#pragma unroll
        for (int q = 0; q < kDPT; ++q) {
            excl[q] = 0;
            k[q] = (long)tile - 1;
            pending |= 1u << q;
        }
        u32 spins = 0;
        while (pending) {
            bool waited = false;
#pragma unroll
            for (int q = 0; q < kDPT; ++q) {
                if (!(pending & (1u << q))) continue;
                const u32 s = ld_relaxed(lookback + (u64)k[q] * kRadix + tid * kDPT + q);
                const u32 flag = s & kFlagMask;
                if (flag == 0) {
                    waited = true;
                    continue;
                }
                excl[q] += s & kValMask;
                if (flag == kFlagPre) pending &= ~(1u << q);
                else --k[q];  // tile 0 always publishes a prefix, so k stays >= 0
            }
            if (waited && pending) {
                if (++spins > kSpinLimit) {
                    set_error(err, kErrTimeout);
                    break;
                }
                if (spins > 32) __nanosleep(64);
            }
        }
#pragma unroll
        for (int q = 0; q < kDPT; ++q)
            st_relaxed(lookback + (u64)tile * kRadix + tid * kDPT + q,
                       kFlagPre | ((excl[q] + count[q]) & kValMask));
    } else {
#pragma unroll
        for (int q = 0; q < kDPT; ++q) excl[q] = 0;
    }
#pragma unroll
    for (int q = 0; q < kDPT; ++q) {
        const int d = tid * kDPT + q;
        S.tile_excl[d] = run;
        S.base[d] = plan->offsets[pass][d] + excl[q] - run;
        run += count[q];
    }
    __syncthreads();

    // -- stage in shared memory in digit order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const bool valid = warp_base + (u64)j * 32 + lane < n;
        if (valid) {
            const u32 dj = digit_bits(keys[j], shift, kMask);
            const u32 lp = S.tile_excl[dj] + S.warp_hist[warp][dj] + ranks[j];
            S.keys[lp] = keys[j];
            if constexpr (kHasValues) S.vals[lp] = vals[j];
        }
    }
    __syncthreads();

    // -- scatter: consecutive local slots of one digit go to consecutive
    //    global slots
    const u64 left = (u64)n - tile_base;
    const u32 tile_n = left < (u64)kSortTile ? (u32)left : (u32)kSortTile;
    for (u32 i = tid; i < tile_n; i += kSortThreads) {
        const u64 key = S.keys[i];
        const u32 pos = S.base[digit_bits(key, shift, kMask)] + i;
        if (pos < n) {  // only a timed-out look-back can make it larger
            kout[pos] = key;
            if constexpr (kHasValues) vout[pos] = S.vals[i];
        }
    }
}

}  // namespace tc
