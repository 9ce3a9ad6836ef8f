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
//     keys per warp with 8 ballots per key (peers with equal digits), adds
//     the warp histograms up, publishes its per-digit tile count and walks
//     back over earlier tiles' published counts / inclusive prefixes
//     (decoupled look-back) to find where its keys go;
//   * keys are re-ordered by digit in shared memory first so that the scatter
//     to global memory writes runs of consecutive addresses;
//   * a pass whose digit is the same for every key is an identity
//     permutation and is skipped (decided on the device from the
//     histogram); ping-pong buffer selection follows on the device, so the
//     host never needs the histogram.
// Look-back waits are bounded: after kSpinLimit polls the CTA records
// kErrTimeout and proceeds (the batch is then rejected, never hung).
#pragma once

#include "tc_common.cuh"

namespace tc {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;  // one thread per digit in the per-digit phases
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMaxPasses = 8;
constexpr u32 kSpinLimit = 1u << 21;

constexpr u32 kFlagAgg = 1u << 30;   // tile count published
constexpr u32 kFlagPre = 2u << 30;   // inclusive prefix published
constexpr u32 kFlagMask = 3u << 30;
constexpr u32 kValMask = (1u << 30) - 1;

static_assert(kSortThreads == kRadix, "per-digit phases use one thread per digit");

// Sort plan in device memory (one per sort and batch).
struct SortPlan {
    u32 counts[kMaxPasses][kRadix];   // digit histograms (filled by the key build)
    u32 offsets[kMaxPasses][kRadix];  // exclusive bucket offsets
    u32 skip[kMaxPasses];             // 1 if every key has the same digit
    u32 sel[kMaxPasses + 1];          // ping-pong buffer holding keys before pass p
    u32 tile_counter[kMaxPasses];
    u32 pad[8];
};

__device__ __forceinline__ u32 digit_of(u64 key, u32 shift) {
    return (u32)(key >> shift) & (kRadix - 1);
}

// Exclusive prefix over the kSortThreads values `x` of a CTA.  `s_tmp` must
// hold kSortWarps words.  Must be called by all threads.
__device__ __forceinline__ u32 block_exclusive_sum(u32 x, u32 *s_tmp, u32 *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u32 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    u32 before = 0, all = 0;
#pragma unroll
    for (int w2 = 0; w2 < kSortWarps; ++w2) {
        u32 s = s_tmp[w2];
        if (w2 < warp) before += s;
        all += s;
    }
    if (total) *total = all;
    __syncthreads();
    return before + inc - x;
}

// Turn the histograms of `npass` passes over `n` keys into bucket offsets,
// skip flags and buffer selections.  One CTA of kSortThreads per plan.
__global__ void __launch_bounds__(kSortThreads) sort_plan_kernel(SortPlan *plans, int npass0,
                                                                  u32 n0, int npass1, u32 n1) {
    __shared__ u32 s_tmp[kSortWarps];
    SortPlan *plan = plans + blockIdx.x;
    const int npass = blockIdx.x == 0 ? npass0 : npass1;
    const u32 n = blockIdx.x == 0 ? n0 : n1;
    const int d = threadIdx.x;
    for (int p = 0; p < npass; ++p) {
        u32 c = plan->counts[p][d];
        plan->offsets[p][d] = block_exclusive_sum(c, s_tmp, nullptr);
        int single = __syncthreads_or(c == n);
        if (d == 0) plan->skip[p] = single ? 1u : 0u;
    }
    __syncthreads();
    if (d == 0) {
        u32 sel = 0;
        for (int p = 0; p < kMaxPasses; ++p) {
            plan->sel[p] = sel;
            if (p < npass && !plan->skip[p]) sel ^= 1u;
        }
        plan->sel[kMaxPasses] = sel;
        // passes beyond npass are never launched; make the final selection
        // readable at a fixed index
    }
}

template <bool kHasValues>
struct OnesweepSmem {
    u32 warp_hist[kSortWarps][kRadix];
    u32 tile_excl[kRadix];
    u32 base[kRadix];
    u32 scan_tmp[kSortWarps];
    u32 tile;
    u64 keys[kSortTile];
    u32 vals[kHasValues ? kSortTile : 1];
};

// One digit pass.  keys/vals ping-pong between buffers 0 and 1 as selected
// by plan->sel[pass]; `lookback` holds this pass's [tiles][kRadix] status
// words, zeroed before the pass.
template <bool kHasValues>
__global__ void __launch_bounds__(kSortThreads) onesweep_pass_kernel(
    u64 *keys0, u64 *keys1, u32 *vals0, u32 *vals1, u32 n, u32 shift, int pass,
    SortPlan *plan, u32 *lookback, u32 *err, Control *ctl) {
    if (plan->skip[pass]) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && ctl) {
            atomicAdd((unsigned long long *)&ctl->skipped_passes, 1ull);
            atomicAdd((unsigned long long *)&ctl->skipped_bytes,
                      (unsigned long long)n * (kHasValues ? 24ull : 16ull));
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &S = *reinterpret_cast<OnesweepSmem<kHasValues> *>(smem_raw);

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

    // -- warp-ballot ranking: peers = lanes holding the same digit
    const u32 lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const bool valid = warp_base + (u64)j * 32 + lane < n;
        const u32 d = digit_of(keys[j], shift);
        u32 peers = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
        for (int b = 0; b < kRadixBits; ++b) {
            const bool bit = (d >> b) & 1u;
            const u32 vote = __ballot_sync(0xFFFFFFFFu, bit);
            peers &= bit ? vote : ~vote;
        }
        u32 before = 0;
        if (valid) before = S.warp_hist[warp][d];
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) S.warp_hist[warp][d] = before + __popc(peers);
        __syncwarp();
        ranks[j] = before + __popc(peers & lt_mask);
    }
    __syncthreads();

    // -- per digit: warp-exclusive offsets and the tile count
    const int d = tid;
    u32 count = 0;
#pragma unroll
    for (int w2 = 0; w2 < kSortWarps; ++w2) {
        const u32 t = S.warp_hist[w2][d];
        S.warp_hist[w2][d] = count;
        count += t;
    }
    u32 *my_status = lookback + (u64)tile * kRadix + d;
    st_relaxed(my_status, (tile == 0 ? kFlagPre : kFlagAgg) | count);
    S.tile_excl[d] = block_exclusive_sum(count, S.scan_tmp, nullptr);

    // -- decoupled look-back over earlier tiles, one thread per digit
    u32 excl = 0;
    if (tile > 0) {
        long k = (long)tile - 1;
        u32 spins = 0;
        while (k >= 0) {
            const u32 s = ld_relaxed(lookback + (u64)k * kRadix + d);
            const u32 flag = s & kFlagMask;
            if (flag == 0) {
                if (++spins > kSpinLimit) {
                    set_error(err, kErrTimeout);
                    break;
                }
                if (spins > 32) __nanosleep(64);
                continue;
            }
            excl += s & kValMask;
            if (flag == kFlagPre) break;
            --k;
        }
        st_relaxed(my_status, kFlagPre | ((excl + count) & kValMask));
    }
    S.base[d] = plan->offsets[pass][d] + excl - S.tile_excl[d];
    __syncthreads();

    // -- stage in shared memory in digit order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const bool valid = warp_base + (u64)j * 32 + lane < n;
        if (valid) {
            const u32 dj = digit_of(keys[j], shift);
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
        const u32 pos = S.base[digit_of(key, shift)] + i;
        if (pos < n) {  // only a timed-out look-back can make it larger
            kout[pos] = key;
            if constexpr (kHasValues) vout[pos] = S.vals[i];
        }
    }
}

}  // namespace tc
