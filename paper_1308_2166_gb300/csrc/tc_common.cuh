// Shared device helpers for the streaming triangle-count kernels.
#pragma once

#include <cstdint>
#include <cmath>
#include <cuda_runtime.h>

#include "tc.h"

namespace tc {

using u32 = uint32_t;
using u64 = uint64_t;

constexpr u64 kEmpty = TC_EMPTY_EDGE;
constexpr u32 kMask32 = 0xFFFFFFFFu;

// Device-side error bits (the first nonzero code wins, see set_error).
enum : u32 {
    kErrNone = 0,
    kErrInput = 1,    // batch breaks the stream model
    kErrTimeout = 2,  // a bounded spin wait gave up
};

// Per-context control block in device memory.  `err` is cleared at the start
// of every batch; `sticky` keeps the first error of any batch until the host
// reads it.
struct Control {
    u64 m;        // |E|: edges folded in so far
    u64 batches;  // batch counter b (part of the Philox counter)
    u32 err;      // error of the batch in flight
    u32 sticky;   // first error since the host last looked
    u64 skipped_passes;  // sort digit passes that found a single digit value
    u64 skipped_bytes;   // their algorithmic bytes (not moved)
    u32 epoch;           // batches enqueued (accepted or not); tags directory entries
    u32 pad;
    // Lemma 3.1 aggregate of the state after the last accepted batch:
    // S (128-bit), closed count, |E|.
    u64 est[4];
};

// Per-batch accumulator at the head of the zeroed scratch: the sweep adds
// each estimator's final chi (if closed) into it; the batch's finish step
// commits it to Control::est when the batch is accepted.
struct BatchAcc {
    u64 s_lo, s_hi, closed;
    u64 pad[29];  // keeps what follows 256-byte aligned
};

// Per-vertex segment directory entry: the run [start, end) of vertex x in a
// sorted array, valid only when `epoch` equals the batch's epoch (entries of
// earlier batches are stale without being cleared).
struct __align__(16) DirEntry {
    u32 epoch;
    u32 start;
    u32 end;
    u32 pad;
};

__device__ __forceinline__ void set_error(u32 *err, u32 code) {
    atomicCAS(err, 0u, code);
}

// Relaxed loads/stores at GPU scope: bypass L1 so that flags written by other
// CTAs of the same kernel become visible.
__device__ __forceinline__ u32 ld_relaxed(const u32 *p) {
    u32 v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(u32 *p, u32 v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// First index i in [0, n) with a[i] >= key (n if none).  The loop count
// depends only on n, so a warp's lanes stay converged.
__device__ __forceinline__ u64 lower_bound_u64(const u64 *__restrict__ a, u64 n, u64 key) {
    const u64 *base = a;
    u64 len = n;
    while (len > 1) {
        u64 half = len >> 1;
        base = (__ldg(base + half - 1) < key) ? base + half : base;
        len -= half;
    }
    return (u64)(base - a) + ((len == 1 && __ldg(base) < key) ? 1 : 0);
}

// Same, restricted to [lo, hi).
__device__ __forceinline__ u64 lower_bound_range(const u64 *__restrict__ a, u64 lo, u64 hi,
                                                 u64 key) {
    return lo + lower_bound_u64(a + lo, hi - lo, key);
}

// ---------------------------------------------------------------------------
// Lemma 3.1's estimate from the committed sums, shared by host and device so
// that every entry point returns the same record bit for bit: N = m * S
// exactly in 128 bits, tau_hat = q + rem / r with q = N div r (q converted
// to double with round-to-nearest-even, rem / r one correctly rounded
// division of two exact doubles, then one rounded addition).
// ---------------------------------------------------------------------------
using u128 = unsigned __int128;

__host__ __device__ __forceinline__ double u64_to_double_rn(u64 x) {
#ifdef __CUDA_ARCH__
    return __ull2double_rn(x);
#else
    return (double)x;  // correctly rounded under the default rounding mode
#endif
}

// Round-to-nearest-even conversion of a 128-bit unsigned integer: the top 64
// significant bits are converted with the bits shifted out below them folded
// into bit 0 as a sticky bit (bit 0 lies below the rounding point, so it can
// only break an exact tie, as those bits do).
__host__ __device__ __forceinline__ double u128_to_double_rn(u128 x) {
    const u64 hi = (u64)(x >> 64), lo = (u64)x;
    if (hi == 0) return u64_to_double_rn(lo);
#ifdef __CUDA_ARCH__
    const int s = __clzll((long long)hi);
#else
    const int s = __builtin_clzll(hi);
#endif
    const u64 top = s ? (hi << s) | (lo >> (64 - s)) : hi;
    const u64 below = s ? lo << s : lo;
    const double t = u64_to_double_rn(top | (below != 0 ? 1ull : 0ull));
    return ldexp(t, 64 - s);  // exact: a power-of-two scaling in range
}

__host__ __device__ __forceinline__ void finish_estimate(u64 s_lo, u64 s_hi, u64 closed, u64 m,
                                                         u64 r, u64 batches,
                                                         tc_estimate_t *out) {
    const u128 S = ((u128)s_hi << 64) | s_lo;
    const u128 N = S * (u128)m;
    out->num_lo = (u64)N;
    out->num_hi = (u64)(N >> 64);
    out->r = r;
    out->m = m;
    out->n_closed = closed;
    const u128 q = N / r;
    const u64 rem = (u64)(N % r);
    out->tau_hat = u128_to_double_rn(q) + (double)rem / (double)r;
    out->sum_lo = s_lo;
    out->sum_hi = s_hi;
    out->batches = batches;
}

// A fresh random key for the Step-3 edge hash (host; defined in tc_api.cu).
u64 random_hash_key();

__host__ __device__ __forceinline__ u32 bits_for(u64 x) {
    // number of bits needed to hold values 0..x (at least 1)
    u32 b = 1;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

}  // namespace tc
