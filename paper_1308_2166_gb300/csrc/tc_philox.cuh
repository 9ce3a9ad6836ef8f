// Philox4x32-10 and the bounded draws of the estimator update (device side).
//
// Philox4x32-10 is written from Salmon, Moraes, Dror, Shaw, "Parallel Random
// Numbers: As Easy as 1, 2, 3" (SC'11, Sec. 3): each round multiplies words
// 0 and 2 by the two Philox multipliers, swaps and xors the high halves with
// the round key; the key advances by the two Weyl constants between rounds.
//
// Draw conventions (the triangle-counting paper leaves its randInt open,
// Sec. 4.2 and Sec. 4.3):
//   counter = (estimator i, batch b, stream id, slot), key = (seed lo, seed hi);
//   one call yields two 64-bit words (x0 | x1 << 32) and (x2 | x3 << 32);
//   Step 1 uses slots 0, 2, 4, ..., Step 2 slots 1, 3, 5, ...; a rejected
//   word is replaced by the next word of the same step;
//   U(n) is Lemire's nearly-divisionless bounded draw (ACM TOMACS 2019):
//   the high half of word * n, rejecting words whose low half is below
//   (2^64 - n) mod n.
#pragma once

#include "tc_common.cuh"

namespace tc {

constexpr u32 kPhiloxM0 = 0xD2511F53u;
constexpr u32 kPhiloxM1 = 0xCD9E8D57u;
constexpr u32 kPhiloxW0 = 0x9E3779B9u;
constexpr u32 kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k.x += kPhiloxW0;
            k.y += kPhiloxW1;
        }
        const u32 lo0 = kPhiloxM0 * c.x;
        const u32 hi0 = __umulhi(kPhiloxM0, c.x);
        const u32 lo1 = kPhiloxM1 * c.z;
        const u32 hi1 = __umulhi(kPhiloxM1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Which estimator-update step a draw belongs to.
enum : u32 { kStep1 = 0, kStep2 = 1 };

struct DrawKey {
    uint2 key;   // (seed lo, seed hi)
    u32 batch;   // b
    u32 stream;  // stream id
};

// U(n) for estimator i, n >= 1.
__device__ __forceinline__ u64 draw_bounded(const DrawKey &dk, u32 i, u32 purpose, u64 n) {
    u32 slot = purpose;
    uint4 x = philox4x32_10(make_uint4(i, dk.batch, dk.stream, slot), dk.key);
    u64 word = (u64)x.x | ((u64)x.y << 32);
    u64 low = word * n;
    if (low < n) {
        const u64 threshold = (0ull - n) % n;
        bool second_half = false;
        while (low < threshold) {
            if (!second_half) {
                word = (u64)x.z | ((u64)x.w << 32);
                second_half = true;
            } else {
                slot += 2;
                x = philox4x32_10(make_uint4(i, dk.batch, dk.stream, slot), dk.key);
                word = (u64)x.x | ((u64)x.y << 32);
                second_half = false;
            }
            low = word * n;
        }
    }
    return __umul64hi(word, n);
}

}  // namespace tc
