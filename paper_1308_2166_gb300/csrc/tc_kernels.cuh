// Kernels of one batch update (bulkUpdateAll, Sec. 4 of Tangwongsan, Pavan,
// Tirthapura, "Parallel Triangle Counting in Massive Streaming Graphs").
//
// Data layout in HBM (per stream context):
//   estimator state, structure of arrays over i = 0..r-1:
//     f1[i], f2[i]  uint64 packed edges (min << 32) | max, kEmpty if empty
//     chi[i]        uint64 |Gamma(f1)|
//     flags[i]      uint32, bit 0 = closed (f3 present)
//   per-batch scratch:
//     arcs[2][2w]   uint64 arc keys  src << (bw+1) | (w-1-pos) << 1 | side
//                   (side 0: src is the smaller endpoint).  Written in
//                   decreasing pos order and sorted stably on the src bits
//                   only, which yields Lemma 4.3's order (src asc, pos desc)
//                   and makes the arc's rank its offset in the src segment.
//     ekeys[2][w]   uint64 Step-3 keys  h(u, v) << bw | pos, h the 32-bit mix
//                   of the packed edge (edge_hash), sorted on the top hs bits
//                   of h only (hs >= hb: whole digits covering the bucket
//                   bits): every edge lies in its hash bucket, in the run of
//                   keys sharing its top hs bits, and so does a repeat.
//     adir          per-vertex directory over the sorted arcs (vertex ids
//                   < 2^kDirMaxBits), epoch-tagged, for batches with
//                   2^B > 8w; otherwise
//     aoff, pdir    the dense CSR offsets of the sorted arcs (2^B + 1 u32)
//                   and the same packed 12 vertices to 16 bytes;
//     bdir          dense directory of the 2^hb hash buckets (top hb bits of
//                   h) over the sorted Step-3 keys: {first index, filter mask}.
//   bw = bits of w-1, B = vertex id bits, hb = bucket bits (about w/4
//   buckets), she = bw + 32 - hs the first sorted bit of a Step-3 key.
#pragma once

#include "tc_common.cuh"
#include "tc_onesweep.cuh"
#include "tc_philox.cuh"

namespace tc {

// Host-computed shape of one batch.
struct BatchShape {
    u32 w;          // batch size
    u32 bw;         // bits of w-1
    u32 B;          // vertex id bits
    u32 sha;        // arc key: src shift = bw + 1
    u32 hb;         // Step-3 hash bucket bits
    u32 hs;         // Step-3 hash bits sorted (top of h, hb <= hs <= 32)
    u32 she;        // Step-3 key: first sorted bit, bw + 32 - hs
    int npa;        // arc sort passes
    int npe;        // edge sort passes
    u32 bits_a;     // arc sort digit width
    u32 bits_e;     // edge sort digit width
    u64 hkey;       // key of the Step-3 edge hash
};

// 32-bit keyed mix of a packed edge (u << 32) | v for the Step-3 keys: the
// edge xor a 64-bit key, through the finaliser of Steele, Lea and Flood's
// SplitMix64 (OOPSLA 2014, constants as published by Vigna), high half.
// Any key gives the same lookup results -- a lookup verifies the edge
// itself -- and a key drawn at random per context keeps the buckets even
// whatever the batch: a batch crafted to pile its edges into a few runs of
// equal sorted bits (which the repeat check and the lookups scan) would have
// to know the key.
__host__ __device__ __forceinline__ u32 edge_hash(u64 x, u64 key) {
    x ^= key;
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return (u32)(x >> 32);
}

// ---------------------------------------------------------------------------
// Key build + all digit histograms (one pass over the batch).
// Validates the stream model (Sec. 2): u < v and v < 2^B.
// Dynamic shared memory: npa << bits_a arc counters, then npe << bits_e edge
// counters.
// ---------------------------------------------------------------------------
constexpr int kPrepThreads = 256;
constexpr int kPrepItems = 4;  // edges per thread whose loads are issued together

static __global__ void __launch_bounds__(kPrepThreads) prep_kernel(
    const u64 *__restrict__ W, BatchShape s, u64 *__restrict__ arcs0, u64 *__restrict__ ekeys0,
    SortPlan *plans, u32 *err, int build_edges) {
    extern __shared__ u32 h[];
    const u32 ra = 1u << s.bits_a, re = 1u << s.bits_e;
    const u32 ma = ra - 1, me = re - 1;
    const u32 na = (u32)s.npa * ra;
    const u32 nh = na + (build_edges ? (u32)s.npe * re : 0u);
    u32 *he = h + na;
    for (u32 k = threadIdx.x; k < nh; k += kPrepThreads) h[k] = 0;
    __syncthreads();
    const u64 id_lim = (s.B >= 32) ? (1ull << 32) : (1ull << s.B);
    const u32 wm1 = s.w - 1;
    bool bad = false;
    const u64 stride = (u64)gridDim.x * kPrepThreads;
    for (u64 j0 = (u64)blockIdx.x * kPrepThreads + threadIdx.x; j0 < s.w;
         j0 += kPrepItems * stride) {
        // the group's loads first, all in flight together
        u64 eg[kPrepItems];
#pragma unroll
        for (int t = 0; t < kPrepItems; ++t) {
            const u64 j = j0 + t * stride;
            eg[t] = j < s.w ? W[j] : 0ull;
        }
#pragma unroll
        for (int t = 0; t < kPrepItems; ++t) {
            const u64 j = j0 + t * stride;
            if (j >= s.w) break;
            const u64 e = eg[t];
            const u64 u = e >> 32, v = e & kMask32;
            bad |= !(u < v) || v >= id_lim;
            const u64 rpos = (u64)(wm1 - (u32)j) << 1;
            const u64 au = (u << s.sha) | rpos;
            const u64 av = (v << s.sha) | rpos | 1ull;
            reinterpret_cast<ulonglong2 *>(arcs0)[wm1 - (u32)j] = make_ulonglong2(au, av);
            for (int p = 0; p < s.npa; ++p) {
                atomicAdd(&h[p * ra + digit_bits(au, s.sha + p * s.bits_a, ma)], 1u);
                atomicAdd(&h[p * ra + digit_bits(av, s.sha + p * s.bits_a, ma)], 1u);
            }
            if (build_edges) {
                const u64 ek = ((u64)edge_hash(e, s.hkey) << s.bw) | j;
                ekeys0[j] = ek;
                for (int p = 0; p < s.npe; ++p)
                    atomicAdd(&he[p * re + digit_bits(ek, s.she + p * s.bits_e, me)], 1u);
            }
        }
    }
    if (bad) set_error(err, kErrInput);
    __syncthreads();
    for (u32 k = threadIdx.x; k < nh; k += kPrepThreads) {
        const u32 c = h[k];
        if (!c) continue;
        if (k < na) atomicAdd(&plans[0].counts[k / ra][k % ra], c);
        else atomicAdd(&plans[1].counts[(k - na) / re][(k - na) % re], c);
    }
}

constexpr u32 kDirMaxBits = 26;

// Segment [start, end) of src x in the sorted arcs, by binary search.
__device__ __forceinline__ void arc_segment(const u64 *arcs, u64 n, u32 sha, u64 x, u64 &start,
                                            u64 &end) {
    start = lower_bound_u64(arcs, n, x << sha);
    const u64 next = (x + 1) << sha;
    end = (next == 0) ? n : lower_bound_range(arcs, start, n, next);
}

// Segment [start, end) of vertex x from a directory (empty if x is absent).
// The entry is clamped to start <= end <= n, so that a directory built over
// an array that is not sorted (only possible after a rejected batch, whose
// sweep does not run) could never send a search outside the array.
__device__ __forceinline__ void dir_segment(const DirEntry *dir, u32 epoch, u64 x, u64 n,
                                            u64 &start, u64 &end) {
    const uint4 e = __ldg(reinterpret_cast<const uint4 *>(dir + x));
    const bool hit = e.x == epoch;
    const u64 s0 = hit ? e.y : 0, e0 = hit ? e.z : 0;
    end = e0 < n ? e0 : n;
    start = s0 < end ? s0 : end;
}

// The same with 32-bit bounds (n < 2^32).
__device__ __forceinline__ void dir_segment32(const DirEntry *dir, u32 epoch, u64 x, u32 n,
                                              u32 &start, u32 &end) {
    const uint4 e = __ldg(reinterpret_cast<const uint4 *>(dir + x));
    const bool hit = e.x == epoch;
    end = hit ? min(e.z, n) : 0u;
    start = hit ? min(e.y, end) : 0u;
}

// lower_bound_range with 32-bit indices (loop count depends only on the
// range length, so a warp's lanes stay converged).
__device__ __forceinline__ u32 lower_bound_idx32(const u64 *__restrict__ a, u32 lo, u32 hi,
                                                 u64 key) {
    const u64 *base = a + lo;
    u32 len = hi - lo;
    while (len > 1) {
        const u32 half = len >> 1;
        base = (__ldg(base + half - 1) < key) ? base + half : base;
        len -= half;
    }
    return (u32)(base - a) + ((len == 1 && __ldg(base) < key) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Tagged arc directory (batches with 2^B > 8w, vertex ids below 2^kDirMaxBits):
// per vertex x = src, the first arc of its run writes (epoch, start) and the
// last one writes end; entries of other vertices keep an older epoch and read
// as empty.  A block stages tiles of kIdxTile sorted keys (plus one key either
// side) in shared memory with coalesced loads, then each thread examines
// kIdxItems keys of the tile at a stride of the block.  (The Step-3 bucket
// directory and the repeat check are step3_index_kernel's.)
// ---------------------------------------------------------------------------
constexpr int kIdxThreads = 256;
constexpr int kIdxItems = 8;
constexpr int kIdxTile = kIdxThreads * kIdxItems;

static __global__ void __launch_bounds__(kIdxThreads) index_kernel(const u64 *keys0,
                                                                  const u64 *keys1,
                                                                  const SortPlan *plan,
                                                                  BatchShape s, DirEntry *dir,
                                                                  u32 epoch) {
    __shared__ u64 st[kIdxTile + 2];  // st[1 + i] = key t0 + i; st[0], st[kIdxTile + 1]: halo
    const u64 *__restrict__ K = plan_final_sel(plan) ? keys1 : keys0;
    const u64 n = 2ull * s.w;
    const u64 nverts = 1ull << s.B;
    const u32 sh = s.sha;  // key -> src
    const int tid = threadIdx.x;
    for (u64 t0 = (u64)blockIdx.x * kIdxTile; t0 < n; t0 += (u64)gridDim.x * kIdxTile) {
#pragma unroll
        for (int j = 0; j < kIdxItems; ++j) {
            const u64 k = t0 + (u64)(j * kIdxThreads + tid);
            st[1 + j * kIdxThreads + tid] = k < n ? __ldg(K + k) : 0ull;
        }
        if (tid == 0) st[0] = t0 ? __ldg(K + t0 - 1) : 0ull;
        if (tid == 1) st[kIdxTile + 1] = t0 + kIdxTile < n ? __ldg(K + t0 + kIdxTile) : 0ull;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kIdxItems; ++j) {
            const int i = j * kIdxThreads + tid;
            const u64 k = t0 + (u64)i;
            if (k >= n) break;
            const u64 x = st[1 + i] >> sh;
            const u64 prev = k ? st[i] >> sh : ~0ull;
            const u64 next = k + 1 < n ? st[i + 2] >> sh : ~0ull;
            if (x >= nverts) continue;  // invalid batch (already flagged by the key build)
            if (x != prev) *reinterpret_cast<u64 *>(&dir[x].epoch) = (k << 32) | epoch;
            if (x != next) dir[x].end = (u32)(k + 1);
        }
        __syncthreads();  // the tile is restaged next
    }
}

// ---------------------------------------------------------------------------
// Dense arc directory (CSR offsets): off[x] = the first index of the sorted
// arcs whose src is >= x, for x in [0, 2^B], so that vertex x's arcs are
// [off[x], off[x+1]) and deg_W(x) = off[x+1] - off[x] (Def. 4.2).  Every
// entry is written every batch, so nothing is tagged or cleared: sorted key
// k writes the entries of the vertices in (src(k-1), src(k)], and the entries
// past the largest src get 2w.  4 bytes per vertex id, written whole: used
// when 2^B <= 8w (the write then costs at most what one arc pass moves).
// A run of more than 32 absent vertices is filled by the whole warp.
// ---------------------------------------------------------------------------
// A block stages tiles of kIdxTile sorted keys (plus the key before the
// tile) in shared memory with coalesced loads, as index_kernel does.  The
// tile owns the vertices (src of the key before it, src of its last key];
// the entries past the largest src are written by every thread of the grid
// before the tiles (they all get 2w).  When the tile's span fits a shared
// array of kOffSpan entries, each run head marks its vertex with its index,
// a block-wide suffix minimum carries every mark down over the absent
// vertices below it, and the span is written with coalesced stores.  A
// wider span (sparse ids) is filled warp by warp instead: each warp owns the
// vertices below its 32 keys and fills them 32 at a time, lane l finding by
// a five-step shuffle search how many of the warp's keys have src < v.
constexpr u32 kOffSpan = 8192;
constexpr u32 kOffNone = 0xFFFFFFFFu;

__device__ __forceinline__ u32 block_suffix_min(u32 x, u32 *s_tmp) {
    // exclusive suffix minimum over threads (thread t gets min of t+1 .. end)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_down_sync(0xFFFFFFFFu, inc, o);
        if (lane + o < 32) inc = min(inc, t);
    }
    if (lane == 0) s_tmp[warp] = inc;
    __syncthreads();
    u32 after = kOffNone;
    for (int w2 = warp + 1; w2 < kIdxThreads / 32; ++w2) after = min(after, s_tmp[w2]);
    __syncthreads();
    const u32 next_lane = __shfl_down_sync(0xFFFFFFFFu, inc, 1);
    return lane < 31 ? min(after, next_lane) : after;
}

static __global__ void __launch_bounds__(kIdxThreads) offsets_kernel(const u64 *keys0,
                                                                    const u64 *keys1,
                                                                    const SortPlan *plan,
                                                                    BatchShape s, u32 *off) {
    __shared__ u32 st[kIdxTile + 1];  // st[1 + i] = src of key t0 + i; st[0]: the key before
    __shared__ u32 mark[kOffSpan];
    __shared__ u32 s_tmp[kIdxThreads / 32];
    const u64 *__restrict__ K = plan_final_sel(plan) ? keys1 : keys0;
    const u64 n = 2ull * s.w;
    const u32 nv = 1u << s.B;  // B <= kDirMaxBits here
    const int tid = threadIdx.x, lane = tid & 31;
    {
        const u64 xg = __ldg(K + n - 1) >> s.sha;  // the largest src
        const u64 stride = (u64)gridDim.x * kIdxThreads;
        for (u64 v = xg + 1 + (u64)blockIdx.x * kIdxThreads + tid; v <= nv; v += stride)
            off[v] = (u32)n;
    }
    for (u64 t0 = (u64)blockIdx.x * kIdxTile; t0 < n; t0 += (u64)gridDim.x * kIdxTile) {
#pragma unroll
        for (int j = 0; j < kIdxItems; ++j) {
            const u64 k = t0 + (u64)(j * kIdxThreads + tid);
            st[1 + j * kIdxThreads + tid] = k < n ? (u32)(__ldg(K + k) >> s.sha) : kOffNone;
        }
        if (tid == 0) st[0] = t0 ? (u32)(__ldg(K + t0 - 1) >> s.sha) : 0u;
        __syncthreads();
        const u32 cnt = (u32)min((u64)kIdxTile, n - t0);
        const u32 x_last = st[cnt];
        const u32 vlo = t0 ? st[0] + 1 : 0u;
        const u32 vhi = x_last < nv ? x_last + 1 : nv + 1;  // exclusive
        const u32 span = vhi > vlo ? vhi - vlo : 0u;
        if (span <= kOffSpan) {
            for (u32 q = tid; q < span; q += kIdxThreads) mark[q] = kOffNone;
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kIdxItems; ++j) {
                const int i = j * kIdxThreads + tid;
                if ((u32)i >= cnt) break;
                const u32 x = st[1 + i];
                const bool head = (t0 + (u64)i == 0) || x != st[i];
                if (head && x >= vlo && x - vlo < span) mark[x - vlo] = (u32)(t0 + (u64)i);
            }
            __syncthreads();
            // suffix minimum over the span: thread t takes a contiguous block
            const u32 per = (span + kIdxThreads - 1) / kIdxThreads;
            const u32 q0 = min(span, (u32)tid * per), q1 = min(span, q0 + per);
            u32 m = kOffNone;
            for (u32 q = q0; q < q1; ++q) m = min(m, mark[q]);
            u32 carry = block_suffix_min(m, s_tmp);
            for (u32 q = q1; q > q0; --q) {
                carry = min(carry, mark[q - 1]);
                mark[q - 1] = carry;
            }
            __syncthreads();
            for (u32 q = tid; q < span; q += kIdxThreads) off[vlo + q] = mark[q];
        } else {
#pragma unroll
            for (int j = 0; j < kIdxItems; ++j) {
                const int i0 = j * kIdxThreads + (tid & ~31);  // the warp's first item
                const u64 k0 = t0 + (u64)i0;
                if (k0 >= n) break;  // warp-uniform
                const u32 x = st[1 + i0 + lane];  // sorted across the lanes; past n: maximum
                const u32 nvalid = (u32)min((u64)32, n - k0);
                const u32 xl = __shfl_sync(0xFFFFFFFFu, x, nvalid - 1);
                const u32 wlo = k0 ? st[i0] + 1 : 0u;
                const u32 whi = xl < nv ? xl + 1 : nv + 1;  // exclusive
                for (u32 cb = wlo; cb < whi; cb += 32) {    // warp-uniform bounds
                    const u32 v = cb + lane;
                    int pos = 0;  // lanes with src < v (at most nvalid - 1 while v <= xl)
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const u32 probe = __shfl_sync(0xFFFFFFFFu, x, pos + step - 1);
                        if (probe < v) pos += step;
                    }
                    if (v < whi) off[v] = (u32)(k0 + (u64)pos);
                }
            }
        }
        __syncthreads();  // the tile is restaged next
    }
}

// ---------------------------------------------------------------------------
// Packed arc offsets: the dense offsets again, in 16 bytes per group of
// kPackVerts vertices, {off[x0], then for j < kPackVerts the byte
// off[x0 + j + 1] - off[x0]}, x0 = kPackVerts * g, so that one load gives a
// vertex's whole run [off[x], off[x+1]).  A group with more than 255 arcs
// (one holding a high-degree vertex) is marked kPackWide and its lookups
// read the offsets themselves.  At 2^25 ids this is 45 MB against the
// offsets' 128 MB: it stays in L2 beside the Step-3 bucket directory through
// the sweep, whose two degree lookups per estimator would otherwise be
// random DRAM reads.  One thread per group; a block stages its groups'
// offsets in shared memory with coalesced loads.
// ---------------------------------------------------------------------------
constexpr u32 kPackVerts = 12;
constexpr u32 kPackWide = 0xFFFFFFFFu;  // offsets are below 2^30: never a base

__host__ __device__ constexpr u64 packed_groups(u64 nv) { return (nv + kPackVerts - 1) / kPackVerts; }

static __global__ void __launch_bounds__(kIdxThreads) pack_offsets_kernel(const u32 *off, u32 nv,
                                                                         uint4 *pdir) {
    __shared__ u32 so[kIdxThreads * kPackVerts + 1];
    const u32 ng = (u32)packed_groups(nv);
    for (u32 t0 = blockIdx.x * kIdxThreads; t0 < ng; t0 += gridDim.x * kIdxThreads) {
        const u32 x0 = t0 * kPackVerts;
        for (u32 q = threadIdx.x; q <= kIdxThreads * kPackVerts; q += kIdxThreads)
            so[q] = __ldg(off + min(x0 + q, nv));  // off has nv + 1 entries
        __syncthreads();
        const u32 g = t0 + threadIdx.x;
        if (g < ng) {
            const u32 *o = so + threadIdx.x * kPackVerts;
            const u32 base = o[0];
            uint4 e = make_uint4(kPackWide, 0u, 0u, 0u);
            if (o[kPackVerts] - base <= 255u) {
                u32 wd[3] = {0u, 0u, 0u};
#pragma unroll
                for (u32 j = 0; j < kPackVerts; ++j) wd[j >> 2] |= (o[j + 1] - base) << (8 * (j & 3));
                e = make_uint4(base, wd[0], wd[1], wd[2]);
            }
            pdir[g] = e;
        }
        __syncthreads();  // the groups' offsets are restaged next
    }
}

// Byte j of a packed entry's run ends (j < kPackVerts).
__device__ __forceinline__ u32 pack_end(const uint4 &q, u32 j) {
    const u32 wd = j < 4 ? q.y : (j < 8 ? q.z : q.w);
    return (wd >> (8 * (j & 3))) & 0xFFu;
}

// Run [start, end) of vertex x (< nv) in the sorted arcs, clamped to the n arcs.
__device__ __forceinline__ void packed_segment(const uint4 *pdir, const u32 *off, u32 x, u32 n,
                                               u32 &start, u32 &end) {
    const u32 g = x / kPackVerts, j = x - g * kPackVerts;
    const uint4 q = __ldg(pdir + g);
    if (q.x != kPackWide) {
        end = min(q.x + pack_end(q, j), n);
        start = min(j ? q.x + pack_end(q, j - 1) : q.x, end);
    } else {
        end = min(__ldg(off + x + 1), n);
        start = min(__ldg(off + x), end);
    }
}

// ---------------------------------------------------------------------------
// Dense Step-3 bucket directory with the filter inside: one 8-byte entry per
// hash bucket b (the top hb bits of h), {first index of the sorted Step-3
// keys whose bucket is >= b, mask}, for b in [0, 2^hb] (entry 2^hb = {w, 0}).
// Bucket b's keys are [entry b, entry b+1); the mask has two bits set for
// each of them, bit (h >> (27 - hb)) & 31 (the five hash bits below the
// bucket's) and bit (h * 0x9E3779B1) >> 27 (a multiplicative rehash, so the
// pair stays independent-ish where hb leaves few bits below the bucket), so
// that a closing pair missing either of its bits has no edge in the batch
// and its lookup ends at that one load (about four edges per bucket: a pair
// with no edge passes about one time in twenty, against one in eight with a
// single bit).  Written whole every batch, like the arc offsets: a tile owns
// the buckets (bucket of the key before it, bucket of its last key]; when
// that span fits the shared arrays, run heads mark their bucket's first
// index and every key ORs its bits into its bucket's mask (the last
// owned bucket's keys past the tile are read from global memory), a suffix
// minimum carries each first index down over empty buckets, and the span is
// written with coalesced stores; a wider span is written head by head.  The
// same pass does the in-batch repeat check: a repeated edge has the repeated
// hash, so it lies in the run of keys sharing the sorted hash bits that
// follows (almost always empty), where the edges with the whole hash are
// compared.
// ---------------------------------------------------------------------------
// The 32-bit hash of a Step-3 key (its bits above the bw position bits).
__device__ __forceinline__ u32 key_hash(u64 key, u32 bw) {
    return __funnelshift_r((u32)key, (u32)(key >> 32), bw);
}

__device__ __forceinline__ u32 filter_bits(u64 h, u32 hb) {
    return (1u << ((h >> (27 - hb)) & 31)) | (1u << (((u32)h * 0x9E3779B1u) >> 27));
}

constexpr u32 kBucketSpan = 3072;  // tiles average 512 buckets (4 keys per bucket)

static __global__ void __launch_bounds__(kIdxThreads) step3_index_kernel(
    const u64 *keys0, const u64 *keys1, const SortPlan *plan, BatchShape s, uint2 *bdir,
    const u64 *__restrict__ W, u32 *err) {
    __shared__ u64 st[kIdxTile + 2];  // st[1 + i] = key t0 + i; st[0], st[kIdxTile + 1]: halo
    __shared__ u32 soff[kBucketSpan], smask[kBucketSpan];
    __shared__ u32 s_tmp[kIdxThreads / 32];
    const u64 *__restrict__ K = plan_final_sel(plan) ? keys1 : keys0;
    const u64 n = s.w;
    const u32 nb = 1u << s.hb;
    const u32 sh = s.bw + 32 - s.hb;  // key -> bucket
    const u64 pmask = (1ull << s.bw) - 1;
    const int tid = threadIdx.x;
    {
        // the buckets past the last key's: every thread takes a share
        const u64 bg = __ldg(K + n - 1) >> sh;
        const u64 stride = (u64)gridDim.x * kIdxThreads;
        for (u64 b = bg + 1 + (u64)blockIdx.x * kIdxThreads + tid; b <= nb; b += stride)
            bdir[b] = make_uint2((u32)n, 0u);
    }
    bool dup = false;
    for (u64 t0 = (u64)blockIdx.x * kIdxTile; t0 < n; t0 += (u64)gridDim.x * kIdxTile) {
#pragma unroll
        for (int j = 0; j < kIdxItems; ++j) {
            const u64 k = t0 + (u64)(j * kIdxThreads + tid);
            st[1 + j * kIdxThreads + tid] = k < n ? __ldg(K + k) : ~0ull;
        }
        if (tid == 0) st[0] = t0 ? __ldg(K + t0 - 1) : 0ull;
        if (tid == 1) st[kIdxTile + 1] = t0 + kIdxTile < n ? __ldg(K + t0 + kIdxTile) : ~0ull;
        __syncthreads();
        const u32 cnt = (u32)min((u64)kIdxTile, n - t0);
        const u64 b_last = st[cnt] >> sh;
        const u64 blo = t0 ? (st[0] >> sh) + 1 : 0;
        const u64 bhi = b_last < nb ? b_last + 1 : (u64)nb + 1;  // exclusive
        const u32 span = bhi > blo ? (u32)(bhi - blo) : 0u;
        const bool fits = span <= kBucketSpan;
        if (fits)
            for (u32 q = tid; q < span; q += kIdxThreads) {
                soff[q] = 0xFFFFFFFFu;
                smask[q] = 0u;
            }
        __syncthreads();
        // per key, all in 32 bits: h is the key's hash (its bits above the
        // bw position bits), the sorted bits are the top hs of h, the bucket
        // the top hb, and positions and indices are below 2^29
        const u32 n32 = (u32)n, t32 = (u32)t0;
        const u32 sh_s = 32 - s.hs, sh_b = 32 - s.hb;
        const u32 blo32 = (u32)blo, bhi32 = (u32)bhi;
#pragma unroll
        for (int j = 0; j < kIdxItems; ++j) {
            const int i = j * kIdxThreads + tid;
            const u32 k = t32 + (u32)i;
            if (k >= n32) break;
            const u64 key = st[1 + i];
            const u32 h = key_hash(key, s.bw);
            const u32 b = h >> sh_b;
            // repeat check: the run of equal sorted bits that follows
            {
                const u32 hp = h >> sh_s;
                u64 e = 0;
                bool have_e = false;
                for (u32 q = k + 1; q < n32; ++q) {
                    const u64 kq = (q - t32 < (u32)kIdxTile + 1) ? st[1 + (q - t32)] : __ldg(K + q);
                    const u32 hq = key_hash(kq, s.bw);
                    if ((hq >> sh_s) != hp) break;
                    if (hq != h) continue;
                    if (!have_e) {
                        e = __ldg(W + (key & pmask));
                        have_e = true;
                    }
                    dup |= __ldg(W + (kq & pmask)) == e;
                }
            }
            if (b < blo32 || b >= bhi32) continue;  // a bucket begun in an earlier tile
            const bool head = (k == 0) || (key_hash(st[i], s.bw) >> sh_b) != b;
            if (fits) {
                if (head) soff[b - blo32] = k;
                atomicOr(&smask[b - blo32], filter_bits(h, s.hb));
            } else if (head) {
                // wide span: this head writes its bucket (mask from its keys)
                // and the empty buckets below it
                u32 mask = 0;
                for (u32 q = k; q < n32; ++q) {
                    const u64 kq = (q - t32 < (u32)kIdxTile + 1) ? st[1 + (q - t32)] : __ldg(K + q);
                    const u32 hq = key_hash(kq, s.bw);
                    if ((hq >> sh_b) != b) break;
                    mask |= filter_bits(hq, s.hb);
                }
                const u32 bprev = k ? (key_hash(st[i], s.bw) >> sh_b) + 1 : 0u;
                for (u32 q = bprev; q < b; ++q) bdir[q] = make_uint2(k, 0u);
                bdir[b] = make_uint2(k, mask);
            }
        }
        __syncthreads();
        if (fits && span) {
            // the last owned bucket's keys past the tile
            if (tid == 0 && b_last < nb) {
                u32 mask = 0;
                for (u64 q = t0 + cnt; q < n; ++q) {
                    const u64 kq = __ldg(K + q);
                    if ((kq >> sh) != b_last) break;
                    mask |= filter_bits(kq >> s.bw, s.hb);
                }
                smask[span - 1] |= mask;
            }
            // suffix minimum of the first indices over the span (blocked per thread)
            const u32 per = (span + kIdxThreads - 1) / kIdxThreads;
            const u32 q0 = min(span, (u32)tid * per), q1 = min(span, q0 + per);
            u32 m = 0xFFFFFFFFu;
            for (u32 q = q0; q < q1; ++q) m = min(m, soff[q]);
            u32 carry = block_suffix_min(m, s_tmp);
            for (u32 q = q1; q > q0; --q) {
                carry = min(carry, soff[q - 1]);
                soff[q - 1] = carry;
            }
            __syncthreads();
            for (u32 q = tid; q < span; q += kIdxThreads)
                bdir[blo + q] = make_uint2(soff[q], smask[q]);
        }
        __syncthreads();  // the tile is restaged next
    }
    if (dup) set_error(err, kErrInput);
}

// Blocks of an index launch over n keys.
inline unsigned index_blocks(u64 n) {
    const u64 b = (n + kIdxTile - 1) / kIdxTile;
    return (unsigned)(b < 152 * 8 ? (b ? b : 1) : 152 * 8);
}

// Blocks of a pack_offsets_kernel launch over 2^B vertex ids: one group per
// thread, at most 8 waves' worth of blocks per SM (grid-stride beyond).
inline unsigned pack_blocks(u32 B, int sm_count) {
    const u64 b = (packed_groups(1ull << B) + kIdxThreads - 1) / kIdxThreads;
    const u64 cap = 8ull * (u64)(sm_count > 0 ? sm_count : 1);
    return (unsigned)(b < cap ? b : cap);
}

// ---------------------------------------------------------------------------
// 128-bit sums (Lemma 3.1's S can exceed 64 bits).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void add_u128(u64 *dst_lo_hi, u64 lo, u64 hi) {
    const u64 old = atomicAdd((unsigned long long *)dst_lo_hi, (unsigned long long)lo);
    const u64 carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry)
        atomicAdd((unsigned long long *)(dst_lo_hi + 1), (unsigned long long)(hi + carry));
}

// Sum a per-thread (lo, hi) pair and a count over the CTA; result valid in
// thread 0.  s_* hold blockDim.x / 32 words each.
__device__ __forceinline__ void block_sum_u128(u64 &lo, u64 &hi, u64 &cnt, u64 *s_lo, u64 *s_hi,
                                               u64 *s_cnt) {
    for (int o = 16; o > 0; o >>= 1) {
        const u64 l2 = __shfl_down_sync(0xFFFFFFFFu, lo, o);
        const u64 h2 = __shfl_down_sync(0xFFFFFFFFu, hi, o);
        cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
        const u64 s = lo + l2;
        hi += h2 + (s < lo ? 1 : 0);
        lo = s;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
        s_cnt[warp] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        lo = 0;
        hi = 0;
        cnt = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            const u64 s = lo + s_lo[k];
            hi += s_hi[k] + (s < lo ? 1 : 0);
            lo = s;
            cnt += s_cnt[k];
        }
    }
}

// ---------------------------------------------------------------------------
// Fused Steps 1-3 per estimator, with the Lemma 3.1 reduction of the
// resulting state folded in.
// ---------------------------------------------------------------------------
struct SweepArgs {
    const u64 *W;
    u64 *f1, *f2, *chi;
    u32 *flags;
    u64 r;
    const u64 *arcs0, *arcs1;
    const u64 *ekeys0, *ekeys1;
    const SortPlan *plans;
    const DirEntry *adir;         // tagged arc directory (kArcTagged)
    const u32 *aoff;              // dense arc offsets, 2^B + 1 entries (kArcDense)
    const uint4 *pdir;            // the same packed, packed_groups(2^B) entries (kArcDense)
    const uint2 *bdir;            // Step-3 buckets: {first key index, filter mask}, 2^hb + 1
    Control *ctl;
    BatchAcc *acc;                // per-batch S / closed accumulator (zeroed)
    const u32 *berr;              // this batch's error word (zeroed)
    u32 epoch;                    // this batch's directory tag
    BatchShape s;
    uint2 key;
    u32 stream;
};

constexpr int kSweepThreads = 256;

// The two non-shared endpoints of the wedge (f1, f2): the closing edge
// (gu < gv) that Step 3 looks up.
__device__ __forceinline__ void closing_pair(u64 f1, u64 f2, u64 &gu, u64 &gv) {
    const u64 a1 = f1 >> 32, b1 = f1 & kMask32, a2 = f2 >> 32, b2 = f2 & kMask32;
    const u64 x1 = (a1 == a2 || a1 == b2) ? b1 : a1;
    const u64 x2 = (a2 == a1 || a2 == b1) ? b2 : a2;
    gu = x1 < x2 ? x1 : x2;
    gv = x1 < x2 ? x2 : x1;
}

// How the sweep finds a vertex's arc run: binary search on the sorted arcs,
// the tagged per-vertex directory, or the dense offsets.
enum ArcDir : int { kArcSearch = 0, kArcTagged = 1, kArcDense = 2 };

// One estimator: Steps 1-3 of Sec. 4 applied to its state in place.
template <int kDir>
__device__ __forceinline__ void sweep_one(const SweepArgs &a, u64 i, u64 m, u32 epoch,
                                          const DrawKey &dk, const u64 *__restrict__ arcs,
                                          const u64 *__restrict__ E, u64 &f1, u64 &f2, u64 &chi,
                                          u32 &fl) {
    const BatchShape &s = a.s;
    const u32 n_arcs = 2u * s.w;
    const u32 wm1 = s.w - 1;
    const u32 wmask = (u32)((1ull << s.bw) - 1);

    // ---- Step 1 (Sec. 4.2): level-1 reservoir over E u W
    const u64 x = draw_bounded(dk, (u32)i, kStep1, m + s.w);
    const bool new1 = x >= m;
    u32 p1 = 0;
    if (new1) {
        p1 = (u32)(x - m);
        f1 = __ldg(a.W + p1);
        chi = 0;
        f2 = kEmpty;
        fl = 0;
    }

    // ---- Step 2 (Sec. 4.3): chi+ = rank(u->v) + rank(v->u), coin, rank-select
    // (positions and indices are 32-bit: a batch has fewer than 2^29 arcs)
    const u64 u = f1 >> 32, v = f1 & kMask32;
    u32 su, eu, sv, ev;
    if constexpr (kDir == kArcDense) {
        packed_segment(a.pdir, a.aoff, (u32)u, n_arcs, su, eu);
        packed_segment(a.pdir, a.aoff, (u32)v, n_arcs, sv, ev);
    } else if constexpr (kDir == kArcTagged) {
        dir_segment32(a.adir, epoch, u, n_arcs, su, eu);
        dir_segment32(a.adir, epoch, v, n_arcs, sv, ev);
    } else {
        u64 s0, e0, s1, e1;
        arc_segment(arcs, n_arcs, s.sha, u, s0, e0);
        arc_segment(arcs, n_arcs, s.sha, v, s1, e1);
        su = (u32)s0, eu = (u32)e0, sv = (u32)s1, ev = (u32)e1;
    }
    u32 ld, rd;
    if (new1) {
        // rank of the arc (x, p1): its offset inside the src segment
        const u64 rp = (u64)(wm1 - p1) << 1;
        ld = lower_bound_idx32(arcs, su, eu, (u << s.sha) | rp) - su;
        rd = lower_bound_idx32(arcs, sv, ev, (v << s.sha) | rp) - sv;
    } else {
        ld = eu - su;  // deg_W(u): Def. 4.2 for a pair outside W
        rd = ev - sv;
    }
    const u64 chi_plus = (u64)ld + rd;
    bool new2 = false;
    u32 p2 = 0;
    if (chi_plus > 0) {
        const u64 y = draw_bounded(dk, (u32)i, kStep2, chi + chi_plus);
        if (y >= chi) {
            const u32 phi = (u32)(y - chi);
            const u32 k = (phi < ld) ? su + phi : sv + (phi - ld);
            const u64 akey = __ldg(arcs + k);
            p2 = wm1 - ((u32)(akey >> 1) & wmask);
            f2 = __ldg(a.W + p2);
            fl &= ~TC_FLAG_CLOSED;
            new2 = true;
        }
    }
    chi += chi_plus;

    // ---- Step 3 (Sec. 4.4): closing edge after f2, looked up by its hash
    // bucket and sorted hash bits; the candidates with its whole hash are
    // checked against W itself
    if (f2 != kEmpty && !(fl & TC_FLAG_CLOSED)) {
        u64 gu, gv;
        u32 lo, hi;
        closing_pair(f1, f2, gu, gv);
        const u64 g = (gu << 32) | gv;
        const u64 h = edge_hash(g, s.hkey);
        const u64 hp = h >> (32 - s.hs);  // the sorted bits
        const u64 bucket = h >> (32 - s.hb);
        // no edge of the batch has both of the pair's filter bits: nothing to
        // look up
        const uint2 e0 = __ldg(a.bdir + bucket);
        const u32 fb = filter_bits(h, s.hb);
        if ((e0.y & fb) == fb) {
            hi = min(__ldg(a.bdir + bucket + 1).x, s.w);
            lo = min(e0.x, hi);
        } else {
            lo = hi = 0;
        }
        for (u32 k = lower_bound_idx32(E, lo, hi, hp << s.she); k < hi; ++k) {
            const u64 ek = __ldg(E + k);
            if ((ek >> s.she) != hp) break;
            if ((ek >> s.bw) != h) continue;
            const u32 q = (u32)ek & wmask;
            if (__ldg(a.W + q) == g) {
                if (!new2 || q > p2) fl |= TC_FLAG_CLOSED;
                break;
            }
        }
    }
}

// One estimator per thread and iteration (grid-stride over r; the grid is
// sweep_blocks(r)).  kDir (ArcDir): how arc segments are found.  Adds
// sum(chi over closed) and the closed count of the new state into a.acc.
template <int kDir>
static __global__ void __launch_bounds__(kSweepThreads, 6) sweep_kernel(SweepArgs a) {
    __shared__ u64 s_lo[kSweepThreads / 32], s_hi[kSweepThreads / 32], s_cnt[kSweepThreads / 32];
    if (ld_relaxed(a.berr)) return;  // rejected batch: state stays as it was
    u64 add = 0, hi = 0, closed = 0;
    const u64 m = a.ctl->m;
    const u32 epoch = a.epoch;
    const DrawKey dk{a.key, (u32)a.ctl->batches, a.stream};
    const u64 *arcs = plan_final_sel(&a.plans[0]) ? a.arcs1 : a.arcs0;
    const bool e_sel = plan_final_sel(&a.plans[1]) != 0;
    const u64 *E = e_sel ? a.ekeys1 : a.ekeys0;
    for (u64 i = (u64)blockIdx.x * kSweepThreads + threadIdx.x; i < a.r;
         i += (u64)gridDim.x * kSweepThreads) {
        // the state streams through once: evict-first, so that L2 keeps the
        // directories and sorted arrays the searches hit at random
        u64 f1 = __ldcs(a.f1 + i), f2 = __ldcs(a.f2 + i), chi = __ldcs(a.chi + i);
        u32 fl = __ldcs(a.flags + i);
        sweep_one<kDir>(a, i, m, epoch, dk, arcs, E, f1, f2, chi, fl);
        __stcs(a.f1 + i, f1);
        __stcs(a.f2 + i, f2);
        __stcs(a.chi + i, chi);
        __stcs(a.flags + i, fl);
        if (fl & TC_FLAG_CLOSED) {
            const u64 t = add + chi;
            hi += t < add ? 1 : 0;
            add = t;
            closed += 1;
        }
    }
    block_sum_u128(add, hi, closed, s_lo, s_hi, s_cnt);
    if (threadIdx.x == 0) {
        if (add | hi) add_u128(&a.acc->s_lo, add, hi);
        if (closed) atomicAdd((unsigned long long *)&a.acc->closed, (unsigned long long)closed);
    }
}

// Blocks of a sweep over r estimators: at most one resident wave of
// `per_sm` blocks per SM (6, the most the launch bounds allow, by default),
// each thread then taking every (blocks x threads)-th estimator.  One
// resident wave measured 3% faster per batch than one block per 256
// estimators at r = 2^20.  A wave of fewer blocks per SM leaves room for the
// next batch's sort passes to run beside the sweep (tc_tune_sweep).
constexpr u32 kSweepBlocksPerSM = 6;
inline unsigned sweep_blocks(u64 r, int sm_count, u32 per_sm = kSweepBlocksPerSM) {
    const u64 b = (r + kSweepThreads - 1) / kSweepThreads;
    const u64 cap = (u64)per_sm * (u64)(sm_count > 0 ? sm_count : 1);
    return (unsigned)(b < cap ? b : cap);
}

// Close the batch: if accepted, count it and commit the estimate of the new
// state; otherwise record the error (state, |E|, batch counter and the
// committed estimate stay as they were).
static __global__ void finish_kernel(Control *ctl, const BatchAcc *acc, const u32 *berr, u64 w) {
    const u32 e = *berr;
    if (e) {
        if (!ctl->sticky) ctl->sticky = e;
    } else {
        ctl->m += w;
        ctl->batches += 1;
        ctl->est[0] = acc->s_lo;
        ctl->est[1] = acc->s_hi;
        ctl->est[2] = acc->closed;
        ctl->est[3] = ctl->m;
    }
    ctl->epoch += 1;
}

// tc_estimate_async: the committed estimate as a tc_estimate_t record in
// device memory (one thread; the same arithmetic as the host's tc_estimate).
static __global__ void estimate_record_kernel(const Control *ctl, u64 r, tc_estimate_t *out) {
    finish_estimate(ctl->est[0], ctl->est[1], ctl->est[2], ctl->est[3], r, ctl->batches, out);
}

// Median-of-means groups: CTA k sums group k = [k*r/g, (k+1)*r/g) into
// out[2k], out[2k+1] (128-bit).
constexpr int kReduceThreads = 256;

static __global__ void __launch_bounds__(kReduceThreads) group_sum_kernel(const u64 *chi, const u32 *flags,
                                                                   u64 r, u32 g, u64 *out) {
    __shared__ u64 s_lo[kReduceThreads / 32], s_hi[kReduceThreads / 32],
        s_cnt[kReduceThreads / 32];
    const u64 k = blockIdx.x;
    const u64 lo_i = (u64)(((unsigned __int128)k * r) / g);
    const u64 hi_i = (u64)(((unsigned __int128)(k + 1) * r) / g);
    u64 lo = 0, hi = 0, cnt = 0;
    for (u64 i = lo_i + threadIdx.x; i < hi_i; i += kReduceThreads) {
        if (flags[i] & TC_FLAG_CLOSED) {
            const u64 s = lo + chi[i];
            hi += (s < lo) ? 1 : 0;
            lo = s;
        }
    }
    block_sum_u128(lo, hi, cnt, s_lo, s_hi, s_cnt);
    if (threadIdx.x == 0) {
        out[2 * k] = lo;
        out[2 * k + 1] = hi;
    }
}

// ---------------------------------------------------------------------------
// rankAll output (Lemma 4.3, Fig. 2): (src, dst, pos, rank) per sorted arc.
// rank = index - start of the src segment: a scan with resets (App. B) done
// as a CTA-wide running maximum of segment-head indices, seeded by one
// binary search for the segment that the tile starts in.
// ---------------------------------------------------------------------------
constexpr int kRankThreads = 256;
constexpr int kRankItems = 4;
constexpr int kRankTile = kRankThreads * kRankItems;

static __global__ void __launch_bounds__(kRankThreads) rank_out_kernel(
    const u64 *W, const u64 *arcs0, const u64 *arcs1, const SortPlan *plan, BatchShape s,
    u32 *src_out, u32 *dst_out, u32 *pos_out, u32 *rank_out) {
    __shared__ u64 s_seed;
    __shared__ u64 s_wmax[kRankThreads / 32];
    const u64 *arcs = plan_final_sel(plan) ? arcs1 : arcs0;
    const u64 n = 2ull * s.w;
    const u64 t0 = (u64)blockIdx.x * kRankTile;
    const u32 wm1 = s.w - 1;
    const u64 wmask = (1ull << s.bw) - 1;
    if (threadIdx.x == 0) s_seed = lower_bound_u64(arcs, n, (arcs[t0] >> s.sha) << s.sha);
    __syncthreads();
    const u64 k0 = t0 + (u64)threadIdx.x * kRankItems;
    u64 heads[kRankItems];
    u64 run = s_seed;
#pragma unroll
    for (int j = 0; j < kRankItems; ++j) {
        const u64 k = k0 + j;
        heads[j] = 0;
        if (k < n) {
            const bool head = (k == 0) || ((arcs[k] >> s.sha) != (arcs[k - 1] >> s.sha));
            if (head) heads[j] = k;
        }
        run = max(run, heads[j]);
    }
    // exclusive running max over threads
    u64 inc = run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const u64 t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc = max(inc, t);
    }
    if (lane == 31) s_wmax[warp] = inc;
    __syncthreads();
    u64 excl = s_seed;
    for (int w2 = 0; w2 < warp; ++w2) excl = max(excl, s_wmax[w2]);
    const u64 prev_lane = __shfl_up_sync(0xFFFFFFFFu, inc, 1);
    if (lane > 0) excl = max(excl, prev_lane);
    u64 seg = excl;
#pragma unroll
    for (int j = 0; j < kRankItems; ++j) {
        const u64 k = k0 + j;
        if (k >= n) break;
        seg = max(seg, heads[j]);
        const u64 key = arcs[k];
        u32 pos = wm1 - (u32)((key >> 1) & wmask);
        if (pos > wm1) pos = wm1;  // only keys left by a timed-out sort can get here
        const u64 e = W[pos];
        src_out[k] = (u32)(key >> s.sha);
        dst_out[k] = (key & 1) ? (u32)(e >> 32) : (u32)(e & kMask32);
        pos_out[k] = pos;
        rank_out[k] = (u32)(k - seg);
    }
}

}  // namespace tc
