// Internal interface of the multi-stream round engine, shared by the
// tc_multi_* entry points (tc_multi.cu) and the request server
// (tc_serve.cu).  Not part of the C-ABI.
//
// A round folds one batch into each of K participating stream slots.  Every
// slot owns an MStream record in device memory that points at its own
// estimator state (structure of arrays f1/f2/chi/flags over its r
// estimators), so slots can be opened and closed independently and a round
// sweeps only the estimators of the streams taking part in it.
#pragma once

#include <vector>

#include "tc_common.cuh"

namespace tc {

// Per-slot device record.
struct MStream {
    u64 *f1, *f2, *chi;  // estimator state of this stream (r entries each)
    u32 *flags;
    u64 r;               // estimators (0: slot unused)
    u64 m;               // |E| of this stream
    u64 batches;
    uint2 key;           // Philox key (seed lo, seed hi)
    u32 stream_id;
    u32 pad0;            // (a round's errors live in its scratch, one word per participant)
    u32 sticky;          // first error since the host last looked
    u32 pad;
    u64 est[4];          // committed estimate: S lo, S hi, closed, m
    u64 acc[3];          // this round's S lo, S hi, closed
    u64 pad2;
};

// One participant of a round: its slot and its batch (device memory).
struct RoundItem {
    u32 slot;
    const u64 *edges;
    u64 w;  // >= 1
};

// Six words per participant or query, written on the device:
// status (0 or a kErr* code), batches, S lo, S hi, closed, m.
constexpr int kRecordWords = 6;

constexpr int kRing = 8;

}  // namespace tc

struct tc_multi {
    tc::u32 S = 0;       // stream slots
    tc::u32 B = 32;      // vertex id bits
    tc::u32 sb = 1;      // bits of S-1 (round keys carry at most this many)
    tc::u64 w_max = 0;   // most edges one round carries
    tc::u32 force_a = 0, force_e = 0;
    int rank = 0;
    tc::u64 hash_key = 0;                // Step-3 edge hash key (random per engine)
    tc::u64 *state = nullptr;            // state block of tc_multi_create's streams
    std::vector<tc::MStream> h_rec;      // host copy of each slot's static fields
    tc::MStream *ms = nullptr;           // device records, S
    // round scratch: one set, or two when rounds are pipelined (round k+1
    // sorts into the set that round k's sweep is not reading)
    struct RoundSet {
        tc::u64 *arcs[2] = {nullptr, nullptr};
        tc::u64 *ekeys[2] = {nullptr, nullptr};
        tc::u32 *evals[2] = {nullptr, nullptr};
        unsigned char *zeroed = nullptr;  // SortPlan[2], look-back, round error, participant errors
        tc::DirEntry *adir = nullptr;     // arc bucket directory
        tc::DirEntry *edir = nullptr;     // Step-3 bucket directory
        tc::u32 *tag = nullptr;           // device word: the directories' current tag
    };
    RoundSet rset[2];
    tc::u64 set_rounds[2] = {0, 0};      // rounds (replays included) on each set's tags
    int graph_set = 0;                   // the set a captured round uses
    int nsets = 1;
    tc::u32 rseq = 0;                    // rounds enqueued: set parity
    tc::u64 zeroed_bytes = 0;
    cudaStream_t sa = nullptr;           // a pipelined round's sort phase (with `side`)
    cudaEvent_t ev_sorted[2] = {}, ev_swept[2] = {};
    tc::u64 *desc[tc::kRing] = {};       // device round descriptors
    tc::u64 *h_desc[tc::kRing] = {};     // pinned staging (mapped)
    tc::u64 *h_desc_dev[tc::kRing] = {}; // its device address
    cudaEvent_t ring_ev[tc::kRing] = {};
    int ring = 0;
    tc::u64 launches = 0;
    cudaStream_t side = nullptr;         // the edge sort runs here, beside the arc sort
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    tc::MStream *h_ms = nullptr;         // pinned host copy for reads
    cudaGraphExec_t gexec = nullptr;     // captured round (tc_multi_capture)
    tc::u64 *g_desc = nullptr;           // its fixed descriptor
    tc::u64 graph_launches = 0;          // kernels in the captured round
};

namespace tc {

// Words of a round descriptor for K participants.
inline u64 desc_words(u32 K) { return 4 * (u64)K + 2; }

// Allocate an engine with S slots and `sets` (1 or 2; 2 allows pipelined
// rounds) of round scratch for w_max_round edges; slots start unused
// (r = 0).  Returns a TC_* code.
int multi_alloc(u32 S, u64 w_max_round, u32 vertex_bits, tc_multi **out, int sets = 1);
void multi_free(tc_multi *M);

// Bytes of device memory multi_alloc holds for these sizes.
u64 multi_scratch_bytes(u32 S, u64 w_max_round, u32 vertex_bits, int sets = 1);

// Open slot `slot` with r estimators whose state lives at `state` (device,
// 28 r bytes, 8-byte aligned: f1, f2, chi as u64[r], then flags as u32[r]),
// stream-ordered on st: the record is written and the state reset to the
// empty estimator.  The slot must not take part in rounds still queued
// before this call on other streams.
int multi_open_slot(tc_multi *M, u32 slot, u64 r, u64 seed, u32 stream_id, void *state,
                    cudaStream_t st);

// Copy n words with a kernel on st (either side may be mapped pinned host
// memory, by its device address).  Unlike cudaMemcpyAsync this takes no copy
// engine, so it never queues behind copies on other streams: a round's
// descriptor upload would otherwise wait behind the batch copies admitted
// for later rounds.
int copy_words_async(tc_multi *M, u64 *dst, const u64 *src, u64 n, cudaStream_t st);

// The device address of mapped pinned host memory (from cudaHostAlloc with
// cudaHostAllocMapped), or nullptr.
void *mapped_device_ptr(void *h);

// Enqueue one round whose sweep and bookkeeping land on st.  desc: the
// device descriptor of desc_words(K) words; h_desc: if not null, the device
// address of its mapped pinned host copy (written by write_descriptor),
// copied by the round itself ahead of the key build; out: optional device
// array of K * kRecordWords
// words receiving each participant's record after the round.  Pipelined
// (two sets): the sort phase runs on the engine's own streams once wait_ev
// (if any; e.g. the batches' copies) has fired and the round's set is free,
// beside the previous round's sweep.  ev_sort0 / ev_sort1 (optional, with
// timing): recorded on the sort phase's stream once its waits are over and
// when the sort phase ends.
int multi_enqueue(tc_multi *M, const RoundItem *items, u32 K, u64 *desc, const u64 *h_desc,
                  u64 *out, cudaStream_t st, bool pipelined = false,
                  cudaEvent_t wait_ev = nullptr, cudaEvent_t ev_sort0 = nullptr,
                  cudaEvent_t ev_sort1 = nullptr);

// Fill a host descriptor for the given participants; returns the largest w.
u64 write_descriptor(const tc_multi *M, const RoundItem *items, u32 K, u64 *h_desc);

// Enqueue on st the copy of the records of Q slots (device u32 array) into
// the device array out (Q * kRecordWords words), status word 0.
int multi_gather(tc_multi *M, const u32 *d_slots, u32 Q, u64 *out, cudaStream_t st);

}  // namespace tc
