// G-WFQ (Section III-C).  Placeholder until the slow path lands; the word
// layouts below are final.
#pragma once
#include "gq_lfq.cuh"
namespace gqd {

// Slot <Note 19 | Cycle 19 | Safe 1 | Enq 1 | Index 24> (Fig. "Entry word for
// G-WFQ", widths as read for this build: the 8-bit tags of the figure are too
// narrow for R > Dk/n + 6 at k > n).
constexpr int kWNoteShift = 45, kWCycShift = 26;
constexpr u64 kWSafe = 1ull << 25, kWEnq = 1ull << 24;
constexpr u32 kWIdxMask = (1u << 24) - 1;
constexpr u32 kWBot = kWIdxMask, kWBotC = kWIdxMask - 1;
constexpr u64 kWFieldMask = (1ull << 19) - 1;

__host__ __device__ __forceinline__ u64 wfq_entry(u64 note, u64 cyc, u64 safe, u64 enq, u32 idx) {
    return (note << kWNoteShift) | (cyc << kWCycShift) | (safe ? kWSafe : 0) | (enq ? kWEnq : 0) | idx;
}

// Global Head/Tail <Counter 43 | ThrIdx 21>, ThrIdx 0 = NULL, record r -> r + 1.
constexpr int kGThrBits = 21;
constexpr u64 kGThrMask = (1ull << kGThrBits) - 1;
constexpr u64 kGOne = 1ull << kGThrBits;
__host__ __device__ __forceinline__ u64 wfq_global(u64 cnt, u64 thr) { return (cnt << kGThrBits) | thr; }

template <class T, bool MATCH>
__device__ int wfq_enqueue(const gq_dev& q, T v, u32 tid) { return GQ_ERR_INVALID; }
template <class T, bool MATCH>
__device__ int wfq_dequeue(const gq_dev& q, T* v, u32 tid) { return GQ_ERR_INVALID; }
}  // namespace gqd
