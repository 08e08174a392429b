// Kind dispatch for the queue operations: one enqueue/dequeue entry per
// (payload type, queue kind).  `tid` names the caller's per-thread record
// (G-WFQ and G-WFQ-YMC keep one fixed record per participating thread,
// Section III-A and III-C); G-LFQ ignores it.
#pragma once

#include "gq_atomics.cuh"
#include "gq_lfq.cuh"
#include "gq_wfq.cuh"
#include "gq_ymc.cuh"

namespace gqd {

// tk (nullable, test recorder only): receives the operation's ticket in the
// allocated-index ring (G-LFQ, G-WFQ) or its cell (G-WFQ-YMC); an item's
// enqueue and the dequeue that returns it get the same one.
// CNT: the counting instantiation (per-thread event counts, see gq_atomics.cuh).
// seq (run drivers): the index of the operation among the thread's operations
// on this queue; G-WFQ derives its help delay from it (wfq_maybe_help).
template <class T, int KIND, bool MATCH = false, bool CNT = false>
__device__ __forceinline__ int queue_enqueue(const gq_dev& q, T v, u32 tid, u64* tk = nullptr, u32 seq = kNoSeq) {
    if constexpr (KIND == GQ_LFQ) return lfq_enqueue<T, MATCH, CNT>(q, v, tk);
    else if constexpr (KIND == GQ_WFQ) return wfq_enqueue<T, MATCH, CNT>(q, v, tid, tk, seq);
    else return ymc_enqueue<T, MATCH, CNT>(q, v, tid, tk);
}

template <class T, int KIND, bool MATCH = false, bool CNT = false>
__device__ __forceinline__ int queue_dequeue(const gq_dev& q, T* v, u32 tid, u64* tk = nullptr, u32 seq = kNoSeq) {
    if constexpr (KIND == GQ_LFQ) return lfq_dequeue<T, MATCH, CNT>(q, v, tk);
    else if constexpr (KIND == GQ_WFQ) return wfq_dequeue<T, MATCH, CNT>(q, v, tid, tk, seq);
    else return ymc_dequeue<T, MATCH, CNT>(q, v, tid, tk);
}

// Enqueue (enq, payload *v) or dequeue (!enq, result in *v) chosen per lane.
// G-LFQ and G-WFQ run both on one code path (their operations mirror each
// other over the two index rings); G-WFQ-YMC branches.
template <class T, int KIND, bool CNT = false>
__device__ __forceinline__ int queue_op(const gq_dev& q, bool enq, T* v, u32 tid, u64* tk = nullptr, u32 seq = kNoSeq) {
    if constexpr (KIND == GQ_LFQ) return lfq_op<T, CNT>(q, enq, v, tk);
    else if constexpr (KIND == GQ_WFQ) return wfq_op<T, CNT>(q, enq, v, tid, tk, seq);
    else return enq ? ymc_enqueue<T, false, CNT>(q, *v, tid, tk) : ymc_dequeue<T, false, CNT>(q, v, tid, tk);
}

}  // namespace gqd
