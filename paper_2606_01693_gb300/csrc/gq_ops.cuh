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

template <class T, int KIND, bool MATCH = false>
__device__ __forceinline__ int queue_enqueue(const gq_dev& q, T v, u32 tid) {
    if constexpr (KIND == GQ_LFQ) return lfq_enqueue<T, MATCH>(q, v);
    else if constexpr (KIND == GQ_WFQ) return wfq_enqueue<T, MATCH>(q, v, tid);
    else return ymc_enqueue<T, MATCH>(q, v, tid);
}

template <class T, int KIND, bool MATCH = false>
__device__ __forceinline__ int queue_dequeue(const gq_dev& q, T* v, u32 tid) {
    if constexpr (KIND == GQ_LFQ) return lfq_dequeue<T, MATCH>(q, v);
    else if constexpr (KIND == GQ_WFQ) return wfq_dequeue<T, MATCH>(q, v, tid);
    else return ymc_dequeue<T, MATCH>(q, v, tid);
}

// Enqueue (enq, payload *v) or dequeue (!enq, result in *v) chosen per lane.
// G-LFQ and G-WFQ run both on one code path (their operations mirror each
// other over the two index rings); G-WFQ-YMC branches.
template <class T, int KIND>
__device__ __forceinline__ int queue_op(const gq_dev& q, bool enq, T* v, u32 tid) {
    if constexpr (KIND == GQ_LFQ) return lfq_op<T>(q, enq, v);
    else if constexpr (KIND == GQ_WFQ) return wfq_op<T>(q, enq, v, tid);
    else return enq ? ymc_enqueue<T, false>(q, *v, tid) : ymc_dequeue<T, false>(q, v, tid);
}

}  // namespace gqd
