/*
 * gq_device.cuh -- device-side API of libgq for user kernels.
 *
 * Obtain a gq_dev with gq_device_view() on the host and pass it by value to a
 * kernel compiled for sm_103a with -I <repo>/include.  Then any thread may call
 *
 *   int gq_enqueue(const gq_dev& q, unsigned long long v, unsigned tid);
 *   int gq_dequeue(const gq_dev& q, unsigned long long* v, unsigned tid);
 *
 * returning GQ_OK, GQ_FULL (bounded queues), GQ_EMPTY, or a negative gq_status.
 * These are the queues' Enq / Deq operations (Section III; G-LFQ Algorithm 1,
 * G-WFQ Algorithm 2, G-WFQ-YMC Section III-A), linearizable with the host batch
 * calls and with other kernels on the same queue.
 *
 *   - Any subset of a warp's lanes may call, under divergent control flow; the
 *     lanes converged at a call batch their ticket reservation (WaveFAA), and
 *     lanes that target different queues are grouped by queue address.
 *   - tid names the caller's per-thread record (G-WFQ and G-WFQ-YMC keep one
 *     fixed record per participating thread, Section III-C): it must be below
 *     the queue's max_threads and no two threads that operate at the same time
 *     may use the same tid.  G-LFQ ignores it.
 *   - 4-byte queues store the low 32 bits of v and return them zero-extended.
 *     G-WFQ-YMC 8-byte queues reject v >= 2^64 - 2 (GQ_ERR_RESERVED_VALUE).
 *   - Errors detected on the device are also latched in the queue's error
 *     word (read with gq_sync_status on the host).
 */
#ifndef GQ_DEVICE_CUH
#define GQ_DEVICE_CUH

#include "gq.h"
#include "../paper_2606_01693_gb300/csrc/gq_ops.cuh"

__device__ __forceinline__ int gq_enqueue(const gq_dev& q, unsigned long long v, unsigned tid) {
    if (q.elem_bytes == 4) {
        const unsigned int x = (unsigned int)v;
        switch (q.kind) {
            case GQ_LFQ: return gqd::queue_enqueue<unsigned int, GQ_LFQ, true>(q, x, tid);
            case GQ_WFQ: return gqd::queue_enqueue<unsigned int, GQ_WFQ, true>(q, x, tid);
            default: return gqd::queue_enqueue<unsigned int, GQ_YMC, true>(q, x, tid);
        }
    }
    switch (q.kind) {
        case GQ_LFQ: return gqd::queue_enqueue<unsigned long long, GQ_LFQ, true>(q, v, tid);
        case GQ_WFQ: return gqd::queue_enqueue<unsigned long long, GQ_WFQ, true>(q, v, tid);
        default: return gqd::queue_enqueue<unsigned long long, GQ_YMC, true>(q, v, tid);
    }
}

__device__ __forceinline__ int gq_dequeue(const gq_dev& q, unsigned long long* v, unsigned tid) {
    if (q.elem_bytes == 4) {
        unsigned int x = 0;
        int s;
        switch (q.kind) {
            case GQ_LFQ: s = gqd::queue_dequeue<unsigned int, GQ_LFQ, true>(q, &x, tid); break;
            case GQ_WFQ: s = gqd::queue_dequeue<unsigned int, GQ_WFQ, true>(q, &x, tid); break;
            default: s = gqd::queue_dequeue<unsigned int, GQ_YMC, true>(q, &x, tid); break;
        }
        if (s == GQ_OK) *v = x;
        return s;
    }
    switch (q.kind) {
        case GQ_LFQ: return gqd::queue_dequeue<unsigned long long, GQ_LFQ, true>(q, v, tid);
        case GQ_WFQ: return gqd::queue_dequeue<unsigned long long, GQ_WFQ, true>(q, v, tid);
        default: return gqd::queue_dequeue<unsigned long long, GQ_YMC, true>(q, v, tid);
    }
}

#endif /* GQ_DEVICE_CUH */
