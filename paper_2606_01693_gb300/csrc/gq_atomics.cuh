// Device-side primitives shared by the three queues: scoped atomics, the
// warp-batched ticket reservation (WaveFAA), lane helpers and error latching.
//
// Memory model.  All shared queue words are accessed through
// cuda::atomic_ref<..., thread_scope_device> (PTX .gpu scope):
//   * slot and record RMWs are acq_rel, slot loads are acquire, so a value
//     published by a release CAS (payload stored, then index installed) is seen
//     with everything written before it;
//   * ticket counters use relaxed fetch-add: the ticket order itself is the
//     only thing they carry, and every decision that depends on a counter value
//     read later is ordered after an acquire on the slot it concerns.
#pragma once

#include <cuda/atomic>
#include <stdint.h>

#include "../../include/gq.h"

namespace gqd {

typedef unsigned long long u64;
typedef long long i64;
typedef unsigned int u32;

template <class T>
using aref = cuda::atomic_ref<T, cuda::thread_scope_device>;

constexpr cuda::std::memory_order kRlx = cuda::std::memory_order_relaxed;
constexpr cuda::std::memory_order kAcq = cuda::std::memory_order_acquire;
constexpr cuda::std::memory_order kRel = cuda::std::memory_order_release;
constexpr cuda::std::memory_order kAR = cuda::std::memory_order_acq_rel;

// Upper bound on the retries of any lock-free loop.  Reaching it is not an
// expected outcome; it exists so that no kernel can spin without end: the
// operation latches GQ_ERR_TIMEOUT and returns.
constexpr u32 kRetryLimit = 1u << 16;

__device__ __forceinline__ u64 ld_acq(u64* p) { return aref<u64>(*p).load(kAcq); }
__device__ __forceinline__ u64 ld_rlx(u64* p) { return aref<u64>(*p).load(kRlx); }
__device__ __forceinline__ i64 ld_rlx(i64* p) { return aref<i64>(*p).load(kRlx); }
__device__ __forceinline__ void st_rlx(u64* p, u64 v) { aref<u64>(*p).store(v, kRlx); }
__device__ __forceinline__ void st_rel(u64* p, u64 v) { aref<u64>(*p).store(v, kRel); }
__device__ __forceinline__ u32 ld_rlx32(u32* p) { return aref<u32>(*p).load(kRlx); }
__device__ __forceinline__ void st_rlx32(u32* p, u32 v) { aref<u32>(*p).store(v, kRlx); }

// CAS with acq_rel on success, acquire on failure; `expected` receives the
// current value when it fails.
__device__ __forceinline__ bool cas(u64* p, u64& expected, u64 desired) {
    return aref<u64>(*p).compare_exchange_strong(expected, desired, kAR, kAcq);
}
__device__ __forceinline__ bool cas_rlx(u64* p, u64& expected, u64 desired) {
    return aref<u64>(*p).compare_exchange_strong(expected, desired, kRlx, kRlx);
}
__device__ __forceinline__ u64 faa_rlx(u64* p, u64 v) { return aref<u64>(*p).fetch_add(v, kRlx); }
__device__ __forceinline__ i64 faa(i64* p, i64 v) { return aref<i64>(*p).fetch_add(v, kAR); }
__device__ __forceinline__ u64 fetch_or(u64* p, u64 v) { return aref<u64>(*p).fetch_or(v, kAR); }
__device__ __forceinline__ u64 fetch_and(u64* p, u64 v) { return aref<u64>(*p).fetch_and(v, kAR); }
__device__ __forceinline__ i64 exch(i64* p, i64 v) { return aref<i64>(*p).exchange(v, kAR); }
// Relaxed atomic maximum that returns nothing.
__device__ __forceinline__ void red_max_rlx(u64* p, u64 v) {
    asm volatile("red.relaxed.gpu.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Relaxed atomic OR that returns nothing (a reduction): the issuing thread does
// not wait for it.  Later release operations of the thread still order it.
__device__ __forceinline__ void red_or_rlx(u64* p, u64 v) {
    asm volatile("red.relaxed.gpu.or.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ u32 lane_id() {
    u32 r;
    asm volatile("mov.u32 %0, %%laneid;" : "=r"(r));
    return r;
}
__device__ __forceinline__ u32 lanemask_lt() {
    u32 r;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}
__device__ __forceinline__ u64 globaltimer() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// WaveFAA (Algorithm 1, Lemma "WaveFAA preserves ticket order").  The lanes of
// the warp that are converged at the call form the batch: the lowest lane
// performs one fetch-and-add of popc(mask) * step on the counter, broadcasts
// the old value, and every lane adds its rank (popc of the lower lanes) * step.
// The batch receives consecutive tickets; one global atomic per batch.
// `width` (a power of two <= 32) splits the warp into aligned groups of that
// many lanes, each batching on its own (width 1 = one atomic per thread).
// MATCH groups lanes by counter address first (__match_any_sync), for callers
// whose lanes may target different queues.
// ---- operation counters (counting instantiations only) ---------------------
// Kernels instantiated with CNT = true count the events of each operation's
// fast path per thread in shared memory (one column per thread of the block;
// a thread only touches its own entries, so plain increments suffice) and sum
// them per warp at the end.  Kernels instantiated with CNT = false -- every
// timed kernel -- contain none of it.  Event kinds (GQ_OC_* in gq_drivers.h):
enum : int {
    kOcTicket = 0,   // tickets taken (one per lane per counter reservation)
    kOcFaa = 1,      // counter fetch-and-adds issued (one per WaveFAA batch)
    kOcCas = 2,      // CAS attempts on slots / cells (install, repair, consume, claim)
    kOcCasFail = 3,  // ... of which failed
    kOcRmw = 4,      // other slot RMWs (the atomic-OR fallback of Consume)
    kOcThr = 5,      // Threshold RMWs (reset exchange, decrement)
    kOcCatch = 6,    // catch-up operations on Tail / T / H
    kOcBurn = 7,     // tickets given up without an install or an item (RETRY, EMPTY)
    kOcLoad = 8,     // slot / cell loads (first read of the ticket's slot or cell)
    kOcSlow = 9,     // slow-path requests (G-WFQ, G-WFQ-YMC)
    kOcSpin = 10,    // further reads of an empty slot / cell while its enqueuer is due
    kOcMark = 11,    // G-WFQ-YMC: cells marked unusable by a dequeuer
    kOcN = 12
};
constexpr int kOcMaxBlock = 256;

__device__ __forceinline__ u32* oc_table() {
    __shared__ u32 s_oc[kOcN * kOcMaxBlock];
    return s_oc;
}
template <bool CNT>
__device__ __forceinline__ void oc_add(int what, u32 n = 1) {
    if constexpr (CNT) oc_table()[what * kOcMaxBlock + threadIdx.x] += n;
}
template <bool CNT>
__device__ __forceinline__ void oc_cas(bool ok) {
    if constexpr (CNT) {
        oc_table()[kOcCas * kOcMaxBlock + threadIdx.x] += 1;
        if (!ok) oc_table()[kOcCasFail * kOcMaxBlock + threadIdx.x] += 1;
    }
}

template <bool MATCH = false, bool CNT = false>
__device__ __forceinline__ u64 warp_faa(u64* ctr, u64 step, u32 width = 32) {
    u32 mask = __activemask();
    if (MATCH) mask = __match_any_sync(mask, reinterpret_cast<u64>(ctr));
    if (width < 32) mask &= ((1u << width) - 1u) << (lane_id() & ~(width - 1u));
    const u32 leader = __ffs(mask) - 1;
    u64 base = 0;
    oc_add<CNT>(kOcTicket);
    if (lane_id() == leader) {
        oc_add<CNT>(kOcFaa);
        base = faa_rlx(ctr, step * (u64)__popc(mask));
    }
    base = __shfl_sync(mask, base, leader);
    return base + step * (u64)__popc(mask & lanemask_lt());
}

// One fetch-and-add per thread (batch width 1): the un-batched baseline of
// the warp-batching ablation.
__device__ __forceinline__ u64 thread_faa(u64* ctr, u64 step) { return faa_rlx(ctr, step); }

// Latches the first device-side error; later errors keep the first one.
__device__ __forceinline__ void latch_error(unsigned int* err, int code) {
    if (err) atomicCAS(err, 0u, (unsigned int)(-code));
}

// Sum of a per-thread value over the warp, added to *dst by one lane.  Kernels
// call it once, at their end, from every thread of the block; a partial last
// warp (block size not a multiple of 32) falls back to one atomic per lane.
__device__ __forceinline__ void warp_add_full(unsigned long long* dst, u64 v) {
    if (__activemask() != 0xffffffffu) {
        if (v) atomicAdd(dst, v);
        return;
    }
    __syncwarp();
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0 && v) atomicAdd(dst, v);
}

// Counting kernels: zero this thread's counters at the start, add the warp's
// sums to dst[0 .. kOcN) at the end.  Every thread of the block calls both, and
// blocks are whole warps.  The end first gathers all 32 lanes (__syncwarp), so
// the reductions run in lockstep: lanes that arrive at different times must not
// meet in one reduction at different counters (warp_add_full inside a loop
// could: its active-mask test sees lanes of different iterations at one PC).
template <bool CNT>
__device__ __forceinline__ void oc_begin() {
    if constexpr (CNT)
        for (int k = 0; k < kOcN; ++k) oc_table()[k * kOcMaxBlock + threadIdx.x] = 0;
}
template <bool CNT>
__device__ __forceinline__ void oc_end(unsigned long long* dst) {
    if constexpr (CNT) {
        __syncwarp();
        for (int k = 0; k < kOcN; ++k) {
            u64 v = oc_table()[k * kOcMaxBlock + threadIdx.x];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane_id() == 0 && v) atomicAdd(dst + k, v);
        }
    }
}

}  // namespace gqd
