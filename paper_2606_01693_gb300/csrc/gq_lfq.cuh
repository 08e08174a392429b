// G-LFQ: bounded lock-free ring with warp-batched tickets (Section III-B,
// Algorithm 1), and the index-indirection layer around it.
//
// Inner ring ("Data structure", Section III-B): 2n physical slots, logical
// capacity n, monotonically increasing Head and Tail tickets, a Threshold for
// empty detection.  Ticket t maps to slot(t) = t mod 2n and
// cycle(t) = floor(t / 2n) mod R, R = 2^cycle_bits.  Each slot is one 64-bit word
//     bits 63..33  Cycle (cycle_bits <= 31 wide, the rest zero)
//     bit  32      Safe
//     bits 31..0   Index:  a value < 2^32 - 2,  BOT = 2^32 - 1 (empty),
//                          BOTC = 2^32 - 2 (consumed)
// Consume marks the index field BOTC and keeps the Cycle and Safe bits: a CAS
// from the entry the dequeuer read to the same entry with index BOTC, falling
// back to an atomic OR of BOTC into the index bits (any index then becomes
// BOTC or BOT, both of the "empty class") if a concurrent Safe change made the
// CAS fail.  Writing exactly BOTC keeps a consumed slot's value predictable.
// Cycles are compared modulo R (a is older than b iff 0 < (b - a) mod R < R/2),
// sound while the live skew on a slot stays below R/2 (Lemma "Reduced-width
// cycle tags").
//
// The ring itself does not detect FULL: it relies on never holding more than n
// indices.  The outer queue guarantees that: "fq" starts full with 0..n-1, "aq"
// starts empty, and every user enqueue first takes a free index from fq
// (none left = FULL), stores the payload at data[index] and puts the index in
// aq; a dequeue takes an index from aq, reads the payload and returns the
// index to fq (Section III-B "outer indirection layer that moves indices").
//
// GPU-first choices (differences from the CPU sCQ ring):
//   * tickets of one warp are consecutive, so the 32 slot RMWs of a warp hit two
//     adjacent 128-byte lines and coalesce into few L2 atomic requests; sCQ's
//     cache-line remapping of consecutive tickets is deliberately not used;
//   * a CAS that fails on a slot re-evaluates the same ticket with the value it
//     returned (no ticket is burned for a lost race on a still-usable slot);
//   * an enqueue first CASes against the slot's most likely value, "consumed in
//     the previous cycle" <c-1, Safe, BOTC>, instead of loading it: a right
//     guess saves one L2 round trip, a wrong one returns the current value,
//     which the protocol then evaluates exactly as a load's result.
#pragma once

#include "gq_atomics.cuh"

namespace gqd {

constexpr u64 kSafe = 1ull << 32;
constexpr u32 kBot = 0xFFFFFFFFu;
constexpr u32 kBotC = 0xFFFFFFFEu;

// Ring geometry is precomputed on the host into gq_dev (slot_mask = 2n - 1,
// ring_order = log2(2n), cycle_mask = R - 1, cycle_half = R / 2, thr_reset =
// 3n - 1) and read where it is used: a kernel parameter lives in the constant
// bank, so the geometry costs no registers in the hot loops.

// a is strictly older than b (modular, Lemma on cycle tags)
__device__ __forceinline__ bool cyc_older(u64 a, u64 b, const gq_dev& q) {
    const u64 d = (b - a) & q.cycle_mask;
    return d != 0 && d < q.cycle_half;
}

__device__ __forceinline__ u64 lfq_cycle(u64 e) { return e >> 33; }
__device__ __forceinline__ u32 lfq_index(u64 e) { return (u32)e; }
__device__ __forceinline__ u64 lfq_entry(u64 cyc, u64 safe, u32 idx) { return (cyc << 33) | safe | idx; }

// Threshold updates are relaxed RMWs: the counter carries no payload, and an
// RMW is performed at L2 before the issuing thread continues, so a later
// operation (in real time) reads the updated value.  The reset's old value is
// consumed so that it is issued as a returning atomic, not a fire-and-forget.
__device__ __forceinline__ void thr_reset(i64* thr, i64 v, unsigned int* err) {
    if (aref<i64>(*thr).exchange(v, kRlx) == INT64_MIN) latch_error(err, GQ_ERR_INVALID);
}
__device__ __forceinline__ i64 thr_dec(i64* thr) { return aref<i64>(*thr).fetch_add(-1, kRlx); }

// Catch Tail up to at least `head` = this dequeuer's ticket + 1 (Algorithm 1
// TryDeq, "catch up Tail").  One atomic maximum: Tail only grows, by fetch-add
// (enqueuers) or by this maximum, and afterwards Tail >= head, which is all an
// EMPTY dequeue needs so that later enqueuers take tickets past it.  A CAS loop
// that re-reads Head instead chases every concurrent dequeuer's ticket, and
// with tens of thousands of lanes turning EMPTY together it ran for
// milliseconds.
__device__ __forceinline__ void ring_catchup(const gq_ring_view& r, u64 head) {
    atomicMax(reinterpret_cast<unsigned long long*>(r.tail), head);
}

// Inner-ring enqueue of index `idx` (TryEnq of Algorithm 1, retried until it
// succeeds).  Returns GQ_OK, or GQ_ERR_TIMEOUT if the retry bound expires.
// tk (nullable, test recorder): receives the ticket the index was installed at.
template <bool MATCH>
__device__ int lfq_ring_enq(const gq_dev& q, const gq_ring_view& r, u32 idx, u64* tk = nullptr) {
    for (u32 it = 0; it < kRetryLimit; ++it) {
        const u64 t = warp_faa<MATCH>(r.tail, 1, q.batch_width);
        u64* slot = r.slots + (t & q.slot_mask);
        const u64 c = (t >> q.ring_order) & q.cycle_mask;
        const u64 ne = lfq_entry(c, kSafe, idx);
        u64 e = lfq_entry((c - 1) & q.cycle_mask, kSafe, kBotC);   // predicted current value
        bool done = cas(slot, e, ne);
        for (; !done && it < kRetryLimit; ++it) {
            if (!cyc_older(lfq_cycle(e), c, q) || lfq_index(e) < kBotC) break;
            if (!(e & kSafe)) {
                // an unsafe slot may be reused only if no dequeuer has passed t
                if ((i64)(ld_rlx(r.head) - t) > 0) break;
            }
            done = cas(slot, e, ne);
            // CAS lost: e holds the current entry; re-evaluate the same ticket
        }
        if (done) {
            if (ld_rlx(r.threshold) != q.thr_reset) thr_reset(r.threshold, q.thr_reset, q.err);
            if (tk) *tk = t;
            return GQ_OK;
        }
        if (q.backoff_ns) __nanosleep(q.backoff_ns);
    }
    latch_error(q.err, GQ_ERR_TIMEOUT);
    return GQ_ERR_TIMEOUT;
}

// Inner-ring dequeue (TryDeq of Algorithm 1, retried while it returns RETRY).
// Returns GQ_OK with *idx, GQ_EMPTY, or GQ_ERR_TIMEOUT.  tk (nullable): the
// ticket the index was taken at.
template <bool MATCH>
__device__ int lfq_ring_deq(const gq_dev& q, const gq_ring_view& r, u32* idx, u64* tk = nullptr) {
    if (ld_rlx(r.threshold) < 0) return GQ_EMPTY;
    for (u32 it = 0; it < kRetryLimit; ++it) {
        const u64 h = warp_faa<MATCH>(r.head, 1, q.batch_width);
        u64* slot = r.slots + (h & q.slot_mask);
        const u64 c = (h >> q.ring_order) & q.cycle_mask;
        u64 e = ld_acq(slot);
        for (; it < kRetryLimit; ++it) {
            const u64 ec = lfq_cycle(e);
            if (ec == c) {
                if (lfq_index(e) < kBotC) {          // Consume and return the index
                    *idx = lfq_index(e);
                    if (tk) *tk = h;
                    // relaxed: the acquire load of e already ordered the payload read
                    if (!aref<u64>(*slot).compare_exchange_strong(e, (e & ~0xFFFFFFFFull) | kBotC, kRlx, kRlx))
                        aref<u64>(*slot).fetch_or(kBotC, kRlx);
                    return GQ_OK;
                }
                break;
            }
            if (!cyc_older(ec, c, q)) break;         // slot already belongs to a later cycle
            // empty class: advance the slot to cycle c (still empty);
            // occupied by an older cycle: clear Safe so the enqueuer of t = h
            // does not reuse it once Head has passed h.
            const u64 ne = (lfq_index(e) >= kBotC) ? lfq_entry(c, e & kSafe, kBot) : (e & ~kSafe);
            if (cas(slot, e, ne)) break;
        }
        const u64 tl = ld_rlx(r.tail);
        if ((i64)(tl - (h + 1)) <= 0) {
            ring_catchup(r, h + 1);
            thr_dec(r.threshold);
            return GQ_EMPTY;
        }
        if (thr_dec(r.threshold) <= 0) return GQ_EMPTY;
        if (q.backoff_ns) __nanosleep(q.backoff_ns);
    }
    latch_error(q.err, GQ_ERR_TIMEOUT);
    return GQ_ERR_TIMEOUT;
}

// ---------------------------------------------------------------------------
// Outer queue over two rings (indirection layer)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void data_store(const gq_dev& q, u32 i, T v) {
    aref<T>(static_cast<T*>(q.data)[i]).store(v, kRlx);
}
template <class T>
__device__ __forceinline__ T data_load(const gq_dev& q, u32 i) {
    return aref<T>(static_cast<T*>(q.data)[i]).load(kRlx);
}

// tk (nullable, test recorder): the aq ticket of the operation (an item's
// enqueue and its dequeue share it).
template <class T, bool MATCH>
__device__ int lfq_enqueue(const gq_dev& q, T v, u64* tk = nullptr) {
    u32 i;
    int s = lfq_ring_deq<MATCH>(q, q.fq, &i);
    if (s == GQ_EMPTY) return GQ_FULL;
    if (s != GQ_OK) return s;
    if (i >= q.capacity) {                            // never expected: a corrupt ring entry
        latch_error(q.err, GQ_ERR_INVALID);
        return GQ_ERR_INVALID;
    }
    data_store<T>(q, i, v);                           // ordered before the release CAS in aq
    return lfq_ring_enq<MATCH>(q, q.aq, i, tk);
}

template <class T, bool MATCH>
__device__ int lfq_dequeue(const gq_dev& q, T* v, u64* tk = nullptr) {
    u32 i;
    int s = lfq_ring_deq<MATCH>(q, q.aq, &i, tk);
    if (s != GQ_OK) return s;
    if (i >= q.capacity) {                            // never expected: a corrupt ring entry
        latch_error(q.err, GQ_ERR_INVALID);
        return GQ_ERR_INVALID;
    }
    *v = data_load<T>(q, i);                          // after the acquire on the aq slot
    s = lfq_ring_enq<MATCH>(q, q.fq, i);              // release: the read precedes reuse
    return s == GQ_OK ? GQ_OK : s;
}

// Enqueue (enq = true, payload *v) or dequeue (enq = false, result in *v) on
// one code path.  Both are "take an index from one ring, move the payload,
// give the index to the other ring": enqueue takes from fq and gives to aq,
// dequeue the reverse.  Selecting the rings per lane lets a warp whose lanes
// mix enqueues and dequeues run them together instead of one after the other
// (divergent branches); WaveFAA groups the lanes by counter address.  Each
// lane performs exactly the steps of its own operation.
template <class T>
__device__ int lfq_op(const gq_dev& q, bool enq, T* v, u64* tk = nullptr) {
    const gq_ring_view& from = enq ? q.fq : q.aq;
    const gq_ring_view& to = enq ? q.aq : q.fq;
    u32 i;
    int s = lfq_ring_deq<true>(q, from, &i, enq ? nullptr : tk);
    if (s == GQ_EMPTY) return enq ? GQ_FULL : GQ_EMPTY;
    if (s != GQ_OK) return s;
    if (i >= q.capacity) {                            // never expected: a corrupt ring entry
        latch_error(q.err, GQ_ERR_INVALID);
        return GQ_ERR_INVALID;
    }
    if (enq) data_store<T>(q, i, *v);                 // ordered before the release CAS in aq
    else *v = data_load<T>(q, i);                     // after the acquire on the aq slot
    return lfq_ring_enq<true>(q, to, i, enq ? tk : nullptr);
}

}  // namespace gqd
