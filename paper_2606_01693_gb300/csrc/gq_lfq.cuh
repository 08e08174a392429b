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
// Consume empties the index field and keeps the Cycle and Safe bits: one
// atomic OR of all ones into the index bits, so a consumed slot always reads
// <cycle, Safe, BOT> (BOT and BOTC are both of the "empty class"; the ring
// treats them alike).  While a slot holds a live index only its consumer
// changes the index bits (others CAS the Safe bit), so the OR needs no expected
// value and returns nothing: the dequeuer does not wait for it.
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
//   * an enqueue first CASes against the slot's most likely value, "emptied in
//     the previous cycle" <c-1, Safe, BOT>, instead of loading it: a right
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

// ---- warp-aggregated updates of the hot Threshold and Tail words -----------
// In near-empty and near-full rings most ring operations end on the Threshold
// word (a decrement per failed dequeue, a reset per install that finds it
// changed), all on one address per ring: at one RMW per lane those serialise
// at the single-address rate.  The converged lanes that update the same word
// do it with one RMW, as WaveFAA does for tickets, and every lane sees the
// outcome its own update would have had with the group's updates applied in
// lane order.  Each helper gathers the group (lanes at this call with the same
// target word), lets its lowest lane perform the update, and releases the
// group only after that RMW returned (__syncwarp), so no lane goes on before
// its share of the update is done.

__device__ __forceinline__ u32 group_of(const void* p) {
    return __match_any_sync(__activemask(), reinterpret_cast<u64>(p));
}

// Threshold decrement by the group: returns this lane's old value (the value
// minus the decrements of the lower lanes of its group).
template <bool CNT = false>
__device__ __forceinline__ i64 thr_dec_group(i64* thr) {
    const u32 mask = group_of(thr);
    const u32 leader = __ffs(mask) - 1;
    u64 base = 0;
    if (lane_id() == leader) {
        oc_add<CNT>(kOcThr);
        base = (u64)aref<i64>(*thr).fetch_add(-(i64)__popc(mask), kRlx);
    }
    base = __shfl_sync(mask, base, leader);
    return (i64)base - (i64)__popc(mask & lanemask_lt());
}

// Threshold reset after installs: the group's lowest lane resets it (if it
// changed) once for all of them; every lane's install precedes the reset.
template <bool CNT = false>
__device__ __forceinline__ void thr_reset_group(i64* thr, i64 v, unsigned int* err) {
    const u32 mask = group_of(thr);
    if (lane_id() == __ffs(mask) - 1 && ld_rlx(thr) != v) {
        oc_add<CNT>(kOcThr);
        thr_reset(thr, v, err);
    }
    __syncwarp(mask);
}

// Largest head of the group (tickets of concurrent operations lie within 2^31
// of one another, so offsets from the lowest lane's head fit in 32 bits and
// the maximum is taken modulo the counter width).
__device__ __forceinline__ u64 group_max_head(u32 mask, u64 head) {
    const u32 leader = __ffs(mask) - 1;
    const u64 lead = __shfl_sync(mask, head, leader);
    const int off = __reduce_max_sync(mask, (int)(i64)(head - lead));
    return lead + (u64)(i64)off;
}

// Tail catch-up by the group: one atomic maximum to the largest head of the
// group (returning, so it is performed before the group goes on).
template <bool CNT = false>
__device__ __forceinline__ void ring_catchup_group(const gq_ring_view& r, u64 head) {
    const u32 mask = group_of(r.tail);
    const u64 target = group_max_head(mask, head);
    if (lane_id() == __ffs(mask) - 1) {
        oc_add<CNT>(kOcCatch);
        const u64 old = atomicMax(reinterpret_cast<unsigned long long*>(r.tail), target);
        asm volatile("" ::"l"(old));
    }
    __syncwarp(mask);
}

// Due install (GPU-first): a dequeuer whose slot still holds an older cycle's
// empty entry while Tail is past its ticket has a partner enqueuer that took
// that ticket and will install there shortly.  Ruling the slot out at once
// (Algorithm 1 TryDeq) sends both of them round for new tickets, and in
// near-empty or near-full rings those retries feed each other (the partners of
// the next tickets are overtaken in turn).  So the dequeuer first re-reads the
// slot a bounded number of times, `due_wait` polls about 32 ns apart; after
// that it proceeds exactly as TryDeq does with what it read last.  Waiting
// changes no step of the protocol, only when the dequeuer takes it.  A Tail
// moved by a catch-up (no partner) costs the wait and nothing else.  Off by
// default (gq_options.due_wait): on the benchmark workloads it measured no
// better than ruling the slot out at once; the batched form can tune it.
template <bool CNT, class StillEmpty>
__device__ __forceinline__ u64 wait_due_install(u64* slot, u64 e, u32 polls, StillEmpty still_empty) {
    for (u32 w = 0; w < polls && still_empty(e); ++w) {
        __nanosleep(32);
        oc_add<CNT>(kOcSpin);
        e = ld_acq(slot);
    }
    return e;
}

// Inner-ring enqueue of index `idx` (TryEnq of Algorithm 1, retried until it
// succeeds).  Returns GQ_OK, or GQ_ERR_TIMEOUT if the retry bound expires.
// tk (nullable, test recorder): receives the ticket the index was installed at.
template <bool MATCH, bool CNT = false>
__device__ int lfq_ring_enq(const gq_dev& q, const gq_ring_view& r, u32 idx, u64* tk = nullptr) {
    for (u32 it = 0; it < kRetryLimit; ++it) {
        const u64 t = warp_faa<MATCH, CNT>(r.tail, 1, q.batch_width);
        u64* slot = r.slots + (t & q.slot_mask);
        const u64 c = (t >> q.ring_order) & q.cycle_mask;
        const u64 ne = lfq_entry(c, kSafe, idx);
        u64 e = lfq_entry((c - 1) & q.cycle_mask, kSafe, kBot);    // predicted current value
        bool done = cas(slot, e, ne);
        oc_cas<CNT>(done);
        for (; !done && it < kRetryLimit; ++it) {
            if (!cyc_older(lfq_cycle(e), c, q) || lfq_index(e) < kBotC) break;
            if (!(e & kSafe)) {
                // an unsafe slot may be reused only if no dequeuer has passed t
                if ((i64)(ld_rlx(r.head) - t) > 0) break;
            }
            done = cas(slot, e, ne);
            oc_cas<CNT>(done);
            // CAS lost: e holds the current entry; re-evaluate the same ticket
        }
        if (done) {
            thr_reset_group<CNT>(r.threshold, q.thr_reset, q.err);
            if (tk) *tk = t;
            return GQ_OK;
        }
        oc_add<CNT>(kOcBurn);
        if (q.backoff_ns) __nanosleep(q.backoff_ns);
    }
    latch_error(q.err, GQ_ERR_TIMEOUT);
    return GQ_ERR_TIMEOUT;
}

// Inner-ring dequeue (TryDeq of Algorithm 1, retried while it returns RETRY).
// Returns GQ_OK with *idx, GQ_EMPTY, or GQ_ERR_TIMEOUT.  tk (nullable): the
// ticket the index was taken at.
template <bool MATCH, bool CNT = false>
__device__ int lfq_ring_deq(const gq_dev& q, const gq_ring_view& r, u32* idx, u64* tk = nullptr) {
    if (ld_rlx(r.threshold) < 0) return GQ_EMPTY;
    for (u32 it = 0; it < kRetryLimit; ++it) {
        const u64 h = warp_faa<MATCH, CNT>(r.head, 1, q.batch_width);
        u64* slot = r.slots + (h & q.slot_mask);
        const u64 c = (h >> q.ring_order) & q.cycle_mask;
        u64 e = ld_acq(slot);
        oc_add<CNT>(kOcLoad);
        auto empty_older = [&](u64 x) { return lfq_index(x) >= kBotC && cyc_older(lfq_cycle(x), c, q); };
        if (q.due_wait && empty_older(e) && (i64)(ld_rlx(r.tail) - h) > 0)
            e = wait_due_install<CNT>(slot, e, q.due_wait, empty_older);
        for (; it < kRetryLimit; ++it) {
            const u64 ec = lfq_cycle(e);
            if (ec == c) {
                if (lfq_index(e) < kBotC) {          // Consume and return the index
                    *idx = lfq_index(e);
                    if (tk) *tk = h;
                    // relaxed: the acquire load of e already ordered the payload
                    // read; the release CAS that hands the index on orders the OR
                    red_or_rlx(slot, kBot);
                    oc_add<CNT>(kOcRmw);
                    return GQ_OK;
                }
                break;
            }
            if (!cyc_older(ec, c, q)) break;         // slot already belongs to a later cycle
            // empty class: advance the slot to cycle c (still empty);
            // occupied by an older cycle: clear Safe so the enqueuer of t = h
            // does not reuse it once Head has passed h.
            const u64 ne = (lfq_index(e) >= kBotC) ? lfq_entry(c, e & kSafe, kBot) : (e & ~kSafe);
            const bool ok = cas(slot, e, ne);
            oc_cas<CNT>(ok);
            if (ok) break;
        }
        oc_add<CNT>(kOcBurn);
        const u64 tl = ld_rlx(r.tail);
        if ((i64)(tl - (h + 1)) <= 0) {
            ring_catchup_group<CNT>(r, h + 1);
            thr_dec_group<CNT>(r.threshold);
            return GQ_EMPTY;
        }
        if (thr_dec_group<CNT>(r.threshold) <= 0) return GQ_EMPTY;
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
template <class T, bool MATCH, bool CNT = false>
__device__ int lfq_enqueue(const gq_dev& q, T v, u64* tk = nullptr) {
    u32 i;
    int s = lfq_ring_deq<MATCH, CNT>(q, q.fq, &i);
    if (s == GQ_EMPTY) return GQ_FULL;
    if (s != GQ_OK) return s;
    if (i >= q.capacity) {                            // never expected: a corrupt ring entry
        latch_error(q.err, GQ_ERR_INVALID);
        return GQ_ERR_INVALID;
    }
    data_store<T>(q, i, v);                           // ordered before the release CAS in aq
    return lfq_ring_enq<MATCH, CNT>(q, q.aq, i, tk);
}

template <class T, bool MATCH, bool CNT = false>
__device__ int lfq_dequeue(const gq_dev& q, T* v, u64* tk = nullptr) {
    u32 i;
    int s = lfq_ring_deq<MATCH, CNT>(q, q.aq, &i, tk);
    if (s != GQ_OK) return s;
    if (i >= q.capacity) {                            // never expected: a corrupt ring entry
        latch_error(q.err, GQ_ERR_INVALID);
        return GQ_ERR_INVALID;
    }
    *v = data_load<T>(q, i);                          // after the acquire on the aq slot
    s = lfq_ring_enq<MATCH, CNT>(q, q.fq, i);         // release: the read precedes reuse
    return s == GQ_OK ? GQ_OK : s;
}

// Enqueue (enq = true, payload *v) or dequeue (enq = false, result in *v) on
// one code path.  Both are "take an index from one ring, move the payload,
// give the index to the other ring": enqueue takes from fq and gives to aq,
// dequeue the reverse.  Selecting the rings per lane lets a warp whose lanes
// mix enqueues and dequeues run them together instead of one after the other
// (divergent branches); WaveFAA groups the lanes by counter address.  Each
// lane performs exactly the steps of its own operation.
template <class T, bool CNT = false>
__device__ int lfq_op(const gq_dev& q, bool enq, T* v, u64* tk = nullptr) {
    const gq_ring_view& from = enq ? q.fq : q.aq;
    const gq_ring_view& to = enq ? q.aq : q.fq;
    u32 i;
    int s = lfq_ring_deq<true, CNT>(q, from, &i, enq ? nullptr : tk);
    if (s == GQ_EMPTY) return enq ? GQ_FULL : GQ_EMPTY;
    if (s != GQ_OK) return s;
    if (i >= q.capacity) {                            // never expected: a corrupt ring entry
        latch_error(q.err, GQ_ERR_INVALID);
        return GQ_ERR_INVALID;
    }
    if (enq) data_store<T>(q, i, *v);                 // ordered before the release CAS in aq
    else *v = data_load<T>(q, i);                     // after the acquire on the aq slot
    return lfq_ring_enq<true, CNT>(q, to, i, enq ? tk : nullptr);
}

}  // namespace gqd
