// G-WFQ-YMC: Yang and Mellor-Crummey's wait-free queue on a pre-allocated
// cell pool (Section III-A).
//
// The queue is an infinite array of cells indexed by tickets from two
// fetch-and-add counters, T (enqueue) and H (dequeue).  Section III-A replaces
// the original's dynamically grown segment list and hazard-pointer reclamation
// with a device pool and direct arithmetic lookup: the pool holds `capacity`
// cells for tickets 1..capacity (segment s of SEG cells starts at s * SEG, so
// cell i is simply pool[i]); running past it latches GQ_ERR_POOL_EXHAUSTED.
// Cells are stored as three arrays (structure of arrays), one 64-bit word each:
//   val  payload, or VBOT (2^64 - 1, never written) / VTOP (2^64 - 2, unusable)
//   enq  0 = no request, 1 = unusable, else (id << 24) | (r + 1): the enqueue
//        request of thread r whose id (first failed cell) is id
//   deq  0 = unclaimed, 1 = taken by a fast dequeue, r + 2 = dequeue request of r
// Each thread owns a record (its "handle"): an enqueue request <id, val>, a
// dequeue request <id, idx>, and the private helping cursors.
//
// Fast paths (at most patience + 1 attempts):
//   enqueue: t = FAA(T); CAS val[t] VBOT -> v.
//   dequeue: h = FAA(H); help_enq(h) settles the cell (value, unusable, or
//            EMPTY when T <= h); a value is taken by CAS deq[h] 0 -> 1.
// Slow paths publish the request in the record and are completed by helpers:
//   enqueue: the owner keeps taking tickets and offering its request to cells
//            (CAS enq[i] 0 -> (id << 24) | (r + 1)); a dequeuer that finds an
//            unusable cell with a request attached claims that cell for the
//            request (CAS id -> -i) and commits the value there.  Dequeuers also attach pending peer
//            requests to cells they find empty (round-robin over peers).
//   dequeue: helpers scan cells after the request's id for a candidate (a
//            value not yet taken, or an EMPTY decision), announce it in idx and
//            claim it with CAS deq[i] 0 -> r+2; idx = -i marks completion.
//            The dequeue that took a cell whose index is a multiple of 64
//            inspects one peer's dequeue request: peer (cell / 64) mod k.
// Warp-batched tickets (WaveFAA) serve the fast paths; the ticket order is the
// same as with per-thread fetch-and-add (Lemma "WaveFAA preserves ticket order").
//
// Difference from the CPU original: a cell's enqueue-request reference names
// the request instance (thread and request id), not just the thread's handle.
// Once that instance has been satisfied in another cell, the reference is
// dead: no later request of the same thread can be claimed through this cell.
// That makes an EMPTY decision at a cell final (its value word stays VTOP);
// with a bare handle reference, a later request whose first failed cell lies
// at or below this one (its ticket taken before T passed the cell) could still
// commit a value here after a dequeuer had already answered EMPTY at it.
#pragma once

#include "gq_atomics.cuh"

namespace gqd {

constexpr u64 kVBot = ~0ull;
constexpr u64 kVTop = ~0ull - 1;
constexpr u64 kRefBot = 0, kRefTop = 1;
constexpr u32 kYHelpDelay = 64;   // dequeue tickets per peer inspection
constexpr u32 kYSpin = 16;      // back-to-back reads of an empty cell (its enqueuer may be on its way)
constexpr u32 kYWaitPolls = 256; // then, if T shows the ticket taken, polls 64 ns apart
// Cells one helper may visit in a dequeue request's candidate search.  Every
// step moves to the next cell, so the search always progresses; it can be long
// when the request's cell lies far below T (cells below T hold claimed values
// or were marked unusable while T passed them: 2^12 threads, 90 % consumers,
// patience 0 scanned more than 2^16 cells).  The bound only stops a search that
// has run through millions of cells.
constexpr u32 kYScanLimit = 1u << 22;
// Cells ahead of its own ticket that a fast enqueue asks L2 to prefetch.  The
// pool is touched once per ticket and is far larger than L2, so a cell's first
// access (the enqueue's CAS, or an early dequeuer's read) would otherwise miss
// to DRAM on the operation's dependent chain; T reaches ticket i + kYPrefetch
// a few microseconds later, by which time the line is in L2.
constexpr u64 kYPrefetch = 1ull << 15;

enum : int {
    kYErId = 0,    // enqueue request: > 0 pending from cell id on, < 0 done at cell -id
    kYErVal = 1,
    kYDrId = 2,    // dequeue request: first cell
    kYDrIdx = 3,   // > 0 announced candidate cell, < 0 done at cell -idx
    kYEh = 4,      // private: enqueue-help peer
    kYEi = 5,      // private: id of the peer request being helped
    kYWords = 16
};



__device__ __forceinline__ u64* yrec(const gq_dev& q, u32 r) { return q.ymc_rec + (u64)r * kYWords; }
__device__ __forceinline__ u64 ytag(u64 id, u32 r) { return (id << 24) | (u64)(r + 1); }
__device__ __forceinline__ u32 ytag_thread(u64 e) { return (u32)(e & ((1u << 24) - 1)) - 1; }
__device__ __forceinline__ i64 ytag_id(u64 e) { return (i64)(e >> 24); }
__device__ __forceinline__ i64 ld_i(u64* p) { return (i64)ld_acq(p); }

__device__ __forceinline__ bool ycell_ok(const gq_dev& q, u64 i) {
    if (i >= 1 && i <= q.capacity) return true;
    latch_error(q.err, GQ_ERR_POOL_EXHAUSTED);
    return false;
}

// Raise counter C to at least v + 1 (T or H), so that no later EMPTY decision
// is taken below a cell that holds a committed value.
__device__ __forceinline__ void ymc_advance(u64* C, u64 v) {
    u64 cur = ld_acq(C);
    for (u32 it = 0; it < kRetryLimit && cur <= v; ++it)
        if (cas(C, cur, v + 1)) return;
}

enum { kYValue = 0, kYUnusable = 1, kYEmpty = 2 };

// Cell i's value and dequeue reference sit side by side in one 16-byte pair
// (cell_val[2i], cell_deq[2i] = cell_val[2i + 1]): the dequeue that reads the
// value and then claims the cell touches one L2 sector, already brought in by
// the enqueue's CAS, instead of a second line in a second array.
__device__ __forceinline__ u64* yval(const gq_dev& q, u64 i) { return q.cell_val + 2 * i; }
__device__ __forceinline__ u64* ydeq(const gq_dev& q, u64 i) { return q.cell_deq + 2 * i; }

// help_enq: settles cell i for the dequeuer `me` and returns kYValue with *v,
// kYUnusable (try another cell), or kYEmpty (T <= i: no enqueue reached i).
template <bool CNT = false>
static __device__ __noinline__ int ymc_help_enq(const gq_dev& q, u32 me, u64 i, u64* v) {
    u64* cv = yval(q, i);
    u64* ce = q.cell_enq + i;
    u64 x = ld_acq(cv);
    oc_add<CNT>(kOcLoad);
    for (u32 s = 0; s < kYSpin && x == kVBot; ++s) {   // an enqueuer may be on its way
        oc_add<CNT>(kOcSpin);
        x = ld_acq(cv);
    }
    if (x == kVBot && ld_acq(q.ymc_tail) > i) {
        // T > i: the enqueuer holding ticket i has taken it and its write is
        // due.  Marking the cell unusable now would send that enqueuer round
        // again, and under load such retries feed on themselves (H runs ahead
        // of T, more cells are found empty, more enqueuers retry).  Wait
        // longer for the write, boundedly.
        for (u32 s = 0; s < kYWaitPolls && x == kVBot; ++s) {
            oc_add<CNT>(kOcSpin);
            __nanosleep(64);
            x = ld_acq(cv);
        }
    }
    if (x == kVBot) {
        const bool ok = cas(cv, x, kVTop);
        oc_cas<CNT>(ok);
        if (ok) oc_add<CNT>(kOcMark);
        if (!ok && x != kVTop) { *v = x; return kYValue; }
        x = kVTop;
    } else if (x != kVTop) {
        *v = x;
        return kYValue;
    }
    // the cell is unusable for fast enqueues: offer it to a pending slow enqueue
    u64 e = ld_acq(ce);
    if (e == kRefBot) {
        u64* mine = yrec(q, me);
        u32 p = (u32)mine[kYEh];                   // private cursors: plain access
        i64 s = ld_i(yrec(q, p) + kYErId);
        if (mine[kYEi] != 0 && (i64)mine[kYEi] != s) {
            mine[kYEi] = 0;
            p = (p + 1) % q.max_threads;
            mine[kYEh] = p;
            s = ld_i(yrec(q, p) + kYErId);
        }
        u64 want = kRefBot;
        if (s > 0 && (u64)s <= i && !cas(ce, want, ytag((u64)s, p)) && want != ytag((u64)s, p)) {
            mine[kYEi] = (u64)s;                   // keep helping this request
        } else {
            mine[kYEi] = 0;
            mine[kYEh] = (p + 1) % q.max_threads;
        }
        e = ld_acq(ce);
        if (e == kRefBot) {
            u64 b = kRefBot;
            if (cas(ce, b, kRefTop)) e = kRefTop; else e = b;
        }
    }
    if (e == kRefTop) return (ld_acq(q.ymc_tail) <= i) ? kYEmpty : kYUnusable;
    // the cell names request instance (id_e of thread r)
    u64* er = yrec(q, ytag_thread(e));
    const i64 id_e = ytag_id(e);
    i64 ei = ld_i(er + kYErId);
    const u64 ev = ld_acq(er + kYErVal);
    bool claimed = false;
    if (ei == id_e) {
        u64 cur = (u64)ei;
        if (cas(er + kYErId, cur, (u64)(-(i64)i))) claimed = true;
        else ei = (i64)cur;
    }
    if (claimed || (ei == -(i64)i && ld_acq(cv) == kVTop)) {
        ymc_advance(q.ymc_tail, i);
        st_rel(cv, ev);                            // commit the request's value in cell i
    } else if (ei != -(i64)i) {
        // the instance was satisfied elsewhere: this cell stays unusable for good
        if (ld_acq(cv) == kVTop && ld_acq(q.ymc_tail) <= i) return kYEmpty;
    }
    x = ld_acq(cv);
    if (x == kVTop) return kYUnusable;
    *v = x;
    return kYValue;
}

// Slow enqueue of v by thread me whose fast path last failed at cell id.
// tk (nullable, test recorder): the cell the value was committed in.
static __device__ __noinline__ int ymc_enq_slow(const gq_dev& q, u32 me, u64 v, u64 id, u64* tk) {
    u64* er = yrec(q, me);
    // release: a helper that reads this value must also see the commit of this
    // thread's previous request (its cell value), see ymc_help_enq
    st_rel(er + kYErVal, v);
    st_rel(er + kYErId, id);
    u64 i = id;
    for (u32 it = 0; it < kRetryLimit && ld_i(er + kYErId) > 0; ++it) {
        i = faa_rlx(q.ymc_tail, 1);
        if (!ycell_ok(q, i)) {
            // withdraw the request unless a helper has already claimed a cell
            u64 cur = id;
            if (cas(er + kYErId, cur, 0)) return GQ_ERR_POOL_EXHAUSTED;
            break;
        }
        u64 b = kRefBot;
        if (cas(q.cell_enq + i, b, ytag(id, me)) && ld_acq(yval(q, i)) != kVTop) {
            u64 cur = id;
            cas(er + kYErId, cur, (u64)(-(i64)i));   // claim cell i (a helper may have claimed another)
            break;
        }
    }
    const i64 done = ld_i(er + kYErId);
    if (done >= 0) {
        latch_error(q.err, GQ_ERR_TIMEOUT);
        return GQ_ERR_TIMEOUT;
    }
    const u64 c = (u64)(-done);
    ymc_advance(q.ymc_tail, c);
    st_rel(yval(q, c), v);
    if (tk) *tk = c;
    return GQ_OK;
}

// Helps the dequeue request of thread p (called by me).
static __device__ __noinline__ void ymc_help_deq(const gq_dev& q, u32 me, u32 p) {
    u64* dr = yrec(q, p);
    i64 idx = ld_i(dr + kYDrIdx);
    const i64 id = ld_i(dr + kYDrId);
    if (id <= 0 || idx < id) return;
    i64 i = id, cand = 0, old = idx;
    for (u32 it = 0; it < kRetryLimit; ++it) {
        // find a candidate cell, unless one gets announced meanwhile
        u32 jt = 0;
        for (; jt < kYScanLimit && idx == old && cand == 0; ++jt) {
            ++i;
            if (!ycell_ok(q, (u64)i)) {
                red_max_rlx(q.ymc_hw, (u64)(i - 1));
                return;
            }
            u64 v;
            const int s = ymc_help_enq(q, me, (u64)i, &v);
            if (s == kYEmpty || (s == kYValue && ld_acq(ydeq(q, i)) == kRefBot)) cand = i;
            else idx = ld_i(dr + kYDrIdx);
        }
        // The search may have settled cells above T and H (marked them
        // unusable, attached requests): the reset must clear them too.
        if (jt) red_max_rlx(q.ymc_hw, (u64)i);
        if (jt == kYScanLimit) break;   // never claim the request's own first cell unannounced
        if (cand != 0) {
            u64 cur = (u64)idx;
            if (cas(dr + kYDrIdx, cur, (u64)cand)) idx = cand;
            else idx = (i64)cur;
            if (idx >= cand) cand = 0;
        }
        if (idx < 0 || ld_i(dr + kYDrId) != id) return;    // completed
        u64 b = kRefBot;
        if (ld_acq(yval(q, idx)) == kVTop || cas(ydeq(q, idx), b, (u64)p + 2) || b == (u64)p + 2) {
            u64 cur = (u64)idx;
            cas(dr + kYDrIdx, cur, (u64)(-idx));
            return;
        }
        old = idx;
        if (idx >= i) i = idx;
    }
    latch_error(q.err, GQ_ERR_TIMEOUT);
}


// tk (nullable, test recorder): the cell of the operation (an item's enqueue
// and its dequeue share it).
template <class T, bool MATCH, bool CNT = false>
__device__ int ymc_enqueue(const gq_dev& q, T v, u32 tid, u64* tk = nullptr) {
    if (tid >= q.max_threads) {
        latch_error(q.err, GQ_ERR_TOO_MANY_THREADS);
        return GQ_ERR_TOO_MANY_THREADS;
    }
    const u64 x = (u64)v;
    if (x >= kVTop) return GQ_ERR_RESERVED_VALUE;
    u64 id = 0;
    for (u32 p = 0; p <= q.patience_enq; ++p) {
        const u64 i = warp_faa<MATCH, CNT>(q.ymc_tail, 1, q.batch_width);
        if (!ycell_ok(q, i)) return GQ_ERR_POOL_EXHAUSTED;
        if (i + kYPrefetch <= q.capacity)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(yval(q, i + kYPrefetch)));
        u64 b = kVBot;
        const bool ok = aref<u64>(*yval(q, i)).compare_exchange_strong(b, x, kRel, kRlx);
        oc_cas<CNT>(ok);
        if (ok) {
            if (tk) *tk = i;
            return GQ_OK;
        }
        oc_add<CNT>(kOcBurn);
        id = i;
        if (q.backoff_ns) __nanosleep(q.backoff_ns);
    }
    oc_add<CNT>(kOcSlow);
    return ymc_enq_slow(q, tid, x, id, tk);
}

template <class T, bool MATCH, bool CNT = false>
__device__ int ymc_dequeue(const gq_dev& q, T* out, u32 tid, u64* tk = nullptr) {
    if (tid >= q.max_threads) {
        latch_error(q.err, GQ_ERR_TOO_MANY_THREADS);
        return GQ_ERR_TOO_MANY_THREADS;
    }
    u64 id = 0, v = 0, help_ticket = 0;
    int res = kYUnusable;
    for (u32 p = 0; p <= q.patience_deq && res == kYUnusable; ++p) {
        const u64 i = warp_faa<MATCH, CNT>(q.ymc_head, 1, q.batch_width);
        if (!ycell_ok(q, i)) return GQ_ERR_POOL_EXHAUSTED;
        if ((i & (kYHelpDelay - 1)) == 0) help_ticket = i;
        res = ymc_help_enq<CNT>(q, tid, i, &v);
        if (res == kYValue) {
            u64 b = kRefBot;
            const bool ok = cas(ydeq(q, i), b, kRefTop);
            oc_cas<CNT>(ok);
            if (!ok) res = kYUnusable;   // a slow dequeue took it
        }
        if (res != kYValue) oc_add<CNT>(kOcBurn);
        id = i;
        if (res == kYUnusable && q.backoff_ns) __nanosleep(q.backoff_ns);
    }
    if (res == kYUnusable) {
        oc_add<CNT>(kOcSlow);
        // slow path: publish <id, idx = id> and help it to completion
        u64* dr = yrec(q, tid);
        st_rel(dr + kYDrId, id);
        st_rel(dr + kYDrIdx, id);
        ymc_help_deq(q, tid, tid);
        const i64 idx = ld_i(dr + kYDrIdx);
        if (idx >= 0) {
            latch_error(q.err, GQ_ERR_TIMEOUT);
            return GQ_ERR_TIMEOUT;
        }
        const u64 c = (u64)(-idx);
        ymc_advance(q.ymc_head, c);
        v = ld_acq(yval(q, c));
        res = (v == kVTop) ? kYEmpty : kYValue;
        id = c;
    }
    // Help delay by ticket: the dequeue that took a cell whose index is a
    // multiple of kYHelpDelay (whatever it returns) inspects the dequeue request
    // of peer (cell / kYHelpDelay) mod k.  Every cell index is taken by exactly
    // one dequeue attempt, so each peer is inspected once in every
    // kYHelpDelay * k dequeue tickets: the bound of a per-thread countdown
    // (k threads, one inspection per D dequeues each), without the per-thread
    // countdown's load and store on every dequeue, which the release and
    // acq_rel atomics of the next operations had to wait for.  (The CPU
    // original helps after every dequeue.)
    if (help_ticket) {
        const u32 peer = (u32)((help_ticket / kYHelpDelay) % q.max_threads);
        if (peer != tid) ymc_help_deq(q, tid, peer);
    }
    if (res == kYEmpty) return GQ_EMPTY;
    if (tk) *tk = id;
    *out = (T)v;
    return GQ_OK;
}

}  // namespace gqd
