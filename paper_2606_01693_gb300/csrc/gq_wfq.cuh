// G-WFQ: bounded wait-free ring (Section III-C, Algorithm 2).
//
// Same bounded 2n-slot ring and index-indirection layer as G-LFQ; the fast
// path is G-LFQ's (Algorithm 1) and runs at most `patience` times.  After that
// the operation publishes a request in its fixed per-thread record and every
// thread that sees the request (the owner itself, and peers that inspect one
// record every D operations) runs the same cooperative slow path until the
// request's FIN bit is set.  Every shared word is updated by one 64-bit atomic
// (Lemma "Single-word shared-state atomicity"):
//
//   slot   <Note 19 | Cycle 19 | Safe 1 | Enq 1 | Index 24>
//   Global Head / Tail  <Counter 43 | ThrIdx 21>   ThrIdx 0 = NULL, else helper h + 1
//   Local  head / tail  <Counter 62 | INC 1 | FIN 1>  (Counter holds a 43-bit ticket)
//   phase-2 word of helper h, one per side   <request record r + 1 (21) | Counter 43>
//
// SlowFAA (Algorithm 2) gives all helpers of request r one agreed sequence of
// tickets, each reserved by exactly one CAS on Global <c, NULL> -> <c + 1, h>
// (Lemma "One cooperative increment per round"): a helper first proposes c in
// r's local word with INC set, publishes its phase-2 word (r, c), then CASes
// Global.  Whoever later reads ThrIdx = h completes the phase-2 step: clears
// INC on r's local word (the ticket is now r's) and then clears ThrIdx.
//
// TryEnqSlow installs the entry with Enq = 0; the request finishes when FIN is
// set on its local tail at the installed ticket; the Enq bit then goes to 1.
// A dequeuer that meets an Enq = 0 entry of its own cycle finishes that
// request first (FIN, then Enq = 1) and only then consumes it, so an entry is
// never consumed while helpers could still move its request to a new ticket.
// A slow helper that finds an old-cycle slot unusable for the request's ticket
// advances Note to the ticket's cycle before giving up on it, so a delayed
// helper of the same request can never install at that ticket later (Lemma
// "Stale-slot exclusion").  A slow dequeue only locates the outcome (the
// ticket whose slot holds an item, or an EMPTY decision) and sets FIN there;
// the owner consumes the item, so exactly one consume happens.
//
// Helpers accept a request only if its published sequence fields match
// (seq2 == seq1 with the pending bit set, Section III-C "GPU publication
// discipline") and stop as soon as the owner's seq1 moves on.
#pragma once

#include "gq_lfq.cuh"

namespace gqd {

// ---- word layouts --------------------------------------------------------
constexpr int kWNoteShift = 45, kWCycShift = 26;
constexpr u64 kWSafe = 1ull << 25, kWEnq = 1ull << 24;
constexpr u32 kWIdxMask = (1u << 24) - 1;
constexpr u32 kWBot = kWIdxMask, kWBotC = kWIdxMask - 1;
constexpr u64 kWFieldMask = (1ull << 19) - 1;

__host__ __device__ __forceinline__ u64 wfq_entry(u64 note, u64 cyc, u64 safe, u64 enq, u32 idx) {
    return (note << kWNoteShift) | (cyc << kWCycShift) | (safe ? kWSafe : 0) | (enq ? kWEnq : 0) | idx;
}
__device__ __forceinline__ u64 w_note(u64 e) { return (e >> kWNoteShift) & kWFieldMask; }
__device__ __forceinline__ u64 w_cyc(u64 e) { return (e >> kWCycShift) & kWFieldMask; }
__device__ __forceinline__ u32 w_idx(u64 e) { return (u32)e & kWIdxMask; }
__device__ __forceinline__ u64 w_set_note(u64 e, u64 note) {
    return (e & ~(kWFieldMask << kWNoteShift)) | (note << kWNoteShift);
}

constexpr int kGThrBits = 21;
constexpr u64 kGThrMask = (1ull << kGThrBits) - 1;
constexpr u64 kGOne = 1ull << kGThrBits;
constexpr u64 kCntMask = (1ull << 43) - 1;
__host__ __device__ __forceinline__ u64 wfq_global(u64 cnt, u64 thr) { return (cnt << kGThrBits) | thr; }
__device__ __forceinline__ u64 g_cnt(u64 g) { return g >> kGThrBits; }
__device__ __forceinline__ u64 g_thr(u64 g) { return g & kGThrMask; }

constexpr u64 kLInc = 2, kLFin = 1;
__device__ __forceinline__ u64 l_cnt(u64 l) { return (l >> 2) & kCntMask; }

// 43-bit modular ticket order (sound while live tickets are within 2^42)
__device__ __forceinline__ bool cnt_lt(u64 a, u64 b) {
    const u64 d = (b - a) & kCntMask;
    return d != 0 && d < (1ull << 42);
}
__device__ __forceinline__ bool cnt_le(u64 a, u64 b) { return a == b || cnt_lt(a, b); }

// ---- per-thread record (128 bytes) ----------------------------------------
enum : int {
    kRSeq1 = 0,      // owner: number of finished slow requests
    kRSeq2 = 1,      // published request sequence
    kRPending = 2,   // bit0 pending, bit1 enqueue
    kRInit = 3,      // initial ticket
    kRLocalTail = 4, // <Counter, INC, FIN> of an enqueue request
    kRLocalHead = 5, // <Counter, INC, FIN> of a dequeue request
    kRIndex = 6,     // payload index of an enqueue request
    kRP2Tail = 7,    // this thread's phase-2 word as a helper on Tail
    kRP2Head = 8,    // ... on Head
    kRWords = 16
    // the owner-only help cursor lives in a separate compact array (helpc),
    // so that the per-operation countdown of a warp touches one line
};

// Retry budgets of the cooperative slow path.  Its CAS on the Global word
// loses to every other helper's winning CAS and to fast-path fetch-adds; those
// losses are progress by others, so they do not count as stalls.  Only
// iterations that find the Global word unchanged since the previous one count
// against kSlowStall, and any change resets it (no thread made progress:
// a livelock); kSlowHard caps the
// total iterations of one request by one helper.  Reaching either latches
// GQ_ERR_TIMEOUT.
constexpr u32 kSlowStall = 1u << 16;
constexpr u32 kSlowHard = 1u << 24;

// Rare-path event counters kept in the queue's scratch line: requests
// published, peer requests helped, lost CASes on a Global word, successful
// SlowFAA rounds per side (each advances Counter by exactly one), and the most
// SlowFAA iterations one helper spent on one request.
enum {
    kStatSlowRequests = 1, kStatHelps = 2, kStatGlobalCasFail = 3,
    kStatSlowRoundsTail = 4, kStatSlowRoundsHead = 5, kStatMaxHelpIters = 6
};



// newest of two notes (modular); used to keep Note within one cycle of the slot
__device__ __forceinline__ u64 note_fresh(u64 note, u64 c, const gq_dev& q) {
    const u64 cm1 = (c - 1) & q.cycle_mask;
    return cyc_older(note, cm1, q) ? cm1 : note;
}

__device__ __forceinline__ u64* rec_of(const gq_ring_view& r, u32 id) { return r.rec + (u64)id * kRWords; }

// ---- phase 2 (Algorithm 2: "help the phase-2 request named by u") ----------
// g names helper h; h's phase-2 word (r, c) belongs to the instance named by g
// only if c < Counter(g) (a newer instance of h has c >= Counter(g)).
__device__ __forceinline__ void help_phase2(const gq_ring_view& R, int side, u64* G, u64 g) {
    const u32 h = (u32)g_thr(g) - 1;
    const u64 p = ld_acq(rec_of(R, h) + (side ? kRP2Head : kRP2Tail));
    const u64 rr = p >> 43;
    const u64 c = p & kCntMask;
    if (rr != 0 && cnt_lt(c, g_cnt(g))) {
        u64 want = (c << 2) | kLInc;
        cas(rec_of(R, (u32)rr - 1) + (side ? kRLocalHead : kRLocalTail), want, c << 2);
    }
    u64 gg = g;
    cas(G, gg, g & ~kGThrMask);
}

// Request validity: the owner's seq1 has not moved past `seq`.
__device__ __forceinline__ bool req_live(const gq_ring_view& R, u32 r, u64 seq) {
    return ld_acq(rec_of(R, r) + kRSeq1) == seq;
}

// SlowFAA (Algorithm 2).  Obtains the next ticket of request r (owner's
// sequence `seq`) on `side` (0 tail, 1 head).  *v: the last ticket this helper
// tried for r; on true it holds the new ticket.  Returns false when the request
// is finished (FIN) or no longer live.
// A helper whose CAS on the Global word lost sleeps before its next try, from
// kSlowNapMin ns doubling up to kSlowNapMax: with thousands of requests on
// the slow path at once (a ring far smaller than the number of threads) the
// helpers otherwise hammer one word that only one of them can win per round.
// Lost CASes are counted locally and added to the statistics line once per
// call, not once each (that line is one more hot word).
constexpr u32 kSlowNapMin = 64, kSlowNapMax = 8192;

static __device__ __noinline__ bool slow_faa(const gq_ring_view& R, int side, u32 r, u64 seq, u32 me, u64* v, i64* thld,
                         const gq_dev& q, u32* budget) {
    u64* G = side ? R.head : R.tail;
    u64* L = rec_of(R, r) + (side ? kRLocalHead : kRLocalTail);
    u64* P2 = rec_of(R, me) + (side ? kRP2Head : kRP2Tail);
    u64 last = ~0ull;
    u32 stall = 0, lost = 0, nap = 0;
    auto flush = [&]() {
        if (lost && q.scratch) atomicAdd(q.scratch + kStatGlobalCasFail, (unsigned long long)lost);
    };
    while (*budget && stall < kSlowStall) {
        --*budget;
        const u64 g = ld_acq(G);
        stall = (g == last) ? stall + 1 : 0;
        last = g;
        if (g_thr(g) != 0) {
            help_phase2(R, side, G, g);
            continue;
        }
        u64 l = ld_acq(L);
        if ((l & kLFin) || !req_live(R, r, seq)) {
            flush();
            return false;
        }
        const u64 c = g_cnt(g);
        u64 lc = l_cnt(l);
        if (!(l & kLInc)) {
            if (lc != *v) {               // another helper already moved r to a new ticket
                *v = lc;
                flush();
                return true;
            }
            const u64 prop = (c << 2) | kLInc;   // r's ticket *v failed: propose c
            if (!cas(L, l, prop)) continue;
            l = prop;
            lc = c;
        }
        if (lc != c) {
            // G was read with ThrIdx NULL before L: a proposal older than c was
            // never reserved (its reservation would have cleared INC first)
            if (cnt_lt(lc, c)) cas(L, l, (c << 2) | kLInc);
            continue;
        }
        st_rel(P2, ((u64)(r + 1) << 43) | c);
        u64 gg = g;
        if (cas(G, gg, wfq_global(c + 1, me + 1))) {
            if (q.scratch) atomicAdd(q.scratch + (side ? kStatSlowRoundsHead : kStatSlowRoundsTail), 1ull);
            if (thld) thr_dec(thld);
            u64 want = (c << 2) | kLInc;
            cas(L, want, c << 2);
            for (; *budget; --*budget) {              // clear ThrIdx if it is still ours
                u64 cur = ld_acq(G);
                if (g_thr(cur) != me + 1) break;
                if (cas(G, cur, cur & ~kGThrMask)) break;
            }
            *v = c;
            flush();
            return true;
        }
        ++lost;
        nap = nap ? (nap < kSlowNapMax ? 2 * nap : kSlowNapMax) : kSlowNapMin;
        __nanosleep(nap);
    }
    flush();
    latch_error(q.err, GQ_ERR_TIMEOUT);
    return false;
}

// Catch the Global Tail counter up to at least `head` (keeps ThrIdx).
__device__ __forceinline__ void wfq_catchup(const gq_ring_view& R, u64 head) {
    u64 g = ld_acq(R.tail);
    for (u32 it = 0; it < kRetryLimit; ++it) {
        if (cnt_le(head, g_cnt(g))) return;
        if (cas(R.tail, g, wfq_global(head, g_thr(g)))) return;
    }
}

// Catch-up by the converged lanes that catch up the same Tail word: the
// group's lowest lane raises it to the group's largest target (modulo 2^43),
// once, and the group goes on after that (see the group helpers of G-LFQ).
template <bool CNT = false>
__device__ __forceinline__ void wfq_catchup_group(const gq_ring_view& R, u64 head) {
    const u32 mask = group_of(R.tail);
    const u32 leader = __ffs(mask) - 1;
    const u64 lead = __shfl_sync(mask, head, leader);
    const int off = __reduce_max_sync(mask, (int)((i64)(((head - lead) & kCntMask) << 21) >> 21));
    if (lane_id() == leader) {
        oc_add<CNT>(kOcCatch);
        wfq_catchup(R, (lead + (u64)(i64)off) & kCntMask);
    }
    __syncwarp(mask);
}

// Finishes the slow enqueue that installed entry e (Enq = 0) at ticket t:
// FIN on its request at t (owner looked up by index), then Enq = 1.
static __device__ __noinline__ void wfq_finalize(const gq_ring_view& R, u64* slot, u64 e, u64 t, const gq_dev& q) {
    const u32 i = w_idx(e);
    if (i >= q.capacity) {
        latch_error(q.err, GQ_ERR_INVALID);
        return;
    }
    const u64 o = ld_acq(R.owner + i);
    if (o != 0 && o <= q.max_threads) {
        u64 want = t << 2;
        cas(rec_of(R, (u32)o - 1) + kRLocalTail, want, want | kLFin);
    }
    const u64 c = w_cyc(e);
    for (u32 it = 0; it < kRetryLimit; ++it) {
        if (w_cyc(e) != c || w_idx(e) != i || (e & kWEnq)) return;
        if (cas(slot, e, e | kWEnq)) return;
    }
}

// ---- fast path (Algorithm 1 on the G-WFQ entry) ----------------------------
enum { kTryOk = 0, kTryEmpty = 2, kTryRetry = 3 };

template <bool MATCH, bool CNT = false>
__device__ int wfq_try_enq(const gq_ring_view& R, const gq_dev& q, u32 idx, u64* t_out) {
    const u64 t = warp_faa<MATCH, CNT>(R.tail, kGOne, q.batch_width) >> kGThrBits & kCntMask;
    *t_out = t;
    u64* slot = R.slots + (t & q.slot_mask);
    const u64 c = (t >> q.ring_order) & q.cycle_mask;
    // predicted current value: consumed in the previous cycle, Note one older
    const u64 cm1 = (c - 1) & q.cycle_mask;
    u64 e = wfq_entry((c - 2) & q.cycle_mask, cm1, 1, 1, kWBot);
    bool done = cas(slot, e, wfq_entry(cm1, c, 1, 1, idx));
    oc_cas<CNT>(done);
    for (u32 it = 0; !done && it < kRetryLimit; ++it) {
        if (!cyc_older(w_cyc(e), c, q) || w_idx(e) < kWBotC) break;
        if (!(e & kWSafe) && !cnt_le(g_cnt(ld_rlx(R.head)), t)) break;
        done = cas(slot, e, wfq_entry(note_fresh(w_note(e), c, q), c, 1, 1, idx));
        oc_cas<CNT>(done);
    }
    if (!done) {
        oc_add<CNT>(kOcBurn);
        return kTryRetry;
    }
    thr_reset_group<CNT>(R.threshold, q.thr_reset, q.err);
    return kTryOk;
}

// Consumes the item of ticket h in `slot` (its cycle already checked).
// Consume: index field to BOT, other fields kept, by one atomic OR that
// returns nothing (while the slot holds the item only its consumer changes the
// index bits; helpers and finalisers CAS the other fields); e was read with
// acquire, so the consume can be relaxed.
template <bool CNT = false>
__device__ __forceinline__ u32 wfq_consume(const gq_ring_view& R, u64* slot, u64 e, u64 h, const gq_dev& q) {
    if (!(e & kWEnq)) {
        wfq_finalize(R, slot, e, h, q);
        e |= kWEnq;
    }
    const u32 i = w_idx(e);
    red_or_rlx(slot, kWIdxMask);
    oc_add<CNT>(kOcRmw);
    return i;
}

template <bool MATCH, bool CNT = false>
__device__ int wfq_try_deq(const gq_ring_view& R, const gq_dev& q, u32* idx, u64* h_out) {
    const u64 h = warp_faa<MATCH, CNT>(R.head, kGOne, q.batch_width) >> kGThrBits & kCntMask;
    *h_out = h;
    u64* slot = R.slots + (h & q.slot_mask);
    const u64 c = (h >> q.ring_order) & q.cycle_mask;
    u64 e = ld_acq(slot);
    oc_add<CNT>(kOcLoad);
    // due install (see wait_due_install): Tail's Counter past h
    auto empty_older = [&](u64 x) { return w_idx(x) >= kWBotC && cyc_older(w_cyc(x), c, q); };
    if (q.due_wait && empty_older(e) && cnt_lt(h, g_cnt(ld_rlx(R.tail))))
        e = wait_due_install<CNT>(slot, e, q.due_wait, empty_older);
    for (u32 it = 0; it < kRetryLimit; ++it) {
        const u64 ec = w_cyc(e);
        if (ec == c) {
            if (w_idx(e) < kWBotC) {
                *idx = wfq_consume<CNT>(R, slot, e, h, q);
                return kTryOk;
            }
            break;
        }
        if (!cyc_older(ec, c, q)) break;
        const u64 ne = (w_idx(e) >= kWBotC)
                           ? wfq_entry(note_fresh(w_note(e), c, q), c, e & kWSafe, 1, kWBot)
                           : (e & ~kWSafe);
        const bool ok = cas(slot, e, ne);
        oc_cas<CNT>(ok);
        if (ok) break;
        if (it + 1 == kRetryLimit) {
            latch_error(q.err, GQ_ERR_TIMEOUT);
            return kTryRetry;
        }
    }
    oc_add<CNT>(kOcBurn);
    const u64 tl = g_cnt(ld_rlx(R.tail));
    if (cnt_le(tl, h + 1)) {
        wfq_catchup_group<CNT>(R, h + 1);
        thr_dec_group<CNT>(R.threshold);
        return kTryEmpty;
    }
    if (thr_dec_group<CNT>(R.threshold) <= 0) return kTryEmpty;
    return kTryRetry;
}

// ---- slow path slot actions ------------------------------------------------
enum { kSlowDone = 0, kSlowNext = 1 };

// TryEnqSlow: install idx at ticket t (Enq = 0), or rule the slot out (Note).
static __device__ __noinline__ int wfq_try_enq_slow(const gq_ring_view& R, const gq_dev& q, u32 r, u64 t, u32 idx) {
    u64* slot = R.slots + (t & q.slot_mask);
    const u64 c = (t >> q.ring_order) & q.cycle_mask;
    u64 e = ld_acq(slot);
    for (u32 it = 0; it < kRetryLimit; ++it) {
        const u64 ec = w_cyc(e);
        if (ec == c) {
            // only r holds tail ticket t: an item of cycle c here is r's install
            if (w_idx(e) < kWBotC) {
                u64 want = t << 2;
                cas(rec_of(R, r) + kRLocalTail, want, want | kLFin);
                return kSlowDone;
            }
            return kSlowNext;
        }
        if (!cyc_older(ec, c, q) || !cyc_older(w_note(e), c, q)) return kSlowNext;
        const bool usable = (w_idx(e) >= kWBotC) && ((e & kWSafe) || cnt_le(g_cnt(ld_rlx(R.head)), t));
        if (usable) {
            if (cas(slot, e, wfq_entry(note_fresh(w_note(e), c, q), c, 1, 0, idx))) {
                if (ld_rlx(R.threshold) != q.thr_reset) thr_reset(R.threshold, q.thr_reset, q.err);
                u64 want = t << 2;
                cas(rec_of(R, r) + kRLocalTail, want, want | kLFin);
                return kSlowDone;
            }
        } else {
            if (cas(slot, e, w_set_note(e, c))) return kSlowNext;   // stale-slot exclusion
        }
    }
    return kSlowNext;
}

// TryDeqSlow: find the outcome of head ticket h for request r; FIN marks it.
static __device__ __noinline__ int wfq_try_deq_slow(const gq_ring_view& R, const gq_dev& q, u32 r, u64 h) {
    u64* slot = R.slots + (h & q.slot_mask);
    u64* L = rec_of(R, r) + kRLocalHead;
    const u64 c = (h >> q.ring_order) & q.cycle_mask;
    u64 e = ld_acq(slot);
    for (u32 it = 0; it < kRetryLimit; ++it) {
        const u64 ec = w_cyc(e);
        if (ec == c) {
            if (w_idx(e) < kWBotC) {            // the item of ticket h: the owner consumes it
                u64 want = h << 2;
                cas(L, want, want | kLFin);
                return kSlowDone;
            }
            break;                               // ruled out at cycle c already
        }
        if (!cyc_older(ec, c, q)) break;
        u64 ne;
        if (w_idx(e) >= kWBotC) {
            ne = wfq_entry(note_fresh(w_note(e), c, q), c, e & kWSafe, 1, kWBot);
        } else {
            ne = e & ~kWSafe;
            if (cyc_older(w_note(e), c, q)) ne = w_set_note(ne, c);
        }
        if (cas(slot, e, ne)) break;
        if (it + 1 == kRetryLimit) {
            latch_error(q.err, GQ_ERR_TIMEOUT);
            return kSlowNext;
        }
    }
    const u64 tl = g_cnt(ld_rlx(R.tail));
    if (cnt_le(tl, h + 1)) {
        wfq_catchup(R, h + 1);
        u64 want = h << 2;
        cas(L, want, want | kLFin);
        return kSlowDone;
    }
    if (ld_rlx(R.threshold) < 0) {
        u64 want = h << 2;
        cas(L, want, want | kLFin);
        return kSlowDone;
    }
    return kSlowNext;
}

// Runs request r (sequence seq) to completion as one of its helpers.  A slot
// action that reports DONE has tried to set FIN at its ticket; that CAS loses
// if another helper moved the request on first (for a dequeue, an EMPTY
// observation at one moment and a "not empty" one at another are both valid),
// so the loop always returns to SlowFAA, which stops only once FIN is set.
static __device__ __noinline__ void wfq_help_request(const gq_ring_view& R, const gq_dev& q, u32 r, u64 seq, bool enq,
                                                     u64 init, u32 idx, u32 me) {
    u64 v = init;
    const int side = enq ? 0 : 1;
    i64* thld = enq ? nullptr : R.threshold;
    u32 budget = kSlowHard;
    while (budget) {
        if (!slow_faa(R, side, r, seq, me, &v, thld, q, &budget)) break;
        if (enq) wfq_try_enq_slow(R, q, r, v, idx);
        else wfq_try_deq_slow(R, q, r, v);
    }
    if (q.scratch) atomicMax(q.scratch + kStatMaxHelpIters, (unsigned long long)(kSlowHard - budget));
    if (!budget) latch_error(q.err, GQ_ERR_TIMEOUT);
}

// Inspects the next peer record (round robin) and helps it if a request is
// pending with matching sequence fields.
static __device__ __noinline__ void wfq_inspect_peer(const gq_ring_view& R, const gq_dev& q, u32 me, u32 peer) {
    u64* pr = rec_of(R, peer);
    const u64 pend = ld_acq(pr + kRPending);
    if (!(pend & 1)) return;
    const u64 s2 = ld_acq(pr + kRSeq2);
    const u64 init = ld_acq(pr + kRInit);
    const u64 idx = ld_acq(pr + kRIndex);
    const u64 pend2 = ld_acq(pr + kRPending);
    const u64 s1 = ld_acq(pr + kRSeq1);
    if (s1 != s2 || !(pend2 & 1)) return;
    if (q.scratch) atomicAdd(q.scratch + kStatHelps, 1ull);
    wfq_help_request(R, q, peer, s2, (pend2 & 2) != 0, init, (u32)idx, me);
}

// The next peer after `prev` in round-robin order, skipping the caller.
__device__ __forceinline__ u32 wfq_next_peer(const gq_dev& q, u32 me, u32 prev) {
    u32 peer = (prev + 1) % q.max_threads;
    if (peer == me) peer = (peer + 1) % q.max_threads;
    return peer;
}

static __device__ __noinline__ void wfq_help_peer(const gq_ring_view& R, const gq_dev& q, u32 me, u64 pv) {
    // a cursor never used yet (zeroed at reset) starts the round robin at the
    // caller's own id, so that threads do not all inspect the same peers at once
    const u32 peer = wfq_next_peer(q, me, pv ? (u32)(pv >> 32) : me);
    R.helpc[me] = ((u64)peer << 32) | q.help_delay;
    if (peer != me) wfq_inspect_peer(R, q, me, peer);
}

// Help delay D (Section III-C): every D operations a thread inspects one peer
// record, round robin from its own id.  Callers that know the index `seq` of
// this operation among the thread's operations on this ring (the run drivers)
// pass it: the operation inspects peer me + 1 + seq / D when seq is a multiple
// of D, and no per-thread state is read or written.  Otherwise (kNoSeq) the
// countdown is owner-only state in a compact per-thread array (plain accesses;
// the 32 cursors of a warp share one 256-byte span).
constexpr u32 kNoSeq = 0xFFFFFFFFu;
__device__ __forceinline__ void wfq_maybe_help(const gq_ring_view& R, const gq_dev& q, u32 me, u32 seq = kNoSeq) {
    if (seq != kNoSeq) {
        if (seq % q.help_delay == 0) {
            const u32 peer = wfq_next_peer(q, me, (u32)((me + (u64)(seq / q.help_delay)) % q.max_threads));
            if (peer != me) wfq_inspect_peer(R, q, me, peer);
        }
        return;
    }
    const u64 pv = R.helpc[me];
    const u32 countdown = (u32)pv;
    if (countdown > 1 && countdown <= q.help_delay) {
        R.helpc[me] = pv - 1;
        return;
    }
    wfq_help_peer(R, q, me, pv);
}

// Patience stretch: an operation that has used its patience while requests
// of the same ring are already on the slow path keeps trying the fast path,
// up to patience * patience_stretch attempts in all.  Each request on the
// slow path costs rounds of SlowFAA that serialise on the ring's counter;
// when many operations run out of patience together (more threads than
// slots, operations that keep finding their slot taken) their requests queue
// behind each other while fast attempts would have gone through.  The ring's
// pending count is claimed with one fetch-and-add when it reads zero, so of
// the operations that run out of patience at the same moment one publishes
// and the others stretch.  The bound stays finite, so the operation stays
// wait-free.  Returns the new attempt limit; *claimed is set when the caller
// holds a pending count it has to publish under.
__device__ __forceinline__ u32 wfq_stretch(const gq_ring_view& R, const gq_dev& q, u32 patience, bool* claimed) {
    const u64 lim = (u64)patience * q.patience_stretch;
    const u32 big = lim > 0xFFFFFFFFull ? 0xFFFFFFFFu : (u32)lim;
    if (ld_rlx(R.slow_pending) != 0) return big;
    if (atomicAdd(R.slow_pending, 1ull) == 0) {
        *claimed = true;
        return patience;
    }
    atomicAdd(R.slow_pending, ~0ull);   // minus one: another operation publishes first
    return big;
}

// Publishes a request in the caller's record, helps it to completion, and
// retires it.  Returns the final local word (FIN set) or 0 on timeout.
static __device__ __noinline__ u64 wfq_slow_request(const gq_ring_view& R, const gq_dev& q, u32 me, bool enq, u64 init, u32 idx,
                                                    bool claimed) {
    u64* rec = rec_of(R, me);
    const u64 seq = ld_rlx(rec + kRSeq1);
    u64* L = rec + (enq ? kRLocalTail : kRLocalHead);
    st_rlx(rec + kRInit, init);
    st_rlx(rec + kRIndex, idx);
    if (enq) st_rel(R.owner + idx, me + 1);
    st_rel(L, init << 2);
    st_rel(rec + kRSeq2, seq);
    st_rel(rec + kRPending, 1ull | (enq ? 2ull : 0ull));
    if (q.scratch) atomicAdd(q.scratch + kStatSlowRequests, 1ull);
    if (q.patience_stretch > 1 && !claimed) atomicAdd(R.slow_pending, 1ull);
    wfq_help_request(R, q, me, seq, enq, init, idx, me);
    const u64 l = ld_acq(L);
    st_rel(rec + kRPending, 0);
    st_rel(rec + kRSeq1, seq + 1);
    if (q.patience_stretch > 1) atomicAdd(R.slow_pending, ~0ull);   // minus one
    return (l & kLFin) ? l : 0;
}


// Inner-ring enqueue of index idx by thread `me`.  tk (nullable, test
// recorder): the ticket the index was installed at, fast or slow.
template <bool MATCH, bool CNT = false>
__device__ int wfq_ring_enq(const gq_ring_view& R, const gq_dev& q, u32 idx, u32 me, u32 patience,
                            u64* tk = nullptr, u32 seq = kNoSeq) {
    wfq_maybe_help(R, q, me, seq);
    u64 t = 0;
    bool stretched = false, claimed = false;
    for (u32 p = 0, lim = patience; p < lim; ++p) {
        if (wfq_try_enq<MATCH, CNT>(R, q, idx, &t) == kTryOk) {
            if (tk) *tk = t;
            return GQ_OK;
        }
        if (q.backoff_ns) __nanosleep(q.backoff_ns);
        if (p + 1 == lim && !stretched && q.patience_stretch > 1) {
            stretched = true;
            lim = wfq_stretch(R, q, patience, &claimed);
        }
    }
    if (patience == 0) t = (g_cnt(ld_rlx(R.tail)) - 1) & kCntMask;   // a ticket value r never held
    oc_add<CNT>(kOcSlow);
    const u64 l = wfq_slow_request(R, q, me, true, t, idx, claimed);
    if (!l) {
        latch_error(q.err, GQ_ERR_TIMEOUT);
        return GQ_ERR_TIMEOUT;
    }
    // make the entry visible to fast dequeuers if no dequeuer did it yet
    const u64 tf = l_cnt(l);
    u64* slot = R.slots + (tf & q.slot_mask);
    const u64 c = (tf >> q.ring_order) & q.cycle_mask;
    u64 e = ld_acq(slot);
    for (u32 it = 0; it < kRetryLimit; ++it) {
        if (w_cyc(e) != c || w_idx(e) != idx || (e & kWEnq)) break;
        if (cas(slot, e, e | kWEnq)) break;
    }
    if (tk) *tk = tf;
    return GQ_OK;
}

// Inner-ring dequeue by thread `me`: GQ_OK with *idx, or GQ_EMPTY.  tk
// (nullable): the ticket the index was taken at.
template <bool MATCH, bool CNT = false>
__device__ int wfq_ring_deq(const gq_ring_view& R, const gq_dev& q, u32* idx, u32 me, u32 patience,
                            u64* tk = nullptr, u32 seq = kNoSeq) {
    if (ld_rlx(R.threshold) < 0) return GQ_EMPTY;
    wfq_maybe_help(R, q, me, seq);
    u64 h = 0;
    bool stretched = false, claimed = false;
    for (u32 p = 0, lim = patience; p < lim; ++p) {
        const int s = wfq_try_deq<MATCH, CNT>(R, q, idx, &h);
        if (s == kTryOk) {
            if (tk) *tk = h;
            return GQ_OK;
        }
        if (s == kTryEmpty) return GQ_EMPTY;
        if (q.backoff_ns) __nanosleep(q.backoff_ns);
        if (p + 1 == lim && !stretched && q.patience_stretch > 1) {
            stretched = true;
            lim = wfq_stretch(R, q, patience, &claimed);
        }
    }
    if (patience == 0) h = (g_cnt(ld_rlx(R.head)) - 1) & kCntMask;
    oc_add<CNT>(kOcSlow);
    const u64 l = wfq_slow_request(R, q, me, false, h, 0, claimed);
    if (!l) {
        latch_error(q.err, GQ_ERR_TIMEOUT);
        return GQ_ERR_TIMEOUT;
    }
    // the outcome is at ticket hf: an item of its cycle there is ours to consume
    const u64 hf = l_cnt(l);
    u64* slot = R.slots + (hf & q.slot_mask);
    const u64 c = (hf >> q.ring_order) & q.cycle_mask;
    const u64 e = ld_acq(slot);
    if (w_cyc(e) == c && w_idx(e) < kWBotC) {
        *idx = wfq_consume(R, slot, e, hf, q);
        if (tk) *tk = hf;
        return GQ_OK;
    }
    return GQ_EMPTY;
}

// tk (nullable, test recorder): the aq ticket of the operation.
// seq (run drivers): the index of this operation among the thread's
// operations on this queue (see wfq_maybe_help); kNoSeq otherwise.
template <class T, bool MATCH, bool CNT = false>
__device__ int wfq_enqueue(const gq_dev& q, T v, u32 tid, u64* tk = nullptr, u32 seq = kNoSeq) {
    if (tid >= q.max_threads) {
        latch_error(q.err, GQ_ERR_TOO_MANY_THREADS);
        return GQ_ERR_TOO_MANY_THREADS;
    }
    u32 i;
    int s = wfq_ring_deq<MATCH, CNT>(q.fq, q, &i, tid, q.patience_deq, nullptr, seq);
    if (s == GQ_EMPTY) return GQ_FULL;
    if (s != GQ_OK) return s;
    if (i >= q.capacity) {
        latch_error(q.err, GQ_ERR_INVALID);
        return GQ_ERR_INVALID;
    }
    data_store<T>(q, i, v);
    return wfq_ring_enq<MATCH, CNT>(q.aq, q, i, tid, q.patience_enq, tk, seq);
}

template <class T, bool MATCH, bool CNT = false>
__device__ int wfq_dequeue(const gq_dev& q, T* v, u32 tid, u64* tk = nullptr, u32 seq = kNoSeq) {
    if (tid >= q.max_threads) {
        latch_error(q.err, GQ_ERR_TOO_MANY_THREADS);
        return GQ_ERR_TOO_MANY_THREADS;
    }
    u32 i;
    int s = wfq_ring_deq<MATCH, CNT>(q.aq, q, &i, tid, q.patience_deq, tk, seq);
    if (s != GQ_OK) return s;
    if (i >= q.capacity) {
        latch_error(q.err, GQ_ERR_INVALID);
        return GQ_ERR_INVALID;
    }
    *v = data_load<T>(q, i);
    s = wfq_ring_enq<MATCH, CNT>(q.fq, q, i, tid, q.patience_enq, nullptr, seq);
    return s == GQ_OK ? GQ_OK : s;
}

// Enqueue or dequeue on one code path (see lfq_op): the rings are chosen per
// lane, so mixed warps run both kinds of operation together.
template <class T, bool CNT = false>
__device__ int wfq_op(const gq_dev& q, bool enq, T* v, u32 tid, u64* tk = nullptr, u32 seq = kNoSeq) {
    if (tid >= q.max_threads) {
        latch_error(q.err, GQ_ERR_TOO_MANY_THREADS);
        return GQ_ERR_TOO_MANY_THREADS;
    }
    const gq_ring_view& from = enq ? q.fq : q.aq;
    const gq_ring_view& to = enq ? q.aq : q.fq;
    u32 i;
    int s = wfq_ring_deq<true, CNT>(from, q, &i, tid, q.patience_deq, enq ? nullptr : tk, seq);
    if (s == GQ_EMPTY) return enq ? GQ_FULL : GQ_EMPTY;
    if (s != GQ_OK) return s;
    if (i >= q.capacity) {
        latch_error(q.err, GQ_ERR_INVALID);
        return GQ_ERR_INVALID;
    }
    if (enq) data_store<T>(q, i, *v);
    else *v = data_load<T>(q, i);
    return wfq_ring_enq<true, CNT>(to, q, i, tid, q.patience_enq, enq ? tk : nullptr, seq);
}

}  // namespace gqd
