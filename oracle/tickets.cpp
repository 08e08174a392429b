// Ticket checks on large concurrent runs (the fourth invariant of the
// device-side conformance checks, Section IV, made concrete for these queues).
// Test infrastructure only (see oracle.h).
//
// Each successful operation is recorded with a ticket: for the ring queues the
// position in the allocated-index ring at which the index was installed
// (enqueue) or taken (dequeue), for G-WFQ-YMC the cell.  Why each check holds:
//  * matching: a ring slot holds one entry per cycle and a dequeue takes the
//    entry of its own ticket's cycle, so the dequeue that returns an item has
//    the ticket its enqueue installed it at (a cell likewise holds one value);
//  * distinct: tickets come from fetch-and-add counters (or are claimed cells),
//    so no two successful enqueues, and no two successful dequeues, share one;
//  * real-time order: a ticket is drawn from a counter that only grows, inside
//    the operation's interval, so if enqueue A returned before enqueue B was
//    called, A's ticket is the smaller (the same for dequeues).  This is the
//    order the paper's linearization points follow (Section III-B: an
//    operation takes effect at its ticket's slot).
// Tickets live in a counter of `bits` bits (64, or 43 for G-WFQ's packed
// Global words) and may wrap: they are compared as signed distances from the
// first successful ticket, modulo 2^bits.
#include "oracle.h"

#include <algorithm>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

struct Hits {
    orc_report* r;
    void hit(int kind, int64_t idx) {
        if (r->violations == 0) { r->first_kind = kind; r->first_index = idx; }
        ++r->violations;
    }
};

struct Op {
    int64_t j;
    int64_t rel;      // ticket as a signed distance from the base
    uint64_t call, end;
};

// Real-time order among `ops`: every op must have a larger ticket than each op
// that ended before it was called.
void check_order(std::vector<Op>& ops, int kind, Hits& H) {
    std::sort(ops.begin(), ops.end(), [](const Op& a, const Op& b) { return a.call < b.call; });
    std::vector<const Op*> by_end(ops.size());
    for (size_t x = 0; x < ops.size(); ++x) by_end[x] = &ops[x];
    std::sort(by_end.begin(), by_end.end(), [](const Op* a, const Op* b) { return a->end < b->end; });
    size_t p = 0;
    bool any = false;
    int64_t best = 0;
    for (const Op& b : ops) {
        while (p < by_end.size() && by_end[p]->end < b.call) {
            if (!any || by_end[p]->rel > best) best = by_end[p]->rel;
            any = true;
            ++p;
        }
        if (any && b.rel <= best) H.hit(kind, b.j);
    }
}

}  // namespace

extern "C" int64_t orc_check_tickets(int64_t n, const uint8_t* kind, const int8_t* status, const uint64_t* val,
                                     const uint64_t* ticket, const uint64_t* call, const uint64_t* end,
                                     int32_t bits, orc_report* rep) {
    *rep = orc_report{};
    if (n < 0 || !kind || !status || !val || !ticket || bits < 2 || bits > 64) return -1;
    Hits H{rep};
    const uint64_t mask = bits == 64 ? ~0ull : ((1ull << bits) - 1);
    const uint64_t half = 1ull << (bits - 1);
    bool have_base = false;
    uint64_t base = 0;
    auto rel = [&](uint64_t t) -> int64_t {
        const uint64_t d = (t - base) & mask;
        return d >= half ? (int64_t)(d - half) - (int64_t)half : (int64_t)d;
    };

    std::unordered_map<uint64_t, uint64_t> enq_ticket;   // value -> ticket
    std::unordered_map<uint64_t, int64_t> seen_enq, seen_deq;
    std::vector<Op> enqs, deqs;
    for (int64_t j = 0; j < n; ++j) {
        if (status[j] != 0 || (kind[j] != 0 && kind[j] != 1)) continue;
        const uint64_t t = ticket[j];
        if ((t & ~mask) != 0) { H.hit(7, j); continue; }
        if (!have_base) { base = t; have_base = true; }
        if (kind[j] == 1) {
            ++rep->enq_ok;
            if (!seen_enq.emplace(t, j).second) H.hit(9, j);
            enq_ticket[val[j]] = t;
            enqs.push_back({j, rel(t), call ? call[j] : 0, end ? end[j] : 0});
        } else {
            ++rep->deq_ok;
            if (!seen_deq.emplace(t, j).second) H.hit(9, j);
            deqs.push_back({j, rel(t), call ? call[j] : 0, end ? end[j] : 0});
        }
    }
    for (const Op& d : deqs) {
        auto it = enq_ticket.find(val[d.j]);
        if (it == enq_ticket.end() || it->second != ticket[d.j]) H.hit(8, d.j);
    }
    if (call && end) {
        check_order(enqs, 10, H);
        check_order(deqs, 11, H);
    }
    return rep->violations;
}
