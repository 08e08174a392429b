// Invariant checks on large concurrent runs (Section IV "Device-side FIFO
// conformance": exactly once, no out-of-bounds token, monotone sequence per
// producer), plus one consequence of FIFO order on the items left behind.
// Test infrastructure only (see oracle.h).
//
// Why each check holds for any linearizable FIFO:
//  * exactly once: every successfully enqueued token is returned by exactly one
//    successful dequeue or is still in the queue at the end.
//  * per-consumer order: a producer enqueues its tokens in increasing seq, so
//    they are linearized in that order and must leave the queue in that order;
//    a single consumer therefore sees any one producer's tokens with increasing seq.
//  * no overtaking: if token (p, s2) left the queue during the run, every
//    (p, s1) with s1 < s2 left before it, so none can remain at the end.
//  * drained order: a single-threaded drain returns the remaining items in
//    FIFO order, so per producer the seqs increase along the drain.
#include "oracle.h"

#include <algorithm>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {
struct Rec {
    orc_report* r;
    void hit(int kind, int64_t idx) {
        if (r->violations == 0) { r->first_kind = kind; r->first_index = idx; }
        ++r->violations;
    }
};
}  // namespace

extern "C" int64_t orc_check_log(int64_t T, int64_t K, const uint8_t* kind, const int8_t* status,
                                 const uint64_t* val, const uint64_t* drained, int64_t n_drained,
                                 int32_t prod_shift, uint64_t seq_mask, uint64_t seq_bias,
                                 orc_report* rep) {
    *rep = orc_report{};
    Rec R{rep};
    const int64_t N = T * K;
    std::vector<uint64_t> in, out;
    in.reserve(N / 2 + 1);
    out.reserve(N / 2 + 1 + n_drained);
    for (int64_t j = 0; j < N; ++j) {
        if (kind[j] == 1) {
            if (status[j] == 0) { ++rep->enq_ok; in.push_back(val[j]); }
            else if (status[j] == 1) ++rep->enq_full;
            else R.hit(6, j);
        } else if (kind[j] == 0) {
            if (status[j] == 0) { ++rep->deq_ok; out.push_back(val[j]); }
            else if (status[j] == 2) ++rep->deq_empty;
            else R.hit(6, j);
        }
    }
    rep->drained = n_drained;
    for (int64_t d = 0; d < n_drained; ++d) out.push_back(drained[d]);

    // exactly once: multiset(dequeued + drained) == multiset(enqueued OK)
    std::sort(in.begin(), in.end());
    std::sort(out.begin(), out.end());
    {
        size_t a = 0, b = 0;
        while (a < in.size() || b < out.size()) {
            if (a < in.size() && b < out.size() && in[a] == out[b]) { ++a; ++b; continue; }
            if (b >= out.size() || (a < in.size() && in[a] < out[b])) { R.hit(1, (int64_t)a); ++a; }
            else { R.hit(1, (int64_t)b); ++b; }
        }
    }

    auto decode = [&](uint64_t tok, uint64_t* p, uint64_t* s) -> bool {
        *p = tok >> prod_shift;
        uint64_t low = tok & seq_mask;
        if (low < seq_bias) return false;
        *s = low - seq_bias;
        return true;
    };

    // per-consumer order: for each thread, its successful dequeues in program order
    std::unordered_map<uint64_t, uint64_t> max_deq;  // producer -> max seq dequeued during the run
    std::vector<std::pair<uint64_t, std::pair<int64_t, uint64_t>>> mine;
    for (int64_t t = 0; t < T; ++t) {
        mine.clear();
        for (int64_t i = 0; i < K; ++i) {
            int64_t j = i * T + t;
            if (kind[j] != 0 || status[j] != 0) continue;
            uint64_t p, s;
            if (!decode(val[j], &p, &s)) { R.hit(5, j); continue; }
            mine.push_back({p, {i, s}});
            auto it = max_deq.find(p);
            if (it == max_deq.end() || it->second < s) max_deq[p] = s;
        }
        std::sort(mine.begin(), mine.end());
        for (size_t x = 1; x < mine.size(); ++x)
            if (mine[x].first == mine[x - 1].first && mine[x].second.second <= mine[x - 1].second.second)
                R.hit(2, mine[x].second.first * T + t);
    }

    // no overtaking, drained order
    std::unordered_map<uint64_t, uint64_t> last_drained;
    for (int64_t d = 0; d < n_drained; ++d) {
        uint64_t p, s;
        if (!decode(drained[d], &p, &s)) { R.hit(5, d); continue; }
        auto it = max_deq.find(p);
        if (it != max_deq.end() && it->second >= s) R.hit(3, d);
        auto jt = last_drained.find(p);
        if (jt != last_drained.end() && jt->second >= s) R.hit(4, d);
        last_drained[p] = s;
    }
    return rep->violations;
}
