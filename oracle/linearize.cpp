// Brute-force linearizability checker (Wing and Gong, "Testing and verifying
// concurrent objects", JPDC 1993, with the memoisation of visited
// configurations that Lowe describes in "Testing for linearizability", 2017).
// Test infrastructure only (see oracle.h).
//
// A history is linearizable iff its operations can be ordered so that (a) the
// order extends real-time precedence (a before b whenever a ended before b was
// called) and (b) replaying the order on the sequential FIFO reproduces every
// recorded result.  This is the check Section IV runs through Porcupine's queue
// model.  The search repeatedly picks a "minimal" pending operation (one that
// no other pending operation precedes), applies it to the sequential queue if
// its recorded result matches, and backtracks otherwise.
#include "oracle.h"

#include <string>
#include <unordered_set>
#include <vector>

namespace {

struct Search {
    int64_t n;
    const uint8_t* op;
    const uint64_t* val;
    const int8_t* status;
    const uint64_t* call;
    const uint64_t* end;
    uint64_t cap;
    std::vector<int64_t> overlap;
    std::unordered_set<std::string> seen;
    int64_t budget;
    bool exhausted = false;

    std::string key(uint64_t mask, const std::vector<uint64_t>& q) const {
        std::string k(reinterpret_cast<const char*>(&mask), sizeof(mask));
        k.append(reinterpret_cast<const char*>(q.data()), q.size() * sizeof(uint64_t));
        return k;
    }

    // Result of applying operation o to queue state q: true if the recorded
    // result is what the sequential FIFO would return.
    bool legal(int64_t o, const std::vector<uint64_t>& q) const {
        if (op[o] == 1) {
            if (status[o] == 0) return cap == 0 || q.size() < cap;
            if (status[o] == 1) return cap != 0 && (uint64_t)((int64_t)q.size() + overlap[o]) >= cap;
            return false;
        }
        if (status[o] == 2) return q.empty();
        if (status[o] == 0) return !q.empty() && q.front() == val[o];
        return false;
    }

    bool dfs(uint64_t mask, std::vector<uint64_t>& q) {
        uint64_t full = (n == 64) ? ~0ull : ((1ull << n) - 1);
        if (mask == full) return true;
        if (!seen.insert(key(mask, q)).second) return false;
        if ((int64_t)seen.size() > budget) { exhausted = true; return false; }
        uint64_t min_end = ~0ull;
        for (int64_t o = 0; o < n; ++o)
            if (!(mask >> o & 1) && end[o] < min_end) min_end = end[o];
        for (int64_t o = 0; o < n; ++o) {
            if (mask >> o & 1) continue;
            if (call[o] > min_end) continue;  // some pending op ended strictly before o began
            if (!legal(o, q)) continue;
            if (op[o] == 1 && status[o] == 0) {
                q.push_back(val[o]);
                if (dfs(mask | (1ull << o), q)) return true;
                q.pop_back();
            } else if (op[o] == 0 && status[o] == 0) {
                uint64_t front = q.front();
                q.erase(q.begin());
                if (dfs(mask | (1ull << o), q)) return true;
                q.insert(q.begin(), front);
            } else {
                if (dfs(mask | (1ull << o), q)) return true;
            }
            if (exhausted) return false;
        }
        return false;
    }
};

}  // namespace

extern "C" int orc_linearizable(int64_t n, const uint8_t* op, const uint64_t* val,
                                const int8_t* status, const uint64_t* call, const uint64_t* end,
                                uint64_t cap, int64_t max_states) {
    if (n < 0 || n > 63) return -2;
    for (int64_t i = 0; i < n; ++i)
        if (call[i] > end[i] || op[i] > 1) return -2;
    Search s{n, op, val, status, call, end, cap, std::vector<int64_t>(n, 0), {},
             max_states > 0 ? max_states : (int64_t)1 << 22};
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = 0; b < n; ++b)
            if (a != b && !(end[b] < call[a] || end[a] < call[b])) ++s.overlap[a];
    std::vector<uint64_t> q;
    bool ok = s.dfs(0, q);
    if (ok) return 1;
    return s.exhausted ? -1 : 0;
}
