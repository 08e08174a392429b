// Sequential FIFO specification and the mutex-guarded deque baseline.
// Test infrastructure only (see oracle.h).
//
// The sequential object follows the FIFO model the paper checks against in
// Section IV: an enqueue appends to the state list, a dequeue returns the head
// or reports EMPTY.  A bounded queue (Section III-B: ring of logical capacity n)
// additionally reports FULL when it already holds `cap` items.
#include "oracle.h"

#include <array>
#include <chrono>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

namespace {

enum : int8_t { kOK = 0, kFULL = 1, kEMPTY = 2 };

struct SeqFifo {
    uint64_t cap;  // 0 = unbounded
    std::deque<uint64_t> items;
    int8_t enq(uint64_t v) {
        if (cap != 0 && items.size() >= cap) return kFULL;
        items.push_back(v);
        return kOK;
    }
    int8_t deq(uint64_t* v) {
        if (items.empty()) return kEMPTY;
        *v = items.front();
        items.pop_front();
        return kOK;
    }
};

}  // namespace

extern "C" void orc_seqfifo_run(uint64_t cap, const uint8_t* kind, const uint64_t* val, int64_t n,
                                int8_t* status, uint64_t* out, uint64_t* final_contents,
                                int64_t* final_size) {
    SeqFifo q{cap, {}};
    for (int64_t i = 0; i < n; ++i) {
        uint64_t v = 0;
        if (kind[i] == 1) {
            status[i] = q.enq(val[i]);
        } else {
            status[i] = q.deq(&v);
        }
        if (out) out[i] = (kind[i] == 1) ? 0 : v;
    }
    if (final_contents) {
        int64_t k = 0;
        for (uint64_t v : q.items) final_contents[k++] = v;
    }
    if (final_size) *final_size = (int64_t)q.items.size();
}

// ---------------------------------------------------------------------------
// Mutex-guarded std::deque on N host threads (the CPU baseline).
// ---------------------------------------------------------------------------
extern "C" double orc_mutex_run(int32_t mode, int64_t T, int64_t K, const uint64_t* sched,
                                int64_t producers, const int64_t* ops_of, uint64_t cap,
                                int32_t nthreads, int64_t* counts) {
    if (nthreads < 1) nthreads = 1;
    std::mutex mu;
    std::deque<uint64_t> q;
    std::vector<std::array<int64_t, 4>> local(nthreads);

    auto enq = [&](uint64_t v) -> bool {
        std::lock_guard<std::mutex> g(mu);
        if (cap != 0 && q.size() >= cap) return false;
        q.push_back(v);
        return true;
    };
    auto deq = [&](uint64_t* v) -> bool {
        std::lock_guard<std::mutex> g(mu);
        if (q.empty()) return false;
        *v = q.front();
        q.pop_front();
        return true;
    };

    auto body = [&](int h) {
        std::array<int64_t, 4> c = {0, 0, 0, 0};
        uint64_t sink = 0;
        for (int64_t t = h; t < T; t += nthreads) {
            if (mode == 0) {
                for (int64_t s = 0; s < K; ++s) {
                    uint64_t tok = ((uint64_t)t << 16) | (uint64_t)s;
                    if (enq(tok)) ++c[0]; else ++c[1];
                    uint64_t v;
                    if (deq(&v)) { ++c[2]; sink += v; } else ++c[3];
                }
            } else if (mode == 1) {
                uint64_t seq = 0;
                for (int64_t i = 0; i < K; ++i) {
                    int64_t j = t * K + i;
                    bool is_enq = (sched[j >> 6] >> (j & 63)) & 1;
                    if (is_enq) {
                        uint64_t tok = ((uint64_t)t << 32) | (seq + 1);
                        ++seq;
                        if (enq(tok)) ++c[0]; else ++c[1];
                    } else {
                        uint64_t v;
                        if (deq(&v)) { ++c[2]; sink += v; } else ++c[3];
                    }
                }
            } else {
                int64_t k = ops_of[t];
                if (t < producers) {
                    for (int64_t s = 0; s < k; ++s) {
                        uint64_t tok = ((uint64_t)t << 32) | (uint64_t)(s + 1);
                        if (enq(tok)) ++c[0]; else ++c[1];
                    }
                } else {
                    for (int64_t s = 0; s < k; ++s) {
                        uint64_t v;
                        if (deq(&v)) { ++c[2]; sink += v; } else ++c[3];
                    }
                }
            }
        }
        local[h] = c;
        if (sink == 0x5eed) local[h][0] += 0;  // keep the dequeued values live
    };

    auto t0 = std::chrono::steady_clock::now();
    std::vector<std::thread> pool;
    for (int h = 0; h < nthreads; ++h) pool.emplace_back(body, h);
    for (auto& th : pool) th.join();
    auto t1 = std::chrono::steady_clock::now();
    for (int i = 0; i < 4; ++i) {
        counts[i] = 0;
        for (int h = 0; h < nthreads; ++h) counts[i] += local[h][i];
    }
    return std::chrono::duration<double>(t1 - t0).count();
}
