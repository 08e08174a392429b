// Fast seeded graph generation for the synthetic inputs (same definitions as
// synth/__init__.py; no queue arithmetic).  SplitMix64 output k of the stream
// seeded with s:  z = s + (k + 1) * 0x9E3779B97F4A7C15, then the published
// finaliser (shift-xor-multiply by 0xBF58476D1CE4E5B9 and 0x94D049BB133111EB).
#include <stdint.h>

#include <algorithm>
#include <thread>
#include <vector>

static inline uint64_t splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class F>
static void parallel_for(int64_t n, F f) {
    unsigned nt = std::max(1u, std::thread::hardware_concurrency());
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
            f(lo, hi);
        });
    for (auto& x : th) x.join();
}

extern "C" {

// R-MAT edge e picks, at level l, the quadrant of the 32-bit draw
// splitmix64(seed, e * scale + l) >> 32 against thresholds t1 < t2 < t3.
// Writes both directions of every non-loop edge as (src, dst) pairs; returns
// the number of pairs (<= 2 m).
int64_t synth_rmat_pairs(int scale, int64_t m, uint64_t seed, uint64_t t1, uint64_t t2, uint64_t t3, uint32_t* src,
                         uint32_t* dst) {
    std::vector<uint8_t> keep(m);
    std::vector<uint32_t> s(m), d(m);
    parallel_for(m, [&](int64_t lo, int64_t hi) {
        for (int64_t e = lo; e < hi; ++e) {
            uint64_t a = 0, b = 0;
            for (int l = 0; l < scale; ++l) {
                uint64_t r = splitmix64(seed, (uint64_t)e * scale + l) >> 32;
                uint64_t bit = 1ull << (scale - 1 - l);
                if (r >= t2) a |= bit;
                if ((r >= t1 && r < t2) || r >= t3) b |= bit;
            }
            s[e] = (uint32_t)a;
            d[e] = (uint32_t)b;
            keep[e] = a != b;
        }
    });
    int64_t k = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (!keep[e]) continue;
        src[k] = s[e]; dst[k] = d[e]; ++k;
        src[k] = d[e]; dst[k] = s[e]; ++k;
    }
    return k;
}

// CSR with sorted, duplicate-free neighbour lists from k (src, dst) pairs.
// offsets[n + 1]; adj must hold k entries.  Returns the number of edges kept.
int64_t synth_csr(int64_t n, int64_t k, const uint32_t* src, const uint32_t* dst, uint64_t* offsets, uint32_t* adj) {
    std::vector<uint64_t> start(n + 1, 0);
    for (int64_t i = 0; i < k; ++i) ++start[src[i] + 1];
    for (int64_t v = 0; v < n; ++v) start[v + 1] += start[v];
    std::vector<uint32_t> tmp(k);
    std::vector<uint64_t> pos(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < k; ++i) tmp[pos[src[i]]++] = dst[i];
    std::vector<uint64_t> cnt(n, 0);
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; ++v) {
            uint32_t* b = tmp.data() + start[v];
            uint32_t* e = tmp.data() + start[v + 1];
            std::sort(b, e);
            cnt[v] = (uint64_t)(std::unique(b, e) - b);
        }
    });
    offsets[0] = 0;
    for (int64_t v = 0; v < n; ++v) offsets[v + 1] = offsets[v] + cnt[v];
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; ++v)
            std::copy(tmp.data() + start[v], tmp.data() + start[v] + cnt[v], adj + offsets[v]);
    });
    return (int64_t)offsets[n];
}

}  // extern "C"
