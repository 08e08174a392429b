// Textbook sequential breadth-first search (Cormen et al., "Introduction to
// Algorithms", BFS with a FIFO queue).  The level-synchronous queue BFS of
// Section V-B computes the same hop distances: distances are unique, only the
// parent choice may differ between correct traversals.
// Test infrastructure only (see oracle.h).
#include "oracle.h"

#include <vector>

extern "C" int64_t orc_bfs(int64_t n, const uint64_t* offsets, const uint32_t* adj, uint32_t src,
                           uint32_t* dist) {
    const uint32_t INF = 0xFFFFFFFFu;
    for (int64_t v = 0; v < n; ++v) dist[v] = INF;
    if (src >= (uint64_t)n) return 0;
    std::vector<uint32_t> fifo;
    fifo.reserve(1024);
    fifo.push_back(src);
    dist[src] = 0;
    size_t head = 0;
    while (head < fifo.size()) {
        uint32_t u = fifo[head++];
        for (uint64_t e = offsets[u]; e < offsets[u + 1]; ++e) {
            uint32_t w = adj[e];
            if (dist[w] == INF) {
                dist[w] = dist[u] + 1;
                fifo.push_back(w);
            }
        }
    }
    return (int64_t)fifo.size();
}
