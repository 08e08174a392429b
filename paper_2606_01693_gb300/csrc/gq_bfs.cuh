// Device-side BFS building blocks shared by the BFS kernels (Section V-B
// level-synchronous BFS): the neighbour claim and the per-cluster search used
// by the batched and the serving schedulers.
#pragma once

#include <cooperative_groups.h>

#include "gq_ops.cuh"

namespace gqd {

namespace cg = cooperative_groups;

constexpr u32 kUnreached = 0xFFFFFFFFu;

// Claims neighbour w for the next level (distance CAS UNREACHED -> next_level)
// and enqueues it into the next frontier; *cnt counts the enqueued vertices.
template <int KIND>
__device__ __forceinline__ void bfs_visit(const gq_dev& nxt, u32* dist, u32 w, u32 next_level, u32 tid, u32* cnt) {
    if (aref<u32>(dist[w]).load(kRlx) != kUnreached) return;
    if (atomicCAS(dist + w, kUnreached, next_level) != kUnreached) return;
    if (queue_enqueue<unsigned int, KIND>(nxt, w, tid) == GQ_OK) ++*cnt;
}

// Barrier of the threads that run one BFS instance when they form one
// thread-block cluster: the hardware cluster barrier (release / acquire at
// cluster scope).  A barrier object returns false when the group has to give
// the instance up (only a multi-cluster barrier whose bounded wait expired
// does); every thread of the group gets the same answer.
struct ClusterSync {
    cg::cluster_group& cluster;
    __device__ bool operator()() const {
        cluster.sync();
        return true;
    }
};

// Clears the cells an instance used and rewinds T and H (G-WFQ-YMC never reuses cells).
template <class Sync>
__device__ inline bool ymc_group_clear(const gq_dev& q, u32 ct, u32 nct, const Sync& sync) {
    // cells up to max(T, H), plus a margin for cells a slow-dequeue helper may
    // have scanned past the completing candidate
    const u64 used = max(ld_acq(q.ymc_tail), ld_acq(q.ymc_head)) + 65536;
    const u64 hi = used < q.capacity ? used : q.capacity;
    for (u64 i = 1 + ct; i <= hi; i += nct) {
        q.cell_val[2 * i] = ~0ull;    // <value, dequeue reference> pair
        q.cell_deq[2 * i] = 0;
        q.cell_enq[i] = 0;
    }
    if (!sync()) return false;
    if (ct == 0) {
        st_rel(q.ymc_tail, 1);
        st_rel(q.ymc_head, 1);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Work of one warp in one level
// ---------------------------------------------------------------------------
//
// Degrees are skewed (R-MAT hubs have 10^5 neighbours), so neither "the lane
// that dequeued a vertex scans it" nor "its warp scans it" bounds the time of a
// level.  Two mechanisms share the edges instead:
//   * gather: a warp lays the adjacency lists of the (up to 32) vertices it
//     dequeued end to end (warp prefix sum of their degrees) and scans the
//     combined list 32 edges at a time, each lane finding its vertex by binary
//     search over the prefix sums;
//   * chunk map: a vertex of degree >= kHeavyDeg is cut into chunks of kChunk
//     edges.  Its lane reserves that many consecutive map positions (one
//     fetch-add on the level's `reserved` counter) and writes one word per
//     chunk (vertex, chunk index).  Every warp of the search -- those with
//     nothing to dequeue from the start, the others once their dequeues
//     return EMPTY -- takes map positions with a fetch-add on `handed`,
//     waits for the word at its position, scans that chunk and clears the
//     word.  A warp leaves when the dequeuing warps are all done (`done`
//     reached the number of dequeuing warps) and no reserved position is left.
// Positions past the map's capacity are not written: the vertex is gathered
// instead (the part of its reservation inside the map is written as skips).

constexpr u64 kHeavyDeg = 128;
constexpr u64 kChunk = 128;
constexpr u32 kFull = 0xffffffffu;
constexpr u64 kSkipChunk = ~0ull;
constexpr u64 kChunkWaitNs = 4000000000ull;     // bound of any wait for a chunk word (4 s)
constexpr u64 kClusterChunkCap = 1u << 14;      // chunk-map positions of one cluster's search

// Table memory: a header of six 4 KB lines, then the map itself (cap words, all
// zero between levels: every written word is cleared by the warp that scans
// it).  Header lines 0-3 (three words each, rotating by level): reserved,
// handed, done, taken; lines 4 and 5 hold the whole-GPU search's barrier count
// and generation (and, in line 4, the graph's maximum degree).  Hot words on different 4 KB lines land in different L2 slices,
// so the pollers of one word do not queue in front of the atomics on another.
// A map word is (vertex << 32) | (chunk index + 1), or kSkipChunk.
constexpr u64 kTabLine = 512;                   // words per header line (4 KB)
constexpr u64 kTabHeader = 6 * kTabLine;
enum { kTabReserved = 0, kTabHanded = 1, kTabDone = 2, kTabTaken = 3, kTabBarCount = 4, kTabBarGen = 5 };
// the graph's maximum degree (zero between searches), in the barrier-count line
constexpr u64 kTabMaxDeg = kTabBarCount * kTabLine + 8;
__host__ __device__ constexpr u64 chunk_map_bytes(u64 cap) { return (kTabHeader + cap) * sizeof(u64); }

// Called by one thread before a search: clears the per-level counters.
__device__ __forceinline__ void chunk_reset_all(u64* table) {
    for (u32 l = 0; l < 4; ++l)
        for (u32 r = 0; r < 3; ++r) st_rlx(table + l * kTabLine + r, 0);
}

struct LevelCtx {
    const u64* off;
    const u32* adj;
    u32* dist;
    u32 next_level, rec;    // rec: record id for the queue operations
    u64* map;
    u64 cap;
    u64* reserved;
    u64* handed;
    u64* done;
    u64* taken;             // G-WFQ: dequeues reserved this level
    u64 frontier;           // items in the current frontier queue
    u64 dequeuers;          // warps that dequeue this level
};

__device__ __forceinline__ LevelCtx level_ctx(const u64* off, const u32* adj, u32* dist, u32 level, u32 rec,
                                              u64* table, u64 cap, u64 frontier, u64 dequeuers) {
    LevelCtx c;
    c.off = off;
    c.adj = adj;
    c.dist = dist;
    c.next_level = level + 1;
    c.rec = rec;
    c.map = table + kTabHeader;
    c.cap = cap;
    c.reserved = table + kTabReserved * kTabLine + level % 3;
    c.handed = table + kTabHanded * kTabLine + level % 3;
    c.done = table + kTabDone * kTabLine + level % 3;
    c.taken = table + kTabTaken * kTabLine + level % 3;
    c.frontier = frontier;
    c.dequeuers = dequeuers;
    return c;
}

// Called by one thread during level L: clears the counters of level L + 1
// (last used during level L - 2).
__device__ __forceinline__ void chunk_prepare_next(u64* table, u32 level) {
    const u32 r = (level + 1) % 3;
    for (u32 l = 0; l < 4; ++l) st_rlx(table + l * kTabLine + r, 0);
}

// Lane: visits up to kVisitBatch edges at once.  The adjacency loads of the
// batch are issued together, then the distance loads, so a lane has several
// memory requests in flight instead of one dependent chain per edge.
constexpr int kVisitBatch = 4;

template <int KIND>
__device__ __forceinline__ void visit_batch(const gq_dev& nxt, const LevelCtx& c, const u64 (&e)[kVisitBatch],
                                            const bool (&ok)[kVisitBatch], u32* cnt) {
    u32 w[kVisitBatch], d[kVisitBatch];
#pragma unroll
    for (int u = 0; u < kVisitBatch; ++u) w[u] = ok[u] ? __ldg(c.adj + e[u]) : 0u;
#pragma unroll
    for (int u = 0; u < kVisitBatch; ++u) d[u] = ok[u] ? aref<u32>(c.dist[w[u]]).load(kRlx) : 0u;
#pragma unroll
    for (int u = 0; u < kVisitBatch; ++u) {
        if (!ok[u] || d[u] != kUnreached) continue;
        if (atomicCAS(c.dist + w[u], kUnreached, c.next_level) != kUnreached) continue;
        if (queue_enqueue<unsigned int, KIND>(nxt, w[u], c.rec) == GQ_OK) ++*cnt;
    }
}

// Warp: scans the adjacency lists [b, b + d) of its lanes as one combined list.
template <int KIND>
__device__ void warp_gather(const gq_dev& nxt, const LevelCtx& c, u64 b, u64 d, u32* cnt, u64* edges) {
    const u32 lane = threadIdx.x & 31;
    u64 incl = d;
    for (u32 o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const u64 total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    if (lane == 0) *edges += total;
    const u64 start = b - (incl - d);   // combined index x of this lane's list is edge start + x (mod 2^64)
    for (u64 base = 0; base < total; base += 32 * kVisitBatch) {
        u64 e[kVisitBatch];
        bool ok[kVisitBatch];
#pragma unroll
        for (int u = 0; u < kVisitBatch; ++u) {
            const u64 x = base + 32 * u + lane;
            u32 pos = 0;                 // first lane whose inclusive sum exceeds x
            for (u32 step = 16; step; step >>= 1) {
                const u64 v = __shfl_sync(kFull, incl, pos + step - 1);
                if (v <= x) pos += step;
            }
            e[u] = __shfl_sync(kFull, start, pos) + x;
            ok[u] = x < total;
        }
        visit_batch<KIND>(nxt, c, e, ok, cnt);
    }
}

// Lane: cuts vertex v (edges [b, b + d)) into chunks and writes them into the
// map; false if the map has no room (the caller gathers it).
__device__ __forceinline__ bool chunk_publish(const LevelCtx& c, u32 v, u64 d) {
    const u64 n = (d + kChunk - 1) / kChunk;
    const u64 p = faa_rlx(c.reserved, n);
    const bool fits = p + n <= c.cap;
    for (u64 j = 0; j < n && p + j < c.cap; ++j)
        st_rlx(c.map + p + j, fits ? (((u64)v << 32) | (j + 1)) : kSkipChunk);   // never 0 (0 = not written)
    return fits;
}

// Warp: phase 1 -- dequeue the frontier, gather light vertices, publish heavy
// ones.  The level knows its frontier size F, and its dequeuing warps are
// warps 0 .. dequeuers-1: in round r, lane l of warp w does dequeue number
// (r * dequeuers + w) * 32 + l if that is below F.  So exactly F dequeues run,
// every one finds an item and none returns EMPTY (an EMPTY dequeue would cost a
// ticket -- for G-WFQ-YMC a pool cell that the next level's enqueuers would
// have to step over), with no counter to reserve them.  G-WFQ instead reserves
// each dequeue with a warp-aggregated fetch-add on `taken` (also exactly F):
// the fetch-add staggers the warps, and all of them arriving at once sent more
// G-WFQ dequeues to the slow path (4096^2 grid 244 -> 354 ms).  A dequeue that
// fails anyway latches GQ_ERR_INVALID in the queue.  With `chunked`, the warp
// then counts itself in `done` for the chunk phase.
template <int KIND>
__device__ void level_dequeue(const gq_dev& cur, const gq_dev& nxt, const LevelCtx& c, u32 w, bool chunked,
                              u32* cnt, u64* edges) {
    const u32 lane = threadIdx.x & 31;
    for (u64 round = 0;; ++round) {
        bool active;
        if constexpr (KIND == GQ_WFQ) active = warp_faa(c.taken, 1) < c.frontier;
        else active = ((round * c.dequeuers + w) * 32 + lane) < c.frontier;
        if (!__ballot_sync(kFull, active)) break;
        unsigned int v = 0;
        if (active) {
            const int s = queue_dequeue<unsigned int, KIND>(cur, &v, c.rec);
            if (s != GQ_OK) {
                if (s == GQ_EMPTY) latch_error(cur.err, GQ_ERR_INVALID);
                active = false;
            }
        }
        u64 b = 0, d = 0;
        if (active) {
            b = c.off[v];
            d = c.off[v + 1] - b;
            if (d >= kHeavyDeg && chunk_publish(c, v, d)) d = 0;
        }
        warp_gather<KIND>(nxt, c, b, d, cnt, edges);
    }
    if (!chunked) return;
    __syncwarp();
    if (lane == 0) {
        __threadfence();                    // the chunk words are written before `done` counts this warp
        faa_rlx(c.done, 1);
    }
}

// Warp: phase 2 -- take chunks until the level has none left.  Returns false
// if a wait expired (the caller latches an error).
template <int KIND>
__device__ bool level_chunks(const gq_dev& nxt, const LevelCtx& c, u32* cnt, u64* edges) {
    const u32 lane = threadIdx.x & 31;
    const u64 t0 = globaltimer();
    for (u32 polls = 0;; ++polls) {
        // lane 0 decides: 0 = leave, 1 = chunk word in `item`, 2 = poll again, 3 = expired
        u64 item = 0;
        u32 what = 2;
        if (lane == 0) {
            const u64 fin = ld_acq(c.done);
            u64 res = ld_acq(c.reserved);
            if (res > c.cap) res = c.cap;
            const u64 h = ld_rlx(c.handed);
            if (h < res) {
                const u64 g = faa_rlx(c.handed, 1);
                if (g < c.cap) {
                    // position g is (or will be) reserved unless the level closes first
                    for (u32 w = 0;; ++w) {
                        item = ld_acq(c.map + g);
                        if (item) {
                            st_rlx(c.map + g, 0);
                            what = 1;
                            break;
                        }
                        if (ld_acq(c.done) == c.dequeuers) {
                            u64 r2 = ld_acq(c.reserved);
                            if (g >= r2) {
                                what = 0;
                                break;
                            }
                            item = ld_acq(c.map + g);
                            if (item) continue;
                        }
                        if (globaltimer() - t0 > kChunkWaitNs) {
                            what = 3;
                            break;
                        }
                        __nanosleep(64);
                    }
                } else {
                    what = 0;
                }
            } else if (fin == c.dequeuers) {
                what = 0;
            } else if (globaltimer() - t0 > kChunkWaitNs) {
                what = 3;
            }
        }
        what = __shfl_sync(kFull, what, 0);
        if (what == 0) return true;
        if (what == 3) return false;
        if (what == 2) {
            __nanosleep(polls < 64 ? 64 : 256);
            continue;
        }
        item = __shfl_sync(kFull, item, 0);
        if (item == kSkipChunk) continue;
        const u32 v = (u32)(item >> 32);
        const u64 k = (item & 0xFFFFFFFFull) - 1;
        const u64 vb = c.off[v], ve = c.off[v + 1];
        const u64 b = vb + k * kChunk;
        const u64 e = b + kChunk < ve ? b + kChunk : ve;
        if (lane == 0) *edges += e - b;
        for (u64 j = b + lane; j < e; j += 32 * kVisitBatch) {
            u64 ex[kVisitBatch];
            bool ok[kVisitBatch];
#pragma unroll
            for (int u = 0; u < kVisitBatch; ++u) {
                ex[u] = j + 32 * u;
                ok[u] = ex[u] < e;
            }
            visit_batch<KIND>(nxt, c, ex, ok, cnt);
        }
        __syncwarp();
    }
}

constexpr u32 kBfsAborted = 0xFFFFFFFFu;

// One level-synchronous BFS by a group of nct threads (thread ct of the group;
// `sync` is the group's barrier) on the frontier queues qa / qb (left empty).
// ctl[0..2]: rotating frontier counts; table: the group's chunk map of `cap`
// positions.  Returns the number of levels, or kBfsAborted when a barrier gave
// up (the distances are then incomplete); adds scanned edges to *edges; a chunk
// wait that expired is latched in *err (nullable) as 1.  That is the only
// failure of the chunk phase: a vertex whose chunks do not fit in the map is
// scanned by the gather instead (chunk_publish), so a full map is not an error.
template <int KIND, class Sync>
__device__ u32 group_bfs(const gq_dev& qa, const gq_dev& qb, u64* ctl, u64* table, u64 cap,
                         const gq_bfs_instance& g, u32* dist, u32 ct, u32 nct, const Sync& sync,
                         u64* edges, unsigned long long* err) {
    const u32 cw = ct >> 5, nwarps = nct >> 5;
    const u64* off = reinterpret_cast<const u64*>(g.d_offsets);
    u64 maxdeg = 0;
    for (u64 v = ct; v < g.n; v += nct) {
        dist[v] = kUnreached;
        const u64 d = off[v + 1] - off[v];
        maxdeg = d > maxdeg ? d : maxdeg;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const u64 y = __shfl_xor_sync(kFull, maxdeg, o);
        maxdeg = y > maxdeg ? y : maxdeg;
    }
    if ((threadIdx.x & 31) == 0 && maxdeg) atomicMax(reinterpret_cast<unsigned long long*>(table + kTabMaxDeg), maxdeg);
    if (ct == 0) {
        st_rlx(ctl + 0, 0);
        st_rlx(ctl + 1, 0);
        st_rlx(ctl + 2, 0);
        chunk_reset_all(table);
    }
    if (!sync()) return kBfsAborted;
    if (ct == 0) {
        dist[g.src] = 0;
        if (queue_enqueue<unsigned int, KIND>(qa, g.src, 0) == GQ_OK) st_rlx(ctl + 0, 1);
    }
    if (!sync()) return kBfsAborted;
    // without a vertex of degree >= kHeavyDeg no chunk is ever published
    const bool chunks = ld_acq(table + kTabMaxDeg) >= kHeavyDeg;
    u32 level = 0;
    for (;; ++level) {
        const u64 frontier = ld_acq(ctl + level % 3);
        if (frontier == 0) break;
        if (ct == 0) {
            st_rlx(ctl + (level + 2) % 3, 0);
            chunk_prepare_next(table, level);
        }
        const u64 want = (frontier + 31) / 32;
        const u64 dq = want < nwarps ? want : nwarps;
        const LevelCtx c = level_ctx(reinterpret_cast<const u64*>(g.d_offsets), g.d_adj, dist, level, ct, table, cap,
                                     frontier, dq);
        const gq_dev& cur = (level & 1) ? qb : qa;
        const gq_dev& nxt = (level & 1) ? qa : qb;
        u32 cnt = 0;
        if (cw < dq) level_dequeue<KIND>(cur, nxt, c, cw, chunks, &cnt, edges);
        if (chunks && !level_chunks<KIND>(nxt, c, &cnt, edges) && (threadIdx.x & 31) == 0 && err)
            atomicCAS(err, 0ull, 1ull);
        warp_add_full(reinterpret_cast<unsigned long long*>(ctl + (level + 1) % 3), cnt);
        if (!sync()) return kBfsAborted;
    }
    if (KIND == GQ_YMC) {
        if (!ymc_group_clear(qa, ct, nct, sync) || !ymc_group_clear(qb, ct, nct, sync)) return kBfsAborted;
    }
    if (!sync()) return kBfsAborted;
    if (ct == 0) st_rlx(table + kTabMaxDeg, 0);      // every thread read it before the last barrier
    return level;
}

// The group is one thread-block cluster.
template <int KIND>
__device__ u32 cluster_bfs(const gq_dev& qa, const gq_dev& qb, u64* ctl, u64* table, u64 cap,
                           const gq_bfs_instance& g, u32* dist, u32 ct, u32 nct, cg::cluster_group& cluster,
                           u64* edges, unsigned long long* err) {
    return group_bfs<KIND>(qa, qb, ctl, table, cap, g, dist, ct, nct, ClusterSync{cluster}, edges, err);
}

}  // namespace gqd
