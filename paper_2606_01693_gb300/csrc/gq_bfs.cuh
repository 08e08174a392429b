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

// Clears the cells an instance used and rewinds T and H (G-WFQ-YMC never reuses cells).
__device__ inline void ymc_cluster_clear(const gq_dev& q, u32 ct, u32 nct, cg::cluster_group& cluster) {
    // cells up to max(T, H), plus a margin for cells a slow-dequeue helper may
    // have scanned past the completing candidate
    const u64 used = max(ld_acq(q.ymc_tail), ld_acq(q.ymc_head)) + 65536;
    const u64 hi = used < q.capacity ? used : q.capacity;
    for (u64 i = 1 + ct; i <= hi; i += nct) {
        q.cell_val[i] = ~0ull;
        q.cell_enq[i] = 0;
        q.cell_deq[i] = 0;
    }
    cluster.sync();
    if (ct == 0) {
        st_rel(q.ymc_tail, 1);
        st_rel(q.ymc_head, 1);
    }
}

// One level-synchronous BFS by the threads of a thread-block cluster on the
// frontier queues qa / qb (left empty).  ctl[0..2]: rotating frontier counts.
// Returns the number of levels; adds scanned edges to *edges.
template <int KIND>
__device__ u32 cluster_bfs(const gq_dev& qa, const gq_dev& qb, u64* ctl, const gq_bfs_instance& g, u32* dist, u32 ct,
                           u32 nct, cg::cluster_group& cluster, u64* edges) {
    const u32 lane = threadIdx.x & 31;
    const u32 cw = ct >> 5;
    for (u64 v = ct; v < g.n; v += nct) dist[v] = kUnreached;
    if (ct == 0) {
        st_rlx(ctl + 0, 0);
        st_rlx(ctl + 1, 0);
        st_rlx(ctl + 2, 0);
    }
    cluster.sync();
    if (ct == 0) {
        dist[g.src] = 0;
        if (queue_enqueue<unsigned int, KIND>(qa, g.src, 0) == GQ_OK) st_rlx(ctl + 0, 1);
    }
    cluster.sync();
    u32 level = 0;
    for (;; ++level) {
        const u64 frontier = ld_acq(ctl + level % 3);
        if (frontier == 0) break;
        if (ct == 0) st_rlx(ctl + (level + 2) % 3, 0);
        const gq_dev& cur = (level & 1) ? qb : qa;
        const gq_dev& nxt = (level & 1) ? qa : qb;
        u32 cnt = 0;
        if (cw < (frontier + 31) / 32 || cw < 1) {
            bool active = true;
            for (u32 round = 0; round < kRetryLimit; ++round) {
                unsigned int v = 0;
                int s = GQ_EMPTY;
                if (active) s = queue_dequeue<unsigned int, KIND>(cur, &v, ct);
                active = active && (s == GQ_OK);
                if (!__ballot_sync(0xffffffffu, active)) break;
                u64 b = 0, e = 0;
                if (active) {
                    b = g.d_offsets[v];
                    e = g.d_offsets[v + 1];
                    if (e - b < 32) {
                        *edges += e - b;
                        for (u64 k = b; k < e; ++k) bfs_visit<KIND>(nxt, dist, g.d_adj[k], level + 1, ct, &cnt);
                    }
                }
                u32 big = __ballot_sync(0xffffffffu, active && (e - b >= 32));
                while (big) {
                    const u32 owner = __ffs(big) - 1;
                    big &= big - 1;
                    const u64 bb = __shfl_sync(0xffffffffu, b, owner);
                    const u64 ee = __shfl_sync(0xffffffffu, e, owner);
                    if (lane == 0) *edges += ee - bb;
                    for (u64 k = bb + lane; k < ee; k += 32) bfs_visit<KIND>(nxt, dist, g.d_adj[k], level + 1, ct, &cnt);
                    __syncwarp();
                }
            }
        }
        warp_add_full(reinterpret_cast<unsigned long long*>(ctl + (level + 1) % 3), cnt);
        cluster.sync();
    }
    if (KIND == GQ_YMC) {
        ymc_cluster_clear(qa, ct, nct, cluster);
        ymc_cluster_clear(qb, ct, nct, cluster);
    }
    cluster.sync();
    return level;
}

}  // namespace gqd
