/*
 * gq_apps.h -- C ABI of the applications built on the queues (Section V-B).
 *
 *   gq_bfs  level-synchronous breadth-first search over a CSR graph with two
 *           frontier queues that alternate between levels: the current
 *           frontier is dequeued, each vertex's neighbours are scanned, newly
 *           reached vertices are claimed (distance CAS from UNREACHED to
 *           level + 1) and enqueued into the next frontier, until the next
 *           frontier is empty (Section V-B "Level-synchronous BFS").
 *
 * Conventions as in gq.h: int status returns, device pointers d_*, work
 * asynchronous on `stream`, errors latched on the device are returned by
 * gq_sync_status on either queue.
 */
#ifndef GQ_APPS_H
#define GQ_APPS_H

#include <stdint.h>

#include "gq.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GQ_BFS_UNREACHED 0xFFFFFFFFu

/* Breadth-first search from `src`.
 *   q_a, q_b: two empty queues of the same kind with 4-byte elements, each of
 *     capacity >= the largest frontier (|V| always suffices); G-WFQ-YMC, whose
 *     cells are never reused, needs a pool of about 3 |V| + 64 (levels + 1)
 *     cells (each level's dequeuers end with one EMPTY ticket per lane), and
 *     max_threads >= the launch's threads (gq_bfs uses at most
 *     min(max_threads, resident threads) threads).  They are left empty.
 *   n: vertices (< 2^32 - 1); d_offsets[n + 1] (uint64), d_adj[d_offsets[n]]
 *     (uint32 neighbour ids, any order).
 *   d_dist[n] (uint32): written with hop counts, GQ_BFS_UNREACHED elsewhere.
 *   d_stats (nullable, 4 x uint64): levels, vertices reached, edges scanned,
 *     error code of the grid barrier (0 = none).
 * The search runs as one cooperative persistent kernel; a device-wide barrier
 * separates levels (bounded wait: on expiry the kernel sets d_stats[3] and
 * returns).  Errors: GQ_ERR_INVALID, GQ_ERR_CUDA. */
int gq_bfs(gq_handle q_a, gq_handle q_b, uint64_t n, const uint64_t* d_offsets, const uint32_t* d_adj,
           uint32_t src, uint32_t* d_dist, unsigned long long* d_stats, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GQ_APPS_H */
