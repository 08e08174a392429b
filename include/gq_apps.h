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

/* ---- batched BFS: many independent instances in one persistent launch ----
 * Instances are distributed through a queue of instance ids; each thread-block
 * cluster (cluster_blocks blocks of 256 threads, hardware cluster barrier
 * between levels) takes the next id, runs a level-synchronous BFS on its own
 * pair of frontier queues, and repeats until the id queue is empty. */
typedef struct {
    uint64_t n;                  /* vertices                          */
    const uint64_t* d_offsets;   /* n + 1                              */
    const uint32_t* d_adj;
    uint32_t* d_dist;            /* n, written (GQ_BFS_UNREACHED)      */
    uint32_t src;
    uint32_t reserved;
} gq_bfs_instance;

/* Workspace for gq_bfs_batch with `slots` clusters. */
int gq_bfs_batch_workspace_bytes(uint32_t slots, uint64_t* bytes);

/* d_instances: device array of ninst gq_bfs_instance; d_order: device array of
 * the ninst instance ids in the order they are handed out (largest first keeps
 * the tail short).  id_queue: an empty 4-byte queue of capacity >= ninst with
 * max_threads >= slots.  frontier: 2 * slots empty 4-byte queues of the same
 * kind as each other, capacity >= the largest instance's vertices (G-WFQ-YMC:
 * pool >= 3 n + 64 (levels + 1) of the largest instance: the cells used by an
 * instance are cleared on the device before the next one), max_threads >=
 * cluster_blocks * 256.  cluster_blocks in {1, 2, 4, 8}.  All queues are left
 * empty.  d_stats (nullable, 4 x uint64): instances done, edges scanned,
 * levels summed over instances, errors. */
int gq_bfs_batch(gq_handle id_queue, const gq_handle* frontier, uint32_t slots, uint32_t cluster_blocks,
                 const gq_bfs_instance* d_instances, const uint32_t* d_order, uint32_t ninst, void* d_workspace,
                 unsigned long long* d_stats, void* stream);

/* Tile-based wavefront ray tracing (Section V-B "Tile-based wavefront Ray
 * Tracing"): the W x H image is split into tiles_x x tiles_y tiles, each with
 * its own queue.  Primary rays are generated and enqueued per tile (the queue
 * item is the pixel index; the ray state lives in the workspace), then a
 * persistent kernel repeatedly dequeues a ray, traces one segment against all
 * spheres, shades it, and re-enqueues the scattered ray into the same tile's
 * queue, until a device work counter reaches zero.
 * Scene model (the same as the oracle's tracer): spheres with Lambertian
 * albedo; pinhole camera at cam looking along +z with image-plane half extents
 * scale_x, scale_y at distance 1; one sample per pixel centre; sky radiance
 * (1 - s) + s * (0.5, 0.7, 1.0), s = (d.y + 1) / 2, on a miss; at most
 * max_bounces scatterings; scattering direction normalize(n + p), p uniform in
 * the unit ball from a SplitMix64 stream keyed by (pixel, bounce, attempt).
 * fp32 without fused multiply-add, IEEE division and square root. */
typedef struct {
    uint32_t width, height, tiles_x, tiles_y, max_bounces, nspheres;
    float cam_x, cam_y, cam_z, scale_x, scale_y;
    uint32_t reserved;
    uint64_t seed;
    const float* d_centre;   /* nspheres x 3 (device) */
    const float* d_radius;   /* nspheres */
    const float* d_albedo;   /* nspheres x 3 */
} gq_rt_scene;

/* Device workspace gq_render needs (ray state, per-tile counters). */
int gq_render_workspace_bytes(const gq_rt_scene* scene, uint64_t* bytes);

/* Renders the scene into d_image (height x width x 3 float, row-major).
 *   tiles: host array of tiles_x * tiles_y queue handles of one kind, 4-byte
 *     elements, each of capacity >= the pixels of one tile (G-WFQ-YMC: pool
 *     cells >= that tile's segments, at most (max_bounces + 1) x its pixels),
 *     and max_threads >= the threads gq_render launches (it uses at most
 *     min(max_threads, resident threads)).  They are left empty.
 *   nspheres <= 8192 (the spheres are staged in shared memory).
 *   d_stats (nullable, 4 x uint64): segments traced, pixels finished, error
 *     flags (bit 0 idle wait expired, bit 1 a reserved dequeue found the queue
 *     empty), tiles.
 * Errors: GQ_ERR_INVALID, GQ_ERR_CUDA. */
int gq_render(const gq_handle* tiles, const gq_rt_scene* scene, void* d_workspace, float* d_image,
              unsigned long long* d_stats, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GQ_APPS_H */
