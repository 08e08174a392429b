/*
 * gq_serve.h -- C ABI of the BFS serving runtime built on the queues.
 *
 * Requests (graph id, source vertex) arrive at given times; each asks for the
 * hop distances of a level-synchronous BFS (Section V-B) on one graph of a
 * resident pool.  Two ways to serve them on one GPU:
 *   GQ_SERVE_PERSISTENT   one persistent device scheduler: idle thread-block
 *                         clusters poll (bounded) the request ring in mapped
 *                         pinned memory for the next ticket the host has
 *                         published (system-scope release / acquire), take it
 *                         with a CAS on a device claim counter, run the BFS on
 *                         the cluster's own pair of frontier queues, and mark
 *                         the ring entry done (system-scope release), which the
 *                         host polls.  Requests that arrive while others run
 *                         are taken as soon as a cluster frees up.
 *   GQ_SERVE_PER_REQUEST  the plain form: one gq_bfs launch per request
 *                         (the whole GPU, one request at a time), in arrival
 *                         order on one stream; completion is an event the host
 *                         polls.
 *   GQ_SERVE_ADAPTIVE     per-request launches while few requests wait; when
 *                         switch_backlog launched requests are still pending,
 *                         the persistent scheduler is started (after them, on
 *                         the same stream) and takes the following requests;
 *                         after 0.5 ms with nothing to do it is stopped and
 *                         per-request launches resume.
 * Gangs (persistent scheduler, gang_clusters > 1): a cluster takes a ticket
 * only once the host has published it, so idle clusters hold none.  The
 * cluster that takes a request on a large graph offers a gang (one at a time
 * on the GPU); clusters with nothing published to take join it for up to
 * 20 us, and the gang runs the request's BFS on the taker's queues with a
 * barrier of its own between levels (thread 0 of each cluster meets the others
 * on a device counter, bounded wait).  Requests on small graphs, or taken
 * while another gang is forming, run on one cluster.
 * Admission (both modes, first come first served): a request is published or
 * launched only when its device state fits in the budget; it waits on the host
 * otherwise.  A request's state is counted as its graph's CSR (8 (n + 1) +
 * 4 m bytes), its distance array (4 n bytes) and two frontier queues of its own
 * size (gq_workspace_bytes of the kind at capacity max(n, 4096) rounded up to
 * a power of two; G-WFQ-YMC: 4 n + 2^18 cells), with per-thread records for
 * the threads that may run it: a cluster, a gang of clusters for a graph that
 * forms gangs, one gq_bfs grid per request; adaptive mode counts the larger.
 * Latency = the time the host sees the request done minus its arrival time.
 * A request's distances do not depend on what else is being served: BFS hop
 * counts are unique, whatever the claim order.
 */
#ifndef GQ_SERVE_H
#define GQ_SERVE_H

#include <stdint.h>

#include "gq_apps.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { GQ_SERVE_PERSISTENT = 0, GQ_SERVE_PER_REQUEST = 1, GQ_SERVE_ADAPTIVE = 2 };

typedef struct {
    int32_t kind;                   /* frontier queue kind (gq_kind)                           */
    uint32_t mode;                  /* GQ_SERVE_*                                              */
    uint32_t slots;                 /* persistent / adaptive: clusters serving at once; 0 = all */
                                    /* that fit on the GPU at once (fewer if fewer fit)       */
    uint32_t cluster_blocks;        /* persistent / adaptive: blocks of 256 threads per cluster: 1, 2, 4, */
                                    /* 8 or 16 (16 is above the portable cluster size)         */
    uint64_t budget_bytes;          /* admission budget for per-request state                  */
    double wait_limit_s;            /* bound on any one wait of the device scheduler for its   */
                                    /* next request, and on the host's wait for progress;     */
                                    /* 0 = 30 s                                                */
    uint32_t ngraphs;
    uint32_t nrequests;
    const gq_bfs_instance* graphs;  /* host array [ngraphs]; n, d_offsets, d_adj are used      */
    const uint32_t* req_graph;      /* host arrays [nrequests]                                 */
    const uint32_t* req_src;
    const double* req_arrival_s;    /* arrival offsets from the start, seconds, non-decreasing */
    uint32_t* const* req_out;       /* nullable host array [nrequests] of device pointers; a  */
                                    /* non-null entry receives that request's distances (n    */
                                    /* uint32, GQ_BFS_UNREACHED where unreached); null entries */
                                    /* (or a null array) use scratch from a device arena of at */
                                    /* most budget_bytes                                      */
    uint32_t switch_backlog;        /* adaptive: pending launches that start the scheduler;   */
                                    /* 0 = 8                                                   */
    uint32_t gang_clusters;         /* persistent / adaptive: most clusters that serve one     */
                                    /* request together (a gang; at most 64, and at most the  */
                                    /* slots); 1 = one cluster per request; 0 = default 16     */
    uint32_t gang_min_vertices;     /* requests on graphs of at least this many vertices form  */
                                    /* gangs; 0 = default 2^17                                 */
    uint32_t reserved;              /* must be 0                                               */
} gq_serve_config;

typedef struct {
    double* latency_s;              /* caller array [nrequests], filled                        */
    double wall_s;                  /* first arrival to last completion                        */
    uint64_t peak_state_bytes;      /* largest admitted state counted at one time              */
    uint64_t admission_waits;       /* requests that had arrived but waited for budget         */
    uint64_t edges_scanned;         /* by the persistent scheduler, over all its requests      */
    uint64_t persistent_requests;   /* requests the persistent scheduler served                */
    uint32_t slots_used;            /* clusters of the persistent scheduler (0: not used)      */
    int32_t status;                 /* GQ_OK or the first error                                */
    uint64_t gang_requests;         /* requests the persistent scheduler served with a gang    */
                                    /* of two or more clusters                                 */
} gq_serve_result;

/* Serves every request and returns when all are done (synchronous; uses the
 * current device; creates and frees its own queues, arena, ring and stream).
 * res->latency_s must hold nrequests doubles.
 * Errors: GQ_ERR_INVALID (bad configuration, a graph id or source out of
 * range, a request whose state exceeds the budget), GQ_ERR_NOMEM, GQ_ERR_CUDA,
 * GQ_ERR_TIMEOUT (a bounded wait expired), or an error latched by a queue. */
int gq_serve(const gq_serve_config* cfg, gq_serve_result* res);

#ifdef __cplusplus
}
#endif
#endif /* GQ_SERVE_H */
