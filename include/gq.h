/*
 * gq.h -- C ABI of libgq, linearizable concurrent FIFO queues on one GB300 GPU.
 *
 * Three queue kinds from "Scalable Concurrent Queues for GPU" (Section III):
 *   GQ_LFQ  G-LFQ: bounded lock-free ring (Section III-B, Algorithm 1) with
 *           warp-batched ticket reservation (WaveFAA) and packed 64-bit slots
 *           <Cycle, Safe, Index>, wrapped in the index-indirection layer that
 *           moves indices, not payloads (Section III-B "Design goal").
 *   GQ_WFQ  G-WFQ: the same bounded ring with a cooperative slow path
 *           (Section III-C, Algorithm 2): patience-bounded fast path, fixed
 *           per-thread request records, Global <Counter, ThrIdx> and Local
 *           <Counter, INC, FIN> words and slots <Note, Cycle, Safe, Enq, Index>,
 *           every shared word updated by one 64-bit atomic.
 *   GQ_YMC  G-WFQ-YMC: Yang and Mellor-Crummey's wait-free queue with its
 *           segment list replaced by a pre-allocated cell pool addressed by
 *           arithmetic (Section III-A).  Unbounded in the FIFO sense: never FULL;
 *           the pool bounds the total number of tickets between resets.
 *
 * Conventions (all entry points):
 *   - Every function returns an int status: GQ_OK (0) or a negative gq_status.
 *     None throws, none aborts.  Argument errors are returned synchronously.
 *   - Pointers named d_* are CUDA device pointers; h_* are host pointers.
 *     The library never takes ownership of caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Queue work is enqueued asynchronously on that stream; calls on one stream
 *     execute in order.  Calls that overlap on different streams on one handle
 *     are concurrent queue operations and are linearizable, except gq_reset,
 *     which must not overlap any other call on the same handle.
 *   - Errors detected on the device (pool exhausted, bounded loop expired) are
 *     latched in a device error word; gq_sync_status() returns and clears it.
 *   - One handle belongs to one device (the current device at gq_create).
 */
#ifndef GQ_H
#define GQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { GQ_LFQ = 0, GQ_WFQ = 1, GQ_YMC = 2 } gq_kind;

typedef enum {
    GQ_OK = 0,
    GQ_FULL = 1,          /* per-item status: bounded queue full (enqueue)          */
    GQ_EMPTY = 2,         /* per-item status: queue empty (dequeue)                 */
    GQ_ERR_INVALID = -1,  /* bad argument                                           */
    GQ_ERR_NOMEM = -2,    /* device allocation failed                               */
    GQ_ERR_CUDA = -3,     /* a CUDA runtime call failed                             */
    GQ_ERR_TIMEOUT = -4,  /* a bounded device loop expired (latched on the device)  */
    GQ_ERR_POOL_EXHAUSTED = -5,   /* G-WFQ-YMC ran out of pool cells (latched)      */
    GQ_ERR_TOO_MANY_THREADS = -6, /* thread count exceeds records / cycle soundness */
    GQ_ERR_RESERVED_VALUE = -7    /* G-WFQ-YMC 64-bit payload equal to a reserved code */
} gq_status;

/* Opaque queue handle. */
typedef struct gq_queue* gq_handle;

#define GQ_DUE_WAIT_OFF 0xFFFFFFFFu

/* Creation options.  Zero-initialise and set what you need; 0 = default. */
typedef struct {
    /* Width of the cycle tag in bits.  Default 31 for G-LFQ (slot <Cycle 31 |
     * Safe 1 | Index 32>), 19 for G-WFQ (<Note 19 | Cycle 19 | Safe | Enq |
     * Index 24>).  Smaller values exist to test cycle wrap-around. */
    uint32_t cycle_bits;
    /* G-WFQ fast-path attempts before publishing a slow-path request
     * (Section III-C "patience"); UINT32_MAX = never go slow is not allowed.
     * Default 16 (enqueue) and 64 (dequeue).  0 forces every operation onto
     * the slow path (test mode). */
    uint32_t patience_enq, patience_deq;
    uint32_t patience_set;   /* set to 1 to make patience_enq/deq = 0 meaningful */
    /* G-WFQ help delay D: a thread inspects one peer record every D
     * operations (Section III-C).  Default 64. */
    uint32_t help_delay;
    /* WaveFAA batch width: lanes are grouped into aligned groups of this many
     * (a power of two, 1..32); each group reserves its tickets with one
     * fetch-and-add.  Default 32 (the whole warp, Algorithm 1). */
    uint32_t batch_width;
    /* Back-off: a ring operation whose ticket attempt failed sleeps this many
     * nanoseconds (__nanosleep) before taking the next ticket.  Default 0. */
    uint32_t backoff_ns;
    /* Due-install wait of the ring queues (G-LFQ, G-WFQ): a dequeuer whose
     * slot still holds an older cycle's empty entry while Tail is already past
     * its ticket (the enqueuer holding that ticket is about to install)
     * re-reads the slot up to this many times, about 32 ns apart, before
     * ruling it out.  0 = default: no waiting (the plain TryDeq of
     * Algorithm 1; waiting measured no better on the benchmark workloads);
     * GQ_DUE_WAIT_OFF = no waiting either.  At most 65536. */
    uint32_t due_wait;
    /* G-WFQ patience stretch: a ring operation that has used its patience
     * while requests of the same ring are already waiting on the slow path
     * keeps trying the fast path, up to patience * patience_stretch attempts
     * in all, before it publishes its own request (each attempt still bounded,
     * so operations stay wait-free with the larger bound).  1 = off (the
     * plain Section III-C rule).  0 = default 64.  At most 4096. */
    uint32_t patience_stretch;
    uint32_t reserved_opt;   /* must be 0 */
    /* Initial value of every ticket counter (tests of counter wrap-around).
     * Must be a multiple of 2 * capacity.  Default 0. */
    uint64_t start_ticket;
} gq_options;

/* POD view of a queue, passed by value to user kernels (see gq_device.cuh). */
typedef struct {
    unsigned long long* head;       /* ticket counter (G-WFQ: <Counter, ThrIdx>)   */
    unsigned long long* tail;
    long long* threshold;           /* empty-detection counter                     */
    unsigned long long* slots;      /* 2n packed 64-bit entries                    */
    unsigned long long* rec;        /* G-WFQ request records (NULL for G-LFQ)      */
    unsigned long long* owner;      /* G-WFQ: record id that enqueues each index    */
    unsigned long long* helpc;      /* G-WFQ: per-thread help cursor <peer, countdown> */
    unsigned long long* slow_pending; /* G-WFQ: requests published, not yet retired */
} gq_ring_view;

typedef struct {
    int32_t kind;                   /* gq_kind                                     */
    uint32_t elem_bytes;            /* 4 or 8                                      */
    uint32_t log2n;                 /* ring queues: capacity n = 1 << log2n        */
    uint32_t cycle_bits;
    uint32_t max_threads;           /* number of per-thread records                */
    uint32_t patience_enq, patience_deq, help_delay;
    uint32_t batch_width;           /* WaveFAA group width                          */
    uint32_t ring_order;            /* log2(2n)                                    */
    uint32_t backoff_ns;            /* sleep after a failed ticket attempt          */
    uint32_t due_wait;              /* due-install polls of a ring dequeuer (0: none) */
    uint32_t patience_stretch;      /* G-WFQ: fast attempts x this while the slow path is busy */
    uint32_t reserved1;
    uint64_t capacity;              /* ring: n; YMC: pool cells                    */
    uint64_t slot_mask;             /* 2n - 1                                      */
    uint64_t cycle_mask;            /* R - 1, R = 2^cycle_bits                     */
    uint64_t cycle_half;            /* R / 2                                       */
    int64_t thr_reset;              /* 3n - 1                                      */
    gq_ring_view aq, fq;            /* allocated-index ring, free-index ring       */
    void* data;                     /* payload array of n elements                 */
    unsigned int* err;              /* latched device error word                   */
    unsigned long long* scratch;    /* library scratch line (batch counters)       */
    /* G-WFQ-YMC */
    unsigned long long* ymc_tail;   /* T counter                                   */
    unsigned long long* ymc_head;   /* H counter                                   */
    unsigned long long* cell_val;   /* pool cell values: cell i at cell_val[2 i]   */
    unsigned long long* cell_enq;   /* pool cell enqueue-request references        */
    unsigned long long* cell_deq;   /* dequeue references: cell i at cell_deq[2 i]
                                       (= cell_val[2 i + 1], one 16-byte pair)     */
    unsigned long long* ymc_rec;    /* per-thread handles and requests             */
    unsigned long long* ymc_hw;     /* highest cell a slow dequeue's candidate search
                                       visited since the last reset (with T and H it
                                       bounds the cells gq_reset clears)            */
} gq_dev;

/* Bytes of device workspace gq_create needs for this configuration, so a caller
 * (for example PyTorch's allocator) can own the memory.
 *   kind: gq_kind.  capacity: ring queues: logical capacity n, a power of two,
 *   2 <= n <= 2^31 (G-LFQ) or 2^23 (G-WFQ); G-WFQ-YMC: number of pool cells
 *   (tickets between resets), >= 2.  elem_bytes: 4 or 8.  max_threads: number
 *   of device threads that may operate on the queue at once (G-WFQ and
 *   G-WFQ-YMC keep one record per thread; G-LFQ ignores it but requires >= 1).
 * Writes *bytes.  Errors: GQ_ERR_INVALID. */
int gq_workspace_bytes(int kind, uint64_t capacity, uint32_t elem_bytes, uint32_t max_threads,
                       const gq_options* opt, uint64_t* bytes);

/* Creates an empty queue.  d_workspace: NULL lets the library cudaMalloc and
 * own the workspace; otherwise a device buffer of gq_workspace_bytes() bytes,
 * 256-byte aligned, owned by the caller and kept alive until gq_destroy.
 * opt may be NULL.  Initialisation runs on `stream`; the queue is usable by
 * later work on that stream (or after synchronising it).
 * G-WFQ checks the cycle-tag soundness bound of its modular-cycle lemma,
 * R > D*k/n + 6 with R = 2^cycle_bits, D = help delay, k = max_threads, and
 * returns GQ_ERR_TOO_MANY_THREADS if it fails.
 * Errors: GQ_ERR_INVALID, GQ_ERR_NOMEM, GQ_ERR_CUDA, GQ_ERR_TOO_MANY_THREADS. */
int gq_create(int kind, uint64_t capacity, uint32_t elem_bytes, uint32_t max_threads,
              const gq_options* opt, void* d_workspace, void* stream, gq_handle* out);

/* Releases the handle and any library-owned device memory (after a device
 * synchronisation).  NULL is GQ_ERR_INVALID. */
int gq_destroy(gq_handle h);

/* Returns the queue to its freshly created empty state, asynchronously on
 * `stream`, and clears the device error word.  Must not overlap other calls on
 * the handle.  G-WFQ-YMC: clears only the pool cells used since the previous
 * reset (the first reset after gq_create clears the whole pool), so its cost
 * follows the tickets taken, not the pool size. */
int gq_reset(gq_handle h, void* stream);

/* Enqueues d_items[0..n) (elem_bytes each), one attempt per item, concurrently
 * (order among the items of one call is unspecified; successive calls on one
 * stream are ordered).  d_status[i] (nullable) receives GQ_OK or GQ_FULL (or a
 * negative error); *d_num_ok (nullable) is overwritten with the number of
 * successes.  G-WFQ-YMC with 8-byte items rejects the two reserved payloads
 * 2^64-1 and 2^64-2 with per-item status GQ_ERR_RESERVED_VALUE. */
int gq_enqueue_batch(gq_handle h, const void* d_items, uint64_t n, int8_t* d_status,
                     unsigned long long* d_num_ok, void* stream);

/* Attempts n dequeues concurrently.  Successful values are written compacted to
 * d_out[0..num_ok) in an unspecified order; d_status[i] (nullable) receives
 * GQ_OK or GQ_EMPTY for attempt i; *d_num_ok (nullable) is overwritten with
 * the number of successes.  d_out must hold n elements. */
int gq_dequeue_batch(gq_handle h, void* d_out, uint64_t n, int8_t* d_status,
                     unsigned long long* d_num_ok, void* stream);

/* Synchronises `stream`, then returns and clears the latched device error
 * (GQ_OK if none).  A CUDA error on the stream is returned as GQ_ERR_CUDA. */
int gq_sync_status(gq_handle h, void* stream);

/* Copies the POD device view (for user kernels using gq_device.cuh). */
int gq_device_view(gq_handle h, gq_dev* out);

/* Rare-path event counters of a queue since its last reset (G-WFQ slow path,
 * Algorithm 2), and its ticket counters.  Synchronous device-to-host copies;
 * read them while no kernel uses the queue.
 *   slow_requests        requests published on the slow path
 *   helps                peer requests helped
 *   global_cas_failures  lost CASes on a Global word in SlowFAA
 *   slow_rounds_tail/_head  successful SlowFAA rounds on the Tail / Head
 *                        Global words of both rings (each advances that
 *                        word's Counter by exactly one)
 *   max_help_iterations  the most SlowFAA iterations one helper spent on one
 *                        request
 *   aq_head .. fq_tail   current ticket counters: G-LFQ the raw words, G-WFQ
 *                        the Counter field of each Global word, G-WFQ-YMC H
 *                        and T in aq_head / aq_tail (fq_* zero)
 *   aq_slow_pending, fq_slow_pending  G-WFQ with a patience stretch above
 *                        1: requests published on each ring and not yet
 *                        retired (0 between kernels; otherwise zero) */
typedef struct {
    unsigned long long slow_requests;
    unsigned long long helps;
    unsigned long long global_cas_failures;
    unsigned long long slow_rounds_tail;
    unsigned long long slow_rounds_head;
    unsigned long long max_help_iterations;
    unsigned long long aq_head, aq_tail, fq_head, fq_tail;
    unsigned long long aq_slow_pending, fq_slow_pending;
} gq_stats;
int gq_get_stats(gq_handle h, gq_stats* out);

/* Workspace size and whether the library owns it. */
int gq_info(gq_handle h, uint64_t* workspace_bytes, int* library_owned);

/* FIFO round trip that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (for
 * example code running while another framework owns the whole device
 * allocator, or a service that must not allocate after start-up).
 * It enqueues d_items[0..n) into a G-LFQ whose entire workspace lives in one
 * file-scope static device array of the library (2.6 MB per device, held
 * until the process exits), then attempts n dequeues; the dequeued values are
 * written compacted to d_out[0..*d_num_out) in an unspecified order and
 * *d_num_out is overwritten with their number (n when nothing fails).  Same
 * result as gq_create + gq_enqueue_batch + gq_dequeue_batch on a G-LFQ of
 * capacity >= n, without gq_create's allocation.
 *   A device-side failure inside the call (a bounded wait that expired) is
 *   reported only through the count: the call returns before its kernels
 *   run and the next call clears the array's error word, so *d_num_out < n
 *   is the sign of it (with nothing failing every item comes back).
 *   n <= 65536 (the array's capacity); larger n returns GQ_ERR_INVALID before
 *   any work is launched.  d_items, d_out: n 8-byte elements; d_num_out: one
 *   8-byte counter; all caller-owned device memory.
 * Calls no cudaMalloc, cudaFree or allocating routine.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and caches it; make that first call before any stream
 * capture.  Every call shares the array and re-initialises it; calls that
 * overlap on the GPU race and must be serialised by the caller.
 * Errors: GQ_ERR_INVALID, GQ_ERR_CUDA. */
int gq_fifo_static_roundtrip(const unsigned long long* d_items, uint64_t n, unsigned long long* d_out,
                             unsigned long long* d_num_out, void* stream);

/* Static description of a status code. */
const char* gq_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* GQ_H */
