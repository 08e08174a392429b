/*
 * gq_drivers.h -- C ABI of libgq's workload drivers: the kernels that run the
 * paper's micro-benchmarks and correctness checks on a queue.
 *
 *   gq_run          one kernel in which every thread executes a fixed operation
 *                   program (Section V-A micro-benchmarks, with the fixed
 *                   operation counts of the workloads measured here):
 *                     GQ_RUN_PAIRS  "balanced kernel": each thread repeats
 *                                   {enqueue; dequeue} `ops / 2` times;
 *                     GQ_RUN_MIXED  each op is an enqueue or a dequeue as a
 *                                   seeded bit schedule says (50/50 interleaved);
 *                     GQ_RUN_SPLIT  "split producer/consumer kernel": the first
 *                                   `producers` threads only enqueue, the rest
 *                                   only dequeue; `total_ops` split evenly.
 *                   Optionally records, per operation, the status, the value,
 *                   globaltimer timestamps (Section IV: device-recorded histories
 *                   {proc, op, arg, ret, call, end}) and the ticket.
 *   gq_run_sequence a single device thread applies an explicit op list (the
 *                   sequential bit-exactness test against the FIFO specification).
 *   gq_drain        a single device thread dequeues until EMPTY (FIFO order of
 *                   the items left behind).
 *   gq_atomic_peak  same-box L2 atomic micro-benchmarks: the roofline
 *                   denominators (single-address fetch-add, warp-coalesced and
 *                   scattered multi-address CAS).
 *
 * Payload tokens written by gq_run: 8-byte queues (tid << 32) | (seq + 1)
 * (Section IV's conformance token); 4-byte queues (tid << 16) | seq, which
 * requires threads <= 65536 and fewer than 65536 enqueues per thread.
 * seq counts the thread's enqueue attempts, starting at 0.
 *
 * Output arrays are op-major: entry (i * threads + t) is op i of thread t.
 * Conventions as in gq.h (int status returns, asynchronous on `stream`).
 */
#ifndef GQ_DRIVERS_H
#define GQ_DRIVERS_H

#include <stdint.h>

#include "gq.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { GQ_RUN_PAIRS = 0, GQ_RUN_MIXED = 1, GQ_RUN_SPLIT = 2 };

#define GQ_VIEW_BYTES 512   /* upper bound of sizeof(gq_dev) */

/* Counter slots accumulated (atomically added) by gq_run into d_counts[8]. */
enum {
    GQ_CNT_ENQ_OK = 0, GQ_CNT_ENQ_FULL = 1, GQ_CNT_DEQ_OK = 2, GQ_CNT_DEQ_EMPTY = 3,
    GQ_CNT_SUM_ENQ = 4,   /* sum (mod 2^64) of successfully enqueued tokens */
    GQ_CNT_SUM_DEQ = 5,   /* sum (mod 2^64) of successfully dequeued values */
    GQ_CNT_ERRORS = 6,    /* operations that returned a negative status     */
    GQ_CNT_RESERVED = 7
};

/* Event counters of the counting kernels (gq_run / gq_run_multi with
 * d_opcount), summed over all operations.  They measure what each successful
 * operation costs in L2 atomics against the algorithmic count (Section III-B:
 * one slot CAS per ring operation and one counter fetch-add per warp batch).
 * Slow-path internals are not included (gq_get_stats counts those). */
enum {
    GQ_OC_TICKETS = 0,    /* tickets taken (per lane)                                     */
    GQ_OC_FAA = 1,        /* counter fetch-and-adds issued (one per WaveFAA batch)        */
    GQ_OC_CAS = 2,        /* CAS attempts on slots / cells: install, repair, claim        */
    GQ_OC_CAS_FAIL = 3,   /* ... of which failed                                          */
    GQ_OC_RMW = 4,        /* other slot RMWs (the ring Consume's atomic OR)               */
    GQ_OC_THRESHOLD = 5,  /* Threshold RMWs (reset, decrement; one per group of lanes)     */
    GQ_OC_CATCHUP = 6,    /* Tail catch-ups of EMPTY dequeues (one per group of lanes)     */
    GQ_OC_BURNED = 7,     /* tickets given up without an install or an item (RETRY/EMPTY) */
    GQ_OC_LOADS = 8,      /* first loads of a ticket's slot or cell                        */
    GQ_OC_SLOW = 9,       /* slow-path requests (G-WFQ, G-WFQ-YMC)                          */
    GQ_OC_SPIN = 10,      /* further reads of an empty slot / cell whose enqueuer is due     */
    GQ_OC_MARKED = 11,    /* G-WFQ-YMC: cells marked unusable by a dequeuer                 */
    GQ_OC_N = 12
};

typedef struct {
    uint32_t mode;            /* GQ_RUN_*                                                  */
    uint32_t threads;         /* logical threads (one device thread each)                 */
    uint32_t block;           /* threads per block (multiple of 32, <= 256)                */
    uint32_t ops;             /* PAIRS/MIXED: operations per thread (PAIRS: even)          */
    uint32_t producers;       /* SPLIT: threads [0, producers) enqueue                     */
    uint32_t delay_ns;        /* > 0: each op waits a pseudo-random 0..delay_ns-1 ns first */
    uint64_t total_ops;       /* SPLIT: operations over all threads                        */
    const uint64_t* d_sched;  /* MIXED: bit (t * ops + i) set = op i of t is an enqueue   */
    int8_t* d_status;         /* nullable, op-major                                        */
    uint64_t* d_val;          /* nullable, op-major: enqueued token / dequeued value       */
    uint64_t* d_call;         /* nullable, op-major: globaltimer before the op             */
    uint64_t* d_end;          /* nullable, op-major: globaltimer after the op              */
    unsigned long long* d_counts; /* 8 words, added to (the caller zeroes them)           */
    uint64_t* d_ticket;       /* nullable, op-major, test recorder: a successful op's     */
                              /* ticket in the allocated-index ring aq (G-LFQ, G-WFQ;     */
                              /* G-WFQ: the 43-bit Global counter value) or its cell     */
                              /* (G-WFQ-YMC); 2^64-1 for an op that did not succeed.     */
                              /* An item's enqueue and the dequeue that returns it have  */
                              /* the same ticket, and of two enqueues (dequeues) that do */
                              /* not overlap in time the earlier has the smaller one.    */
                              /* Non-null selects a separate recording kernel.           */
    unsigned long long* d_opcount; /* nullable, GQ_OC_N words, added to: event counts of   */
                              /* every operation's fast path (GQ_OC_*).  Non-null selects */
                              /* a separate counting kernel (never the timed one); not   */
                              /* combinable with d_ticket.                               */
} gq_run_args;

/* Launches the driver kernel.  For SPLIT, ops
 * per thread = ceil(total_ops / threads) bounds the op-major arrays; threads
 * t >= total_ops mod threads do floor(total_ops / threads) ops.  G-WFQ /
 * G-WFQ-YMC need threads <= max_threads.  A G-LFQ grid of at least two waves
 * of 768 threads per SM is launched with unused dynamic shared memory that
 * holds residency to 768 threads per SM (fewer requests queue at the hot L2
 * lines; the results do not depend on it).
 * Errors: GQ_ERR_INVALID, GQ_ERR_TOO_MANY_THREADS, GQ_ERR_CUDA. */
int gq_run(gq_handle h, const gq_run_args* args, void* stream);

/* One device thread applies op i = (d_kind[i] == 1 ? enqueue d_val[i] : dequeue)
 * for i in [0, n), writing d_status[i] and d_out[i] (dequeued value or 0). */
int gq_run_sequence(gq_handle h, const uint8_t* d_kind, const uint64_t* d_val, uint64_t n,
                    int8_t* d_status, uint64_t* d_out, void* stream);

/* One device thread dequeues until EMPTY or `max` items; values (zero-extended
 * to 8 bytes) go to d_out in dequeue order and their number to *d_count. */
int gq_drain(gq_handle h, uint64_t* d_out, uint64_t max, unsigned long long* d_count, void* stream);

enum {
    GQ_PEAK_SAME_ADDR_FAA = 0,   /* one lane per warp, fetch-add on one shared word      */
    GQ_PEAK_COALESCED_CAS = 1,   /* each warp CASes 32 consecutive words (2 lines)       */
    GQ_PEAK_SCATTERED_CAS = 2,   /* each lane CASes a pseudo-random word                 */
    GQ_PEAK_COALESCED_LOAD = 3,  /* each warp loads 32 consecutive words (reference)     */
    GQ_PEAK_SPREAD_FAA = 4,      /* one lane per warp, fetch-add on one of 16 counters    */
                                 /* 4096 bytes apart (warp id mod 16)                    */
    GQ_PEAK_PACKED_FAA = 5       /* the same on 16 counters 128 bytes apart              */
};

/* Runs `iters` rounds of the pattern on a grid of blocks x threads over the
 * caller's buffer d_buf[0..buf_words) (L2-resident when small enough).  Each
 * round is one atomic (or load) per participating lane.  d_sink receives a
 * value derived from the results so the work cannot be elided.
 * Time it with events on `stream`; ops = blocks * threads * iters (FAA patterns: / 32).
 * The two 16-counter patterns need buf_words >= 16 * 512 (SPREAD) or 16 * 16 (PACKED); they show
 * whether hot counters at that spacing share an L2 slice (their rates do not add up if they do). */
int gq_atomic_peak(int pattern, uint32_t blocks, uint32_t threads, uint32_t iters,
                   unsigned long long* d_buf, uint64_t buf_words, unsigned long long* d_sink,
                   void* stream);

/* WaveFAA probe (Algorithm 1 WaveFAA; Lemma "WaveFAA preserves ticket order").
 * Thread t of a grid of `threads` threads (blocks of 256) takes one ticket if
 * d_take[t] is non-zero: lanes with d_take[t] == 1 on counter d_counters[0],
 * lanes with 2 on d_counters[1] (lanes of one warp may mix both: they are
 * grouped by counter address), with batch width `width` (1 .. 32, a power of
 * two).  The ticket goes to d_tickets[t] (others get ~0).  Test hook: the
 * tickets of each counter must be exactly 0 .. count-1, and within a warp's
 * group of `width` lanes the lanes that share a counter get consecutive tickets
 * in lane order.  Errors: GQ_ERR_INVALID, GQ_ERR_CUDA. */
int gq_wavefaa_probe(const uint8_t* d_take, uint32_t threads, uint32_t width, unsigned long long* d_counters,
                     unsigned long long* d_tickets, void* stream);

/* ---- many independent queues in one persistent launch (batched form) ----
 *
 * gq_multi_prepare copies the device views of Q queues (same kind and element
 * size) into d_views (Q * sizeof(gq_dev) bytes of device memory; sizeof(gq_dev)
 * never exceeds GQ_VIEW_BYTES).  `tune` (nullable) overrides, in every copied
 * view, the WaveFAA batch width (if non-zero), the back-off, when
 * tune->patience_set is 1 G-WFQ's patience, and when tune->help_delay is
 * non-zero G-WFQ's help delay D (GQ_ERR_TOO_MANY_THREADS if some queue would
 * leave its cycle-tag bound R > D k / n + 6), and when tune->due_wait is
 * non-zero the ring queues' due-install wait (GQ_DUE_WAIT_OFF: none); this is
 * how the autotuner tries settings without recreating queues.  Asynchronous on
 * `stream`. */
int gq_multi_prepare(const gq_handle* queues, uint32_t nqueues, void* d_views, const gq_options* tune,
                     void* stream);

typedef struct {
    uint32_t nqueues;
    uint32_t threads_per_queue;    /* logical threads of each queue, multiple of 32       */
    uint32_t producers_per_queue;  /* the first this many of each queue's threads enqueue */
    uint32_t block;                /* threads per block, multiple of 32, <= 256           */
    uint32_t blocks;               /* grid size; 0 = every resident block                  */
    uint32_t kind, elem_bytes;     /* must match the views                                 */
    uint32_t reserved;
    uint64_t ops_per_queue;        /* split evenly over the queue's threads                */
    unsigned long long* d_counts;  /* 8 words, added to (GQ_CNT_* layout)                  */
    /* Recorder (nullable; d_ticket non-null selects a separate recording kernel
     * and then needs d_status and d_val): op i of logical thread t of queue q
     * goes to entry (q * K + i) * threads_per_queue + t with
     * K = ceil(ops_per_queue / threads_per_queue): its status, its value (the
     * enqueued token, or the dequeued value, 0 if none) and its ticket (as in
     * gq_run_args.d_ticket).  Entries of ops a thread does not run are left
     * untouched. */
    int8_t* d_status;
    uint64_t* d_val;
    uint64_t* d_ticket;
    unsigned long long* d_opcount; /* nullable, GQ_OC_N words: counting kernel (as gq_run) */
} gq_multi_args;

/* Producer/consumer split workload on every queue of d_views at once: logical
 * thread t of queue q enqueues tokens ((q * threads_per_queue + t) << 32) |
 * (seq + 1) if t < producers_per_queue, else dequeues; ops_per_queue split
 * evenly.  A persistent grid strides over the logical threads; each logical
 * thread runs its operations in order and uses record id t in queue q.
 * Errors: GQ_ERR_INVALID, GQ_ERR_CUDA. */
int gq_run_multi(const void* d_views, const gq_multi_args* args, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GQ_DRIVERS_H */
