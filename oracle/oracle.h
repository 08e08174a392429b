/*
 * Oracle for the concurrent FIFO queues of "Scalable Concurrent Queues for GPU"
 * (G-LFQ, G-WFQ, G-WFQ-YMC).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this library: only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header or constant with the CUDA library.
 *
 * What the queues compute is, by the paper's correctness claim (Section IV and
 * the linearizability theorems of Section III), exactly the behaviour of a
 * sequential FIFO queue: every concurrent history must be explainable by some
 * sequential FIFO history that respects real-time order.  The oracle is that
 * definition written out, plus checkers that test recorded GPU histories
 * against it:
 *   - orc_seqfifo_run      sequential FIFO specification (Section IV footnote:
 *                          enqueue appends, dequeue returns the head or EMPTY)
 *   - orc_linearizable     brute-force Wing & Gong linearizability search over a
 *                          recorded history {proc, op, arg, ret, call, end}
 *                          (Section IV "Linearizability via Porcupine")
 *   - orc_check_log        exactly-once / no out-of-range token / per-producer
 *                          order checks (Section IV "Device-side FIFO conformance")
 *   - orc_check_tickets    ticket checks: an item's dequeue has its enqueue's
 *                          ticket, tickets are distinct and follow real time
 *   - orc_mutex_run        a mutex-guarded std::deque running the same seeded
 *                          schedule on N host threads (the timed CPU baseline)
 *   - orc_bfs              textbook sequential breadth-first search (Section V-B
 *                          level-synchronous BFS computes the same distances)
 *
 * Status codes used throughout: 0 = OK, 1 = FULL, 2 = EMPTY.
 * Operation kinds: 1 = enqueue, 0 = dequeue, 255 = no operation.
 */
#ifndef GQ_ORACLE_H
#define GQ_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Sequential FIFO of capacity `cap` (0 = unbounded).  Applies ops in order.
 * kind[i]: 1 enqueue val[i], 0 dequeue.  Writes status[i] and, for dequeues
 * that succeed, out[i] (0 otherwise).  Final contents (front first) go to
 * `final_contents` (may be NULL) and their count to *final_size. */
void orc_seqfifo_run(uint64_t cap, const uint8_t* kind, const uint64_t* val, int64_t n,
                     int8_t* status, uint64_t* out, uint64_t* final_contents, int64_t* final_size);

/* Linearizability of a tiny history (n <= 63 operations).
 * op[i]: 1 enqueue, 0 dequeue.  val[i]: enqueue argument or dequeue result.
 * status[i]: 0 OK, 1 FULL (enqueue only), 2 EMPTY (dequeue only).
 * call[i] <= end[i]: timestamps; op a precedes op b iff end[a] < call[b].
 * cap: queue capacity, 0 = unbounded.  A FULL enqueue is accepted at a point
 * where size >= cap - (number of other operations overlapping it), the bounded
 * queue's relaxed full condition (indices held by in-flight operations).
 * Returns 1 linearizable, 0 not linearizable, -1 search budget exceeded,
 * -2 bad input. */
int orc_linearizable(int64_t n, const uint8_t* op, const uint64_t* val, const int8_t* status,
                     const uint64_t* call, const uint64_t* end, uint64_t cap, int64_t max_states);

/* Report of orc_check_log. */
typedef struct {
    int64_t enq_ok, enq_full, deq_ok, deq_empty;
    int64_t drained;
    int64_t violations;      /* total number of violations found */
    int32_t first_kind;      /* 0 none, 1 multiset mismatch, 2 per-consumer order,
                                3 overtaking (a drained token older than a dequeued one
                                of the same producer), 4 drained order, 5 bad token,
                                6 bad status; orc_check_tickets: 7 a ticket
                                wider than `bits`, 8 a dequeue's ticket differs from
                                its value's enqueue ticket (or the value was never
                                enqueued), 9 two enqueues (dequeues) share a ticket,
                                10 enqueue tickets against real-time order,
                                11 dequeue tickets against real-time order */
    int32_t pad;
    int64_t first_index;     /* flat index (i * T + t) or drained index of the first violation */
} orc_report;

/* Checks a run log of T logical threads with up to K ops each, op-major
 * (entry i * T + t is op i of thread t).
 *   kind: 1 enqueue, 0 dequeue, 255 none; status: 0 OK, 1 FULL, 2 EMPTY;
 *   val:  enqueue payload, or the value a successful dequeue returned.
 *   drained[0..n_drained): items left in the queue after the run, in the
 *   order a single-threaded drain returned them (FIFO order).
 * Tokens encode (producer, seq): producer = tok >> prod_shift,
 * seq = ((tok & seq_mask) - seq_bias).  Returns the number of violations. */
int64_t orc_check_log(int64_t T, int64_t K, const uint8_t* kind, const int8_t* status,
                      const uint64_t* val, const uint64_t* drained, int64_t n_drained,
                      int32_t prod_shift, uint64_t seq_mask, uint64_t seq_bias, orc_report* rep);

/* Ticket checks on a run log of n operations (flat, any order): kind 1
 * enqueue / 0 dequeue / other none, status 0 = OK, val the token, ticket the
 * recorded ticket of a successful op (a `bits`-bit counter value, may wrap),
 * call / end (both nullable) globaltimer stamps.  Checks that every dequeue's
 * ticket equals its value's enqueue ticket, that no two enqueues (dequeues)
 * share one, and, with stamps, that an operation has a larger ticket than
 * every operation of its kind that ended before it was called.  rep counts
 * enq_ok / deq_ok and the violations.  Returns the number of violations, -1
 * on bad arguments. */
int64_t orc_check_tickets(int64_t n, const uint8_t* kind, const int8_t* status, const uint64_t* val,
                          const uint64_t* ticket, const uint64_t* call, const uint64_t* end, int32_t bits,
                          orc_report* rep);

/* Mutex-guarded std::deque running a workload on `nthreads` host threads; host
 * thread h runs logical threads t = h, h + nthreads, ...
 *   mode 0 (pairs):  each logical thread does K enqueue-then-dequeue pairs,
 *                    payload (t << 16) | s  (32-bit tokens)
 *   mode 1 (mixed):  op i of thread t is an enqueue iff bit (t*K+i) of `sched`
 *                    is set; payload (t << 32) | (seq + 1)
 *   mode 2 (split):  threads t < producers only enqueue, the others only
 *                    dequeue; thread t does ops_of[t] operations
 * cap: capacity (0 = unbounded).  counts[4] = enq_ok, enq_full, deq_ok, deq_empty.
 * Returns elapsed wall-clock seconds of the threaded region. */
double orc_mutex_run(int32_t mode, int64_t T, int64_t K, const uint64_t* sched, int64_t producers,
                     const int64_t* ops_of, uint64_t cap, int32_t nthreads, int64_t* counts);

/* Sequential BFS from `src` on a CSR graph; dist[v] = hop count or 0xFFFFFFFF.
 * Returns the number of reached vertices. */
int64_t orc_bfs(int64_t n, const uint64_t* offsets, const uint32_t* adj, uint32_t src, uint32_t* dist);

/* Sequential CPU ray tracer (Section V-B wavefront ray tracing computes the
 * same per-pixel radiance; the queue only schedules the ray segments).
 * Scene and camera as read from the workload description: spheres with
 * Lambertian albedo, pinhole camera at cam looking along +z (image plane
 * x = (2 (px + 0.5) / W - 1) * scale_x, y = (1 - 2 (py + 0.5) / H) * scale_y,
 * z = 1), one sample at each pixel centre, sky radiance
 * (1 - s) + s * (0.5, 0.7, 1.0) with s = (d.y + 1) / 2 on a miss, at most
 * max_bounces scatterings (a hit after the last scattering contributes 0).
 * Scattering direction normalize(n + p), p uniform in the unit ball by
 * rejection from [-1, 1]^3 with 24-bit uniforms
 * u = (splitmix64(seed, ((pixel * 16 + bounce) * 64 + attempt) * 4 + axis) >> 40) * 2^-24,
 * at most 32 attempts (else p = 0); normalize falls back to n when
 * |n + p|^2 <= 1e-12.  Nearest hit with t > 1e-4; equal t: lower sphere id.
 * fp32 throughout, no fused multiply-add, IEEE division and square root. */
typedef struct {
    int32_t width, height, max_bounces, nspheres;
    float cam_x, cam_y, cam_z, scale_x, scale_y;
    uint64_t seed;
    const float* centre;   /* nspheres x 3 */
    const float* radius;   /* nspheres */
    const float* albedo;   /* nspheres x 3 */
} orc_rt_scene;

/* Radiance of the m listed pixels (index py * width + px) into rgb[3 m];
 * segments[m] (nullable) receives the number of traced segments per pixel.
 * Uses `threads` host threads. */
void orc_render_pixels(const orc_rt_scene* scene, const int64_t* pixels, int64_t m, float* rgb,
                       int32_t* segments, int32_t threads);

#ifdef __cplusplus
}
#endif
#endif
