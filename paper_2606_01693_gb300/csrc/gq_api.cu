// libgq host API: workspace layout, create / destroy / reset, and the
// host-launched batch enqueue / dequeue kernels (declared in include/gq.h).
#include <cuda_runtime.h>
#include <algorithm>
#include <stdlib.h>
#include <string.h>

#include "gq_host.h"
#include "gq_ops.cuh"

using namespace gqd;

namespace {

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

uint32_t log2u(uint64_t x) {
    uint32_t r = 0;
    while ((1ull << r) < x) ++r;
    return r;
}

// Fills defaults and validates; returns GQ_OK or an error.
int resolve(int kind, uint64_t cap, uint32_t elem, uint32_t max_threads, const gq_options* in,
            gq_options* out) {
    if (kind < GQ_LFQ || kind > GQ_YMC) return GQ_ERR_INVALID;
    if (elem != 4 && elem != 8) return GQ_ERR_INVALID;
    if (max_threads < 1) return GQ_ERR_INVALID;
    gq_options o;
    memset(&o, 0, sizeof(o));
    if (in) o = *in;
    if (o.batch_width == 0) o.batch_width = 32;
    if (!is_pow2(o.batch_width) || o.batch_width > 32) return GQ_ERR_INVALID;
    if (o.backoff_ns > 1000000) return GQ_ERR_INVALID;
    if (o.due_wait == GQ_DUE_WAIT_OFF) o.due_wait = 0;
    else if (o.due_wait > 65536) return GQ_ERR_INVALID;
    if (kind == GQ_YMC) o.due_wait = 0;
    if (o.reserved_opt != 0 || o.patience_stretch > 4096) return GQ_ERR_INVALID;
    if (kind != GQ_WFQ) o.patience_stretch = 1;
    else if (o.patience_stretch == 0) o.patience_stretch = 64;
    if (kind == GQ_YMC) {
        if (cap < 2 || cap > (1ull << 40)) return GQ_ERR_INVALID;
        if (max_threads > (1u << 24) - 1) return GQ_ERR_TOO_MANY_THREADS;   // 24-bit thread field of cell references
        if (!o.patience_set) { o.patience_enq = 10; o.patience_deq = 10; }
        o.cycle_bits = 0;
        o.help_delay = 0;
        o.start_ticket = 0;
    } else {
        if (!is_pow2(cap) || cap < 2) return GQ_ERR_INVALID;
        const uint32_t maxbits = (kind == GQ_LFQ) ? 31 : 19;
        if (kind == GQ_LFQ && cap > (1ull << 31)) return GQ_ERR_INVALID;
        if (kind == GQ_WFQ && cap > (1ull << 23)) return GQ_ERR_INVALID;
        if (o.cycle_bits == 0) o.cycle_bits = maxbits;
        if (o.cycle_bits < 2 || o.cycle_bits > maxbits) return GQ_ERR_INVALID;
        if (o.start_ticket % (2 * cap)) return GQ_ERR_INVALID;
        if (kind == GQ_WFQ) {
            if (!o.patience_set) { o.patience_enq = 16; o.patience_deq = 64; }
            if (o.help_delay == 0) o.help_delay = 64;
            if (max_threads > (1u << 21) - 2) return GQ_ERR_TOO_MANY_THREADS;
            if (o.start_ticket >= (1ull << 43)) return GQ_ERR_INVALID;   // 43-bit Counter field
            // Lemma "Modular cycle correctness": sound iff R > D k / n + 6
            const double R = (double)(1ull << o.cycle_bits);
            if (!(R > (double)o.help_delay * (double)max_threads / (double)cap + 6.0))
                return GQ_ERR_TOO_MANY_THREADS;
        } else {
            o.patience_enq = o.patience_deq = 0;
            o.help_delay = 0;
        }
    }
    *out = o;
    return GQ_OK;
}

gq_layout make_layout(int kind, uint64_t cap, uint32_t elem, uint32_t max_threads) {
    gq_layout L;
    memset(&L, 0, sizeof(L));
    uint64_t off = 0;
    L.ctrl = off;
    off += kCtlLines * kCtlStride;
    if (kind == GQ_YMC) {
        const uint64_t cells = cap + 1;  // tickets start at 1; cell index = ticket
        // value and dequeue reference of a cell side by side in one 16-byte
        // pair (a dequeue reads one and CASes the other: one L2 sector);
        // enqueue references, touched only by slow enqueues, apart
        off = align_up(off, 256); L.cell_val = off; L.cell_deq = off + 8; off += cells * 16;
        off = align_up(off, 256); L.cell_enq = off; off += cells * 8;
        off = align_up(off, 256); L.ymc_rec = off; off += (uint64_t)max_threads * kYmcRecBytes;
    } else {
        off = align_up(off, 256); L.aq_slots = off; off += 2 * cap * 8;
        off = align_up(off, 256); L.fq_slots = off; off += 2 * cap * 8;
        off = align_up(off, 256); L.data = off; off += cap * elem;
        if (kind == GQ_WFQ) {
            off = align_up(off, 256); L.aq_rec = off; off += (uint64_t)max_threads * kWfqRecBytes;
            off = align_up(off, 256); L.fq_rec = off; off += (uint64_t)max_threads * kWfqRecBytes;
            off = align_up(off, 256); L.aq_owner = off; off += cap * 8;
            off = align_up(off, 256); L.fq_owner = off; off += cap * 8;
            off = align_up(off, 256); L.aq_helpc = off; off += (uint64_t)max_threads * 8;
            off = align_up(off, 256); L.fq_helpc = off; off += (uint64_t)max_threads * 8;
        }
    }
    L.total = align_up(off, 256);
    return L;
}

template <class P>
P* at(void* base, uint64_t off) {
    return reinterpret_cast<P*>(static_cast<char*>(base) + off);
}

// ---------------------------------------------------------------------------
// Reset kernels
// ---------------------------------------------------------------------------

// Control words: error, scratch, counters, thresholds.
__global__ void k_reset_ctrl(gq_dev q, u64 base_ticket) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *q.err = 0;
    for (int i = 0; i < 16; ++i) q.scratch[i] = 0;
    const u64 n = q.capacity;
    if (q.kind == GQ_YMC) {
        *q.ymc_tail = 1;
        *q.ymc_head = 1;
        *q.ymc_hw = 0;
        return;
    }
    if (q.kind == GQ_LFQ) {
        *q.aq.head = base_ticket;
        *q.aq.tail = base_ticket;
        *q.fq.head = base_ticket;
        *q.fq.tail = base_ticket + n;
    } else {
        *q.aq.head = wfq_global(base_ticket, 0);
        *q.aq.tail = wfq_global(base_ticket, 0);
        *q.fq.head = wfq_global(base_ticket, 0);
        *q.fq.tail = wfq_global(base_ticket + n, 0);
    }
    *q.aq.threshold = -1;
    *q.fq.threshold = (long long)(3 * n) - 1;
    if (q.kind == GQ_WFQ) {
        *q.aq.slow_pending = 0;
        *q.fq.slow_pending = 0;
    }
}

// Ring slots: aq empty (cycle c0 - 1); fq holds 0..n-1 at cycle c0.
__global__ void k_reset_slots(gq_dev q, u64 base_ticket) {
    const u64 n = q.capacity;
    const u32 order = q.log2n + 1;
    const u64 cmask = (1ull << q.cycle_bits) - 1;
    const u64 c0 = (base_ticket >> order) & cmask;
    const u64 cm1 = (c0 - 1) & cmask;
    const u64 cm2 = (c0 - 2) & cmask;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    // empty slots start "emptied in the previous cycle" (BOT, Note two cycles
    // back), the value an enqueue predicts
    for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * n; j += stride) {
        if (q.kind == GQ_LFQ) {
            q.aq.slots[j] = lfq_entry(cm1, kSafe, kBot);
            q.fq.slots[j] = (j < n) ? lfq_entry(c0, kSafe, (u32)j) : lfq_entry(cm1, kSafe, kBot);
        } else {
            q.aq.slots[j] = wfq_entry(cm2, cm1, 1, 1, kWBot);
            q.fq.slots[j] = (j < n) ? wfq_entry(cm1, c0, 1, 1, (u32)j) : wfq_entry(cm2, cm1, 1, 1, kWBot);
        }
    }
}

// G-WFQ-YMC cells: every <value, dequeue reference> pair = <BOT, BOT> (one
// 16-byte store per cell) and every enqueue reference = 0, grid-stride.  With
// `known`, only the cells used since the last reset: tickets below T and H
// (every fast path and slow enqueue takes its cell from them) and cells up to
// the slow dequeues' search mark; the rest are still clear.  The first reset
// of a workspace clears all of them.
__global__ void k_reset_cells(gq_dev q, bool known) {
    u64 cells = q.capacity + 1;
    if (known) {
        const u64 used = max(max(*q.ymc_tail, *q.ymc_head), *q.ymc_hw + 1);
        cells = min(cells, used);
    }
    ulonglong2* p = reinterpret_cast<ulonglong2*>(q.cell_val);
    const ulonglong2 e = make_ulonglong2(kVBot, kRefBot);
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < cells; j += stride) {
        p[j] = e;
        q.cell_enq[j] = 0;
    }
}

// ---------------------------------------------------------------------------
// Batch kernels
// ---------------------------------------------------------------------------
// Batch kernels.
// Enqueue batch: one item per lane per grid-stride step (coalesced 8-byte or
// 4-byte loads).  Tiles of two or four items per lane brought in by one 16-byte
// load each measured no better (G-LFQ 15.8 against 17.1, G-WFQ 15.7 against
// 16.0, G-WFQ-YMC 17.0 against 17.3 G items/s for 2^20 8-byte items) and were
// not kept.
template <class T, int KIND>
__global__ void __launch_bounds__(256) k_enqueue_batch(const __grid_constant__ gq_dev q, const T* __restrict__ items, u64 n,
                                                      int8_t* status, unsigned long long* num_ok) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    u64 ok = 0;
    u32 seq = 0;     // the thread's operation index (G-WFQ counts its help delay by it)
    for (u64 k = tid; k < n; k += stride, ++seq) {
        const T v = items[k];
        int s;
        if (KIND == GQ_YMC && sizeof(T) == 8 && (u64)v >= 0xFFFFFFFFFFFFFFFEull)
            s = GQ_ERR_RESERVED_VALUE;
        else
            s = queue_enqueue<T, KIND>(q, v, tid, nullptr, seq);
        if (status) status[k] = (int8_t)s;
        ok += (s == GQ_OK);
    }
    if (num_ok) warp_add_full(num_ok, ok);
}

// Dequeue batch: the warp works in tiles of 32 * V attempts (V = 16 / sizeof(T):
// two per lane for 8-byte items, four for 4-byte ones); its successful values
// are staged in shared memory in lane order, one lane takes the warp's output
// range with one fetch-and-add, and the warp copies the range out with
// consecutive lanes on consecutive elements (coalesced whatever its length);
// each lane's V statuses leave in one store.  A tail shorter than a tile, and a
// status buffer not aligned for that store, take one attempt per lane with a
// warp fetch-and-add per step.  Against one attempt per lane throughout:
// G-LFQ 24.0 against 23.0, G-WFQ-YMC 14.9 against 13.4, G-WFQ 15.9 against
// 16.4 G items/s (2^20 8-byte items; 4-byte: 23.5 / 14.5 / 14.9 against
// 23.0 / 13.4 / 16.4).
template <class T, int KIND>
__global__ void __launch_bounds__(256) k_dequeue_batch(const __grid_constant__ gq_dev q, T* __restrict__ out, u64 n, int8_t* status,
                                                      unsigned long long* pos) {
    constexpr u32 V = 16 / sizeof(T);
    __shared__ T stage[256 / 32][32 * V];
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 lane = threadIdx.x & 31;
    T* my = stage[threadIdx.x >> 5];
    const bool vec = !(reinterpret_cast<uintptr_t>(status) & (V - 1)) && (blockDim.x & 31) == 0;
    const u64 tiles = vec ? n / (32 * V) : 0;
    u32 seq = 0;     // the thread's operation index (G-WFQ counts its help delay by it)
    for (u64 w = tid >> 5; w < tiles; w += stride >> 5) {
        const u64 k0 = (w * 32 + lane) * V;
        T v[V];
        u32 packed = 0, got = 0;
#pragma unroll
        for (u32 j = 0; j < V; ++j) {
            const int s = queue_dequeue<T, KIND>(q, &v[got], tid, nullptr, seq++);
            got += (s == GQ_OK);
            packed |= (u32)(uint8_t)(int8_t)s << (8 * j);
        }
        if (status) {
            if (V == 4) *reinterpret_cast<u32*>(status + k0) = packed;
            else *reinterpret_cast<uint16_t*>(status + k0) = (uint16_t)packed;
        }
        // warp prefix sum of the success counts, then stage in lane order
        __syncwarp();
        u32 before = got;
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, before, o);
            if (lane >= (u32)o) before += y;
        }
        const u32 total = __shfl_sync(0xffffffffu, before, 31);
        before -= got;
        for (u32 j = 0; j < got; ++j) my[before + j] = v[j];
        u64 base = 0;
        if (lane == 0 && total) base = faa_rlx(reinterpret_cast<u64*>(pos), total);
        base = __shfl_sync(0xffffffffu, base, 0);
        __syncwarp();
        for (u32 e = lane; e < total; e += 32) out[base + e] = my[e];
        __syncwarp();
    }
    for (u64 k = tiles * 32 * V + tid; k < n; k += stride) {
        T v;
        const int s = queue_dequeue<T, KIND>(q, &v, tid, nullptr, seq++);
        if (status) status[k] = (int8_t)s;
        if (s == GQ_OK) {
            // compaction: the successful lanes of the warp take consecutive
            // output positions with one atomic, so their stores coalesce
            const u64 p = warp_faa<false>(reinterpret_cast<u64*>(pos), 1, 32);
            out[p] = v;
        }
    }
}

template <class T, int KIND>
int launch_batch(gq_queue* h, bool enq, void* buf, uint64_t n, int8_t* status,
                 unsigned long long* num_ok, cudaStream_t st) {
    int occ = 0;
    if (enq)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_enqueue_batch<T, KIND>, 256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dequeue_batch<T, KIND>, 256, 0);
    uint32_t grid = 0, block = 256;
    if (KIND != GQ_LFQ && h->dev.max_threads < 256) block = h->dev.max_threads;
    gq_grid_for(h, n, occ, block, &grid);
    if (enq) {
        k_enqueue_batch<T, KIND><<<grid, block, 0, st>>>(h->dev, static_cast<const T*>(buf), n, status, num_ok);
    } else {
        k_dequeue_batch<T, KIND><<<grid, block, 0, st>>>(h->dev, static_cast<T*>(buf), n, status, num_ok);
    }
    return gq_check_launch();
}

template <class T>
int dispatch_batch(gq_queue* h, bool enq, void* buf, uint64_t n, int8_t* status,
                   unsigned long long* num_ok, cudaStream_t st) {
    switch (h->dev.kind) {
        case GQ_LFQ: return launch_batch<T, GQ_LFQ>(h, enq, buf, n, status, num_ok, st);
        case GQ_WFQ: return launch_batch<T, GQ_WFQ>(h, enq, buf, n, status, num_ok, st);
        default: return launch_batch<T, GQ_YMC>(h, enq, buf, n, status, num_ok, st);
    }
}

}  // namespace

int gq_check_launch() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GQ_OK : GQ_ERR_CUDA;
}

void gq_grid_for(const gq_queue* q, uint64_t n_items, int occ, uint32_t block, uint32_t* grid_out) {
    uint64_t want = (n_items + block - 1) / block;
    uint64_t resident = (uint64_t)(occ > 0 ? occ : 1) * (uint64_t)(q->sm_count > 0 ? q->sm_count : 1);
    uint64_t g = want < resident ? want : resident;
    if (q->dev.kind != GQ_LFQ) {
        const uint64_t by_records = q->dev.max_threads / block;
        if (g > by_records) g = by_records;
    }
    if (g < 1) g = 1;
    *grid_out = (uint32_t)g;
}

extern "C" int gq_workspace_bytes(int kind, uint64_t capacity, uint32_t elem_bytes, uint32_t max_threads,
                                  const gq_options* opt, uint64_t* bytes) {
    if (!bytes) return GQ_ERR_INVALID;
    gq_options o;
    const int s = resolve(kind, capacity, elem_bytes, max_threads, opt, &o);
    if (s != GQ_OK) return s;
    *bytes = make_layout(kind, capacity, elem_bytes, max_threads).total;
    return GQ_OK;
}

extern "C" int gq_reset(gq_handle h, void* stream) {
    if (!h) return GQ_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gq_dev& d = h->dev;
    const uint64_t base = h->start_ticket + 2 * d.capacity;
    if (d.kind == GQ_YMC) {
        const uint64_t cells = d.capacity + 1;
        // eight 256-thread blocks per SM: one resident wave of the fill
        const uint64_t sms = h->sm_count > 0 ? (uint64_t)h->sm_count : 1;
        const uint64_t blocks = std::min<uint64_t>((cells + 255) / 256, 8 * sms);
        k_reset_cells<<<(uint32_t)blocks, 256, 0, st>>>(d, h->ymc_pool_known);
        if (cudaGetLastError() != cudaSuccess) return GQ_ERR_CUDA;
        h->ymc_pool_known = true;
        if (cudaMemsetAsync(d.ymc_rec, 0, (uint64_t)d.max_threads * kYmcRecBytes, st) != cudaSuccess)
            return GQ_ERR_CUDA;
    } else {
        const uint64_t slots = 2 * d.capacity;
        uint32_t grid = (uint32_t)((slots + 255) / 256);
        if (grid > 4096) grid = 4096;
        k_reset_slots<<<grid, 256, 0, st>>>(d, base);
        if (gq_check_launch() != GQ_OK) return GQ_ERR_CUDA;
        if (d.kind == GQ_WFQ) {
            if (cudaMemsetAsync(d.aq.rec, 0, (uint64_t)d.max_threads * kWfqRecBytes, st) != cudaSuccess ||
                cudaMemsetAsync(d.fq.rec, 0, (uint64_t)d.max_threads * kWfqRecBytes, st) != cudaSuccess ||
                cudaMemsetAsync(d.aq.owner, 0, d.capacity * 8, st) != cudaSuccess ||
                cudaMemsetAsync(d.fq.owner, 0, d.capacity * 8, st) != cudaSuccess ||
                cudaMemsetAsync(d.aq.helpc, 0, (uint64_t)d.max_threads * 8, st) != cudaSuccess ||
                cudaMemsetAsync(d.fq.helpc, 0, (uint64_t)d.max_threads * 8, st) != cudaSuccess)
                return GQ_ERR_CUDA;
        }
    }
    k_reset_ctrl<<<1, 1, 0, st>>>(d, base);
    return gq_check_launch();
}

extern "C" int gq_create(int kind, uint64_t capacity, uint32_t elem_bytes, uint32_t max_threads,
                         const gq_options* opt, void* d_workspace, void* stream, gq_handle* out) {
    if (!out) return GQ_ERR_INVALID;
    *out = nullptr;
    gq_options o;
    int s = resolve(kind, capacity, elem_bytes, max_threads, opt, &o);
    if (s != GQ_OK) return s;
    if (d_workspace && (reinterpret_cast<uintptr_t>(d_workspace) & 255)) return GQ_ERR_INVALID;
    gq_queue* h = new (std::nothrow) gq_queue;
    if (!h) return GQ_ERR_NOMEM;
    memset(h, 0, sizeof(*h));
    h->opt = o;
    h->lay = make_layout(kind, capacity, elem_bytes, max_threads);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess ||
        gq_run_kernels_init(h->device, h->smem_optin) != GQ_OK) {
        delete h;
        return GQ_ERR_CUDA;
    }
    if (d_workspace) {
        h->ws = d_workspace;
        h->owned = false;
    } else {
        if (cudaMalloc(&h->ws, h->lay.total) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return GQ_ERR_NOMEM;
        }
        h->owned = true;
    }
    h->start_ticket = o.start_ticket;
    gq_dev& d = h->dev;
    memset(&d, 0, sizeof(d));
    d.kind = kind;
    d.elem_bytes = elem_bytes;
    d.log2n = (kind == GQ_YMC) ? 0 : log2u(capacity);
    d.cycle_bits = o.cycle_bits;
    d.max_threads = max_threads;
    d.patience_enq = o.patience_enq;
    d.patience_deq = o.patience_deq;
    d.help_delay = o.help_delay;
    d.batch_width = o.batch_width;
    d.backoff_ns = o.backoff_ns;
    d.due_wait = o.due_wait;
    d.patience_stretch = o.patience_stretch;
    d.capacity = capacity;
    if (kind != GQ_YMC) {
        d.ring_order = d.log2n + 1;
        d.slot_mask = 2 * capacity - 1;
        d.cycle_mask = (1ull << o.cycle_bits) - 1;
        d.cycle_half = 1ull << (o.cycle_bits - 1);
        d.thr_reset = (int64_t)(3 * capacity) - 1;
    }
    void* b = h->ws;
    d.err = at<unsigned int>(b, h->lay.ctrl + kCtlErr * kCtlStride);
    d.scratch = at<unsigned long long>(b, h->lay.ctrl + kCtlScratch * kCtlStride);
    if (kind == GQ_YMC) {
        d.ymc_tail = at<unsigned long long>(b, h->lay.ctrl + kCtlYmcTail * kCtlStride);
        d.ymc_head = at<unsigned long long>(b, h->lay.ctrl + kCtlYmcHead * kCtlStride);
        d.ymc_hw = at<unsigned long long>(b, h->lay.ctrl + kCtlYmcHw * kCtlStride);
        d.cell_val = at<unsigned long long>(b, h->lay.cell_val);
        d.cell_enq = at<unsigned long long>(b, h->lay.cell_enq);
        d.cell_deq = at<unsigned long long>(b, h->lay.cell_deq);
        d.ymc_rec = at<unsigned long long>(b, h->lay.ymc_rec);
    } else {
        d.aq.head = at<unsigned long long>(b, h->lay.ctrl + kCtlAqHead * kCtlStride);
        d.aq.tail = at<unsigned long long>(b, h->lay.ctrl + kCtlAqTail * kCtlStride);
        d.aq.threshold = at<long long>(b, h->lay.ctrl + kCtlAqThr * kCtlStride);
        d.fq.head = at<unsigned long long>(b, h->lay.ctrl + kCtlFqHead * kCtlStride);
        d.fq.tail = at<unsigned long long>(b, h->lay.ctrl + kCtlFqTail * kCtlStride);
        d.fq.threshold = at<long long>(b, h->lay.ctrl + kCtlFqThr * kCtlStride);
        d.aq.slots = at<unsigned long long>(b, h->lay.aq_slots);
        d.fq.slots = at<unsigned long long>(b, h->lay.fq_slots);
        d.data = at<void>(b, h->lay.data);
        if (kind == GQ_WFQ) {
            d.aq.rec = at<unsigned long long>(b, h->lay.aq_rec);
            d.fq.rec = at<unsigned long long>(b, h->lay.fq_rec);
            d.aq.owner = at<unsigned long long>(b, h->lay.aq_owner);
            d.fq.owner = at<unsigned long long>(b, h->lay.fq_owner);
            d.aq.helpc = at<unsigned long long>(b, h->lay.aq_helpc);
            d.fq.helpc = at<unsigned long long>(b, h->lay.fq_helpc);
            d.aq.slow_pending = at<unsigned long long>(b, h->lay.ctrl + kCtlAqSlow * kCtlStride);
            d.fq.slow_pending = at<unsigned long long>(b, h->lay.ctrl + kCtlFqSlow * kCtlStride);
        }
    }
    s = gq_reset(h, stream);
    if (s != GQ_OK) {
        gq_destroy(h);
        return s;
    }
    *out = h;
    return GQ_OK;
}

extern "C" int gq_destroy(gq_handle h) {
    if (!h) return GQ_ERR_INVALID;
    int s = GQ_OK;
    if (h->owned || h->aux) {
        if (cudaDeviceSynchronize() != cudaSuccess) s = GQ_ERR_CUDA;
    }
    if (h->owned && cudaFree(h->ws) != cudaSuccess) s = GQ_ERR_CUDA;
    if (h->aux && cudaFree(h->aux) != cudaSuccess) s = GQ_ERR_CUDA;
    delete h;
    return s;
}

extern "C" int gq_enqueue_batch(gq_handle h, const void* d_items, uint64_t n, int8_t* d_status,
                                unsigned long long* d_num_ok, void* stream) {
    if (!h || (n && !d_items)) return GQ_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d_num_ok && cudaMemsetAsync(d_num_ok, 0, 8, st) != cudaSuccess) return GQ_ERR_CUDA;
    if (n == 0) return GQ_OK;
    void* buf = const_cast<void*>(d_items);
    return h->dev.elem_bytes == 4 ? dispatch_batch<unsigned int>(h, true, buf, n, d_status, d_num_ok, st)
                                  : dispatch_batch<unsigned long long>(h, true, buf, n, d_status, d_num_ok, st);
}

extern "C" int gq_dequeue_batch(gq_handle h, void* d_out, uint64_t n, int8_t* d_status,
                                unsigned long long* d_num_ok, void* stream) {
    if (!h || (n && !d_out)) return GQ_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the compaction counter: the caller's d_num_ok, else the library scratch word
    unsigned long long* pos = d_num_ok ? d_num_ok : h->dev.scratch;
    if (cudaMemsetAsync(pos, 0, 8, st) != cudaSuccess) return GQ_ERR_CUDA;
    if (n == 0) return GQ_OK;
    return h->dev.elem_bytes == 4 ? dispatch_batch<unsigned int>(h, false, d_out, n, d_status, pos, st)
                                  : dispatch_batch<unsigned long long>(h, false, d_out, n, d_status, pos, st);
}

extern "C" int gq_sync_status(gq_handle h, void* stream) {
    if (!h) return GQ_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return GQ_ERR_CUDA;
    unsigned int e = 0;
    if (cudaMemcpy(&e, h->dev.err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return GQ_ERR_CUDA;
    if (e) {
        const unsigned int z = 0;
        if (cudaMemcpy(h->dev.err, &z, 4, cudaMemcpyHostToDevice) != cudaSuccess) return GQ_ERR_CUDA;
        return -(int)e;
    }
    return GQ_OK;
}

extern "C" int gq_get_stats(gq_handle h, gq_stats* out) {
    if (!h || !out) return GQ_ERR_INVALID;
    unsigned long long w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (cudaMemcpy(w, h->dev.scratch, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return GQ_ERR_CUDA;
    *out = gq_stats{};
    out->slow_requests = w[kStatSlowRequests];
    out->helps = w[kStatHelps];
    out->global_cas_failures = w[kStatGlobalCasFail];
    out->slow_rounds_tail = w[kStatSlowRoundsTail];
    out->slow_rounds_head = w[kStatSlowRoundsHead];
    out->max_help_iterations = w[kStatMaxHelpIters];
    const gq_dev& d = h->dev;
    unsigned long long* src[4] = {d.aq.head, d.aq.tail, d.fq.head, d.fq.tail};
    if (d.kind == GQ_YMC) {
        src[0] = d.ymc_head;
        src[1] = d.ymc_tail;
        src[2] = src[3] = nullptr;
    }
    unsigned long long* dst[4] = {&out->aq_head, &out->aq_tail, &out->fq_head, &out->fq_tail};
    for (int i = 0; i < 4; ++i) {
        if (!src[i]) continue;
        if (cudaMemcpy(dst[i], src[i], 8, cudaMemcpyDeviceToHost) != cudaSuccess) return GQ_ERR_CUDA;
        if (d.kind == GQ_WFQ) *dst[i] >>= kGThrBits;          // the Counter field of a Global word
    }
    if (d.kind == GQ_WFQ) {
        if (cudaMemcpy(&out->aq_slow_pending, d.aq.slow_pending, 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&out->fq_slow_pending, d.fq.slow_pending, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return GQ_ERR_CUDA;
    }
    return GQ_OK;
}

extern "C" int gq_device_view(gq_handle h, gq_dev* out) {
    if (!h || !out) return GQ_ERR_INVALID;
    *out = h->dev;
    return GQ_OK;
}

extern "C" int gq_info(gq_handle h, uint64_t* workspace_bytes, int* library_owned) {
    if (!h) return GQ_ERR_INVALID;
    if (workspace_bytes) *workspace_bytes = h->lay.total;
    if (library_owned) *library_owned = h->owned ? 1 : 0;
    return GQ_OK;
}

extern "C" const char* gq_status_str(int s) {
    switch (s) {
        case GQ_OK: return "ok";
        case GQ_FULL: return "full";
        case GQ_EMPTY: return "empty";
        case GQ_ERR_INVALID: return "invalid argument";
        case GQ_ERR_NOMEM: return "out of device memory";
        case GQ_ERR_CUDA: return "CUDA runtime error";
        case GQ_ERR_TIMEOUT: return "bounded device loop expired";
        case GQ_ERR_POOL_EXHAUSTED: return "cell pool exhausted";
        case GQ_ERR_TOO_MANY_THREADS: return "too many threads for the records or cycle width";
        case GQ_ERR_RESERVED_VALUE: return "payload equals a reserved code";
        default: return "unknown status";
    }
}
