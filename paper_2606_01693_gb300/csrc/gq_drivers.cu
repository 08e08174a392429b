// Workload drivers (include/gq_drivers.h): the micro-benchmark kernels of
// Section V-A and the recorders used by the correctness checks of Section IV.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "../../include/gq_drivers.h"
#include "gq_host.h"
#include "gq_ops.cuh"

using namespace gqd;

static_assert(sizeof(gq_dev) <= GQ_VIEW_BYTES, "gq_dev must fit GQ_VIEW_BYTES");

namespace {

constexpr int kOcStaticBytes = kOcN * kOcMaxBlock * (int)sizeof(u32);

struct RunK {
    u32 mode, threads, ops, producers, delay_ns;
    u64 total_ops;
    const u64* sched;
    int8_t* status;
    u64* val;
    u64* call;
    u64* end;
    unsigned long long* counts;
    u64* ticket;
    unsigned long long* opcnt;
};

__device__ __forceinline__ u32 mix32(u32 a, u32 b) {
    u32 h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    return h;
}

// 256 threads x 4 blocks per SM caps registers at 64: the rarely taken slow
// paths of G-WFQ / G-WFQ-YMC may spill instead of halving occupancy.
// REC: also record each successful operation's ticket (a.ticket); CNT: count
// the events of every operation (a.opcnt, see gq_atomics.cuh).  Both are
// separate instantiations, so the timed kernels carry none of it.
template <class T, int KIND, bool REC, bool CNT>
__global__ void __launch_bounds__(256, 4) k_run(const __grid_constant__ gq_dev q, const __grid_constant__ RunK a) {
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    oc_begin<CNT>();
    u32 c_enq_ok = 0, c_full = 0, c_deq_ok = 0, c_empty = 0, c_err = 0;   // per-thread counts
    u64 s_enq = 0, s_deq = 0;
    if (t < a.threads) {
        u32 nops = a.ops;
        bool producer = true;
        if (a.mode == GQ_RUN_SPLIT) {
            nops = (u32)(a.total_ops / a.threads) + (t < (u32)(a.total_ops % a.threads) ? 1u : 0u);
            producer = t < a.producers;
        }
        u32 seq = 0;
        for (u32 i = 0; i < nops; ++i) {
            bool is_enq;
            if (a.mode == GQ_RUN_PAIRS) {
                is_enq = !(i & 1u);
            } else if (a.mode == GQ_RUN_MIXED) {
                const u64 j = (u64)t * a.ops + i;
                is_enq = (a.sched[j >> 6] >> (j & 63)) & 1ull;
            } else {
                is_enq = producer;
            }
            if (a.delay_ns) __nanosleep(mix32(t, i) % a.delay_ns);
            const u64 tc = a.call ? globaltimer() : 0;
            int s;
            u64 v = 0;
            u64 tk = ~0ull;
            u64* const tkp = REC ? &tk : nullptr;
            if constexpr (KIND == GQ_YMC) {
                // two operations with little in common: separate branches
                if (is_enq) {
                    v = (sizeof(T) == 4) ? (((u64)t << 16) | seq) : (((u64)t << 32) | (u64)(seq + 1));
                    ++seq;
                    s = queue_enqueue<T, KIND, false, CNT>(q, (T)v, t, tkp);
                    if (s == GQ_OK) { ++c_enq_ok; s_enq += v; }
                    else if (s == GQ_FULL) ++c_full;
                    else ++c_err;
                } else {
                    T x = 0;
                    s = queue_dequeue<T, KIND, false, CNT>(q, &x, t, tkp);
                    v = (s == GQ_OK) ? (u64)x : 0;
                    if (s == GQ_OK) { ++c_deq_ok; s_deq += v; }
                    else if (s == GQ_EMPTY) ++c_empty;
                    else ++c_err;
                }
            } else {
                // mirrored operations: enqueue and dequeue lanes run together
                if (is_enq) {
                    v = (sizeof(T) == 4) ? (((u64)t << 16) | seq) : (((u64)t << 32) | (u64)(seq + 1));
                    ++seq;
                }
                T x = (T)v;
                s = queue_op<T, KIND, CNT>(q, is_enq, &x, t, tkp, i);
                if (is_enq) {
                    if (s == GQ_OK) { ++c_enq_ok; s_enq += v; }
                    else if (s == GQ_FULL) ++c_full;
                    else ++c_err;
                } else {
                    v = (s == GQ_OK) ? (u64)x : 0;
                    if (s == GQ_OK) { ++c_deq_ok; s_deq += v; }
                    else if (s == GQ_EMPTY) ++c_empty;
                    else ++c_err;
                }
            }
            const u64 j = (u64)i * a.threads + t;
            if (a.end) a.end[j] = globaltimer();
            if (a.call) a.call[j] = tc;
            if (a.status) a.status[j] = (int8_t)s;
            if (a.val) a.val[j] = v;
            if (REC) a.ticket[j] = (s == GQ_OK) ? tk : ~0ull;
        }
    }
    warp_add_full(&a.counts[GQ_CNT_ENQ_OK], c_enq_ok);
    warp_add_full(&a.counts[GQ_CNT_ENQ_FULL], c_full);
    warp_add_full(&a.counts[GQ_CNT_DEQ_OK], c_deq_ok);
    warp_add_full(&a.counts[GQ_CNT_DEQ_EMPTY], c_empty);
    warp_add_full(&a.counts[GQ_CNT_SUM_ENQ], s_enq);
    warp_add_full(&a.counts[GQ_CNT_SUM_DEQ], s_deq);
    warp_add_full(&a.counts[GQ_CNT_ERRORS], c_err);
    oc_end<CNT>(a.opcnt);
}

template <class T, int KIND>
__global__ void k_sequence(const __grid_constant__ gq_dev q, const uint8_t* kind, const u64* val, u64 n, int8_t* status, u64* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (u64 i = 0; i < n; ++i) {
        int s;
        u64 r = 0;
        if (kind[i] == 1) {
            s = queue_enqueue<T, KIND>(q, (T)val[i], 0);
        } else {
            T x = 0;
            s = queue_dequeue<T, KIND>(q, &x, 0);
            if (s == GQ_OK) r = (u64)x;
        }
        status[i] = (int8_t)s;
        out[i] = r;
    }
}

template <class T, int KIND>
__global__ void k_drain(const __grid_constant__ gq_dev q, u64* out, u64 max, unsigned long long* count) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    u64 k = 0;
    while (k < max) {
        T x = 0;
        const int s = queue_dequeue<T, KIND>(q, &x, 0);
        if (s != GQ_OK) break;
        out[k++] = (u64)x;
    }
    *count = k;
}

template <class T, int KIND, bool REC, bool CNT>
int launch_run(gq_queue* h, const RunK& a, u32 block, cudaStream_t st) {
    const u32 grid = (a.threads + block - 1) / block;
    // G-LFQ with more threads than ring capacity, on a grid of at least two
    // waves at 768 threads per SM: reserve (unused) dynamic shared memory so
    // that only 768 threads per SM are resident.  Oversubscribed rings run
    // near full or near empty, where the threads meet on the Head / Tail /
    // Threshold lines and on each other's slots; fewer of them at once give
    // up fewer tickets.  The blocks beyond the first wave start as earlier
    // ones finish.  A ring with a slot for every thread (the balanced
    // workloads) runs faster uncapped, and so do G-WFQ, G-WFQ-YMC and a grid
    // that would fit in one uncapped wave.
    size_t smem = 0;
    if (KIND == GQ_LFQ && (u64)a.threads > h->dev.capacity) {
        const u32 per_sm = block >= 768 ? 1u : 768u / block;
        if ((u64)grid >= 2ull * per_sm * (u64)h->sm_count && h->smem_per_sm > 0) {
            // a block's footprint halfway between sm/(per_sm + 1) and sm/per_sm:
            // per_sm blocks fit, one more does not
            const int sm_bytes = h->smem_per_sm;
            const int foot = (sm_bytes / (int)per_sm + sm_bytes / (int)(per_sm + 1)) / 2;
            const int stat = CNT ? kOcStaticBytes : 0;     // the counting kernel's static table
            smem = (size_t)std::min(std::max(foot - h->smem_reserved - stat, 0), h->smem_optin - stat);
        }
    }
    k_run<T, KIND, REC, CNT><<<grid, block, smem, st>>>(h->dev, a);
    return gq_check_launch();
}

template <class T, bool REC, bool CNT>
cudaError_t allow_run_smem(int bytes) {
    // static shared memory (the counting kernel's table) counts against the same per-block limit
    const int stat = CNT ? kOcStaticBytes : 0;
    return cudaFuncSetAttribute(k_run<T, GQ_LFQ, REC, CNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes - stat);
}

template <class T, bool REC, bool CNT>
int dispatch_run_rec(gq_queue* h, const RunK& a, u32 block, cudaStream_t st) {
    switch (h->dev.kind) {
        case GQ_LFQ: return launch_run<T, GQ_LFQ, REC, CNT>(h, a, block, st);
        case GQ_WFQ: return launch_run<T, GQ_WFQ, REC, CNT>(h, a, block, st);
        default: return launch_run<T, GQ_YMC, REC, CNT>(h, a, block, st);
    }
}

template <class T>
int dispatch_run(gq_queue* h, const RunK& a, u32 block, cudaStream_t st) {
    if (a.opcnt) return dispatch_run_rec<T, false, true>(h, a, block, st);
    return a.ticket ? dispatch_run_rec<T, true, false>(h, a, block, st)
                    : dispatch_run_rec<T, false, false>(h, a, block, st);
}

template <class T>
int dispatch_seq(gq_queue* h, const uint8_t* kind, const u64* val, u64 n, int8_t* status, u64* out,
                 cudaStream_t st) {
    switch (h->dev.kind) {
        case GQ_LFQ: k_sequence<T, GQ_LFQ><<<1, 1, 0, st>>>(h->dev, kind, val, n, status, out); break;
        case GQ_WFQ: k_sequence<T, GQ_WFQ><<<1, 1, 0, st>>>(h->dev, kind, val, n, status, out); break;
        default: k_sequence<T, GQ_YMC><<<1, 1, 0, st>>>(h->dev, kind, val, n, status, out); break;
    }
    return gq_check_launch();
}

template <class T>
int dispatch_drain(gq_queue* h, u64* out, u64 max, unsigned long long* count, cudaStream_t st) {
    switch (h->dev.kind) {
        case GQ_LFQ: k_drain<T, GQ_LFQ><<<1, 1, 0, st>>>(h->dev, out, max, count); break;
        case GQ_WFQ: k_drain<T, GQ_WFQ><<<1, 1, 0, st>>>(h->dev, out, max, count); break;
        default: k_drain<T, GQ_YMC><<<1, 1, 0, st>>>(h->dev, out, max, count); break;
    }
    return gq_check_launch();
}

struct MultiK {
    u32 nq, tpq, ppq, kmax;
    u64 opq;
    unsigned long long* counts;
    int8_t* status;
    u64* val;
    u64* ticket;
    unsigned long long* opcnt;
};

// REC: record each operation's status, value and ticket at entry
// ((queue * kmax) + op) * tpq + thread; CNT: count events (a.opcnt).  Both are
// separate instantiations of the timed kernel.
// The lanes of one warp may work on different queues at the same time (a lane
// whose logical thread finished early moves on to the next queue while the
// others still run), so WaveFAA groups lanes by counter address (MATCH): one
// fetch-and-add must never hand one queue's tickets to another queue's lanes.
template <class T, int KIND, bool REC, bool CNT>
__global__ void __launch_bounds__(256, 4) k_run_multi(const gq_dev* __restrict__ views, const __grid_constant__ MultiK a) {
    const u64 total = (u64)a.nq * a.tpq;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    oc_begin<CNT>();
    u32 c_enq_ok = 0, c_full = 0, c_deq_ok = 0, c_empty = 0, c_err = 0;
    u64 s_enq = 0, s_deq = 0;
    for (u64 L = (u64)blockIdx.x * blockDim.x + threadIdx.x; L < total; L += stride) {
        const u32 qi = (u32)(L / a.tpq), t = (u32)(L % a.tpq);
        const gq_dev& q = views[qi];
        const u32 nops = (u32)(a.opq / a.tpq) + (t < (u32)(a.opq % a.tpq) ? 1u : 0u);
        u64 tk = ~0ull;
        u64* const tkp = REC ? &tk : nullptr;
        if (t < a.ppq) {
            for (u32 i = 0; i < nops; ++i) {
                const u64 v = (sizeof(T) == 4) ? ((L << 16) | i) : ((L << 32) | (u64)(i + 1));
                const int s = queue_enqueue<T, KIND, true, CNT>(q, (T)v, t, tkp, i);
                if (s == GQ_OK) { ++c_enq_ok; s_enq += v; }
                else if (s == GQ_FULL) ++c_full;
                else ++c_err;
                if constexpr (REC) {
                    const u64 j = ((u64)qi * a.kmax + i) * a.tpq + t;
                    a.status[j] = (int8_t)s;
                    a.val[j] = v;
                    a.ticket[j] = (s == GQ_OK) ? tk : ~0ull;
                }
            }
        } else {
            for (u32 i = 0; i < nops; ++i) {
                T x = 0;
                const int s = queue_dequeue<T, KIND, true, CNT>(q, &x, t, tkp, i);
                if (s == GQ_OK) { ++c_deq_ok; s_deq += (u64)x; }
                else if (s == GQ_EMPTY) ++c_empty;
                else ++c_err;
                if constexpr (REC) {
                    const u64 j = ((u64)qi * a.kmax + i) * a.tpq + t;
                    a.status[j] = (int8_t)s;
                    a.val[j] = (s == GQ_OK) ? (u64)x : 0;
                    a.ticket[j] = (s == GQ_OK) ? tk : ~0ull;
                }
            }
        }
    }
    warp_add_full(&a.counts[GQ_CNT_ENQ_OK], c_enq_ok);
    warp_add_full(&a.counts[GQ_CNT_ENQ_FULL], c_full);
    warp_add_full(&a.counts[GQ_CNT_DEQ_OK], c_deq_ok);
    warp_add_full(&a.counts[GQ_CNT_DEQ_EMPTY], c_empty);
    warp_add_full(&a.counts[GQ_CNT_SUM_ENQ], s_enq);
    warp_add_full(&a.counts[GQ_CNT_SUM_DEQ], s_deq);
    warp_add_full(&a.counts[GQ_CNT_ERRORS], c_err);
    oc_end<CNT>(a.opcnt);
}

template <class T, int KIND, bool REC, bool CNT>
int launch_multi_k(const gq_dev* views, const gq_multi_args& g, cudaStream_t st) {
    MultiK a;
    a.nq = g.nqueues;
    a.tpq = g.threads_per_queue;
    a.ppq = g.producers_per_queue;
    a.kmax = (uint32_t)((g.ops_per_queue + g.threads_per_queue - 1) / g.threads_per_queue);
    a.opq = g.ops_per_queue;
    a.counts = g.d_counts;
    a.status = g.d_status;
    a.val = reinterpret_cast<u64*>(g.d_val);
    a.ticket = reinterpret_cast<u64*>(g.d_ticket);
    a.opcnt = g.d_opcount;
    uint32_t blocks = g.blocks;
    const uint64_t need = ((uint64_t)g.nqueues * g.threads_per_queue + g.block - 1) / g.block;
    if (blocks == 0) {
        int dev = 0, sms = 0, occ = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_run_multi<T, KIND, REC, CNT>, (int)g.block, 0) !=
                cudaSuccess)
            return GQ_ERR_CUDA;
        blocks = (uint32_t)(occ > 0 ? occ : 1) * (uint32_t)sms;
    }
    if (blocks > need) blocks = (uint32_t)need;
    k_run_multi<T, KIND, REC, CNT><<<blocks, g.block, 0, st>>>(views, a);
    return gq_check_launch();
}

template <class T, int KIND>
int launch_multi(const gq_dev* views, const gq_multi_args& g, cudaStream_t st) {
    if (g.d_opcount) return launch_multi_k<T, KIND, false, true>(views, g, st);
    if (g.d_ticket) return launch_multi_k<T, KIND, true, false>(views, g, st);
    return launch_multi_k<T, KIND, false, false>(views, g, st);
}

__global__ void k_multi_tune(gq_dev* views, u32 n, u32 width, u32 backoff, u32 set_patience, u32 pe, u32 pd,
                             u32 delay, u32 due, u32 stretch) {
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (width) views[i].batch_width = width;
    views[i].backoff_ns = backoff;
    if (set_patience && views[i].kind == GQ_WFQ) {
        views[i].patience_enq = pe;
        views[i].patience_deq = pd;
    }
    if (delay && views[i].kind == GQ_WFQ) views[i].help_delay = delay;
    if (stretch && views[i].kind == GQ_WFQ) views[i].patience_stretch = stretch;
    // due-install wait: 0 keeps the queue's own, GQ_DUE_WAIT_OFF turns it off
    if (due && views[i].kind != GQ_YMC) views[i].due_wait = (due == GQ_DUE_WAIT_OFF) ? 0u : due;
}

}  // namespace

extern "C" int gq_multi_prepare(const gq_handle* queues, uint32_t nqueues, void* d_views, const gq_options* tune,
                                void* stream) {
    if (!queues || !nqueues || !d_views) return GQ_ERR_INVALID;
    for (uint32_t i = 0; i < nqueues; ++i)
        if (!queues[i] || queues[i]->dev.kind != queues[0]->dev.kind ||
            queues[i]->dev.elem_bytes != queues[0]->dev.elem_bytes || queues[i]->device != queues[0]->device)
            return GQ_ERR_INVALID;
    if (tune && tune->batch_width && (tune->batch_width > 32 || (tune->batch_width & (tune->batch_width - 1))))
        return GQ_ERR_INVALID;
    if (tune && tune->due_wait > 65536 && tune->due_wait != GQ_DUE_WAIT_OFF) return GQ_ERR_INVALID;
    if (tune && (tune->patience_stretch > 4096 || tune->reserved_opt != 0)) return GQ_ERR_INVALID;
    // a new G-WFQ help delay D must keep every queue within its modular-cycle bound R > D k / n + 6
    if (tune && tune->help_delay && queues[0]->dev.kind == GQ_WFQ)
        for (uint32_t i = 0; i < nqueues; ++i) {
            const gq_dev& d = queues[i]->dev;
            const double R = (double)(1ull << d.cycle_bits);
            if (!(R > (double)tune->help_delay * (double)d.max_threads / (double)d.capacity + 6.0))
                return GQ_ERR_TOO_MANY_THREADS;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gq_dev* v = static_cast<gq_dev*>(d_views);
    for (uint32_t i = 0; i < nqueues; ++i)
        if (cudaMemcpyAsync(v + i, &queues[i]->dev, sizeof(gq_dev), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return GQ_ERR_CUDA;
    if (tune) {
        k_multi_tune<<<(nqueues + 255) / 256, 256, 0, st>>>(v, nqueues, tune->batch_width, tune->backoff_ns,
                                                            tune->patience_set, tune->patience_enq, tune->patience_deq,
                                                            tune->help_delay, tune->due_wait,
                                                            tune->patience_stretch);
        return gq_check_launch();
    }
    return GQ_OK;
}

extern "C" int gq_run_multi(const void* d_views, const gq_multi_args* args, void* stream) {
    if (!d_views || !args || !args->d_counts || !args->nqueues) return GQ_ERR_INVALID;
    const gq_multi_args& g = *args;
    if (g.threads_per_queue == 0 || (g.threads_per_queue & 31) || g.block == 0 || g.block > 256 || (g.block & 31) ||
        g.producers_per_queue > g.threads_per_queue || g.kind > GQ_YMC || (g.elem_bytes != 4 && g.elem_bytes != 8))
        return GQ_ERR_INVALID;
    if (g.elem_bytes == 4 && ((uint64_t)g.nqueues * g.threads_per_queue > 65536 ||
                              g.ops_per_queue / g.threads_per_queue >= 65536))
        return GQ_ERR_INVALID;
    if (g.d_ticket && (!g.d_status || !g.d_val || g.d_opcount)) return GQ_ERR_INVALID;
    if (g.ops_per_queue / g.threads_per_queue >= (1ull << 32)) return GQ_ERR_INVALID;
    const gq_dev* v = static_cast<const gq_dev*>(d_views);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (g.elem_bytes == 4) {
        switch (g.kind) {
            case GQ_LFQ: return launch_multi<unsigned int, GQ_LFQ>(v, g, st);
            case GQ_WFQ: return launch_multi<unsigned int, GQ_WFQ>(v, g, st);
            default: return launch_multi<unsigned int, GQ_YMC>(v, g, st);
        }
    }
    switch (g.kind) {
        case GQ_LFQ: return launch_multi<unsigned long long, GQ_LFQ>(v, g, st);
        case GQ_WFQ: return launch_multi<unsigned long long, GQ_WFQ>(v, g, st);
        default: return launch_multi<unsigned long long, GQ_YMC>(v, g, st);
    }
}

int gq_run_kernels_init(int device, int smem_optin) {
    static std::atomic<int> done[64];
    if (device >= 0 && device < 64 && done[device].load(std::memory_order_acquire)) return GQ_OK;
    if (allow_run_smem<unsigned int, false, false>(smem_optin) != cudaSuccess ||
        allow_run_smem<unsigned int, true, false>(smem_optin) != cudaSuccess ||
        allow_run_smem<unsigned int, false, true>(smem_optin) != cudaSuccess ||
        allow_run_smem<unsigned long long, false, false>(smem_optin) != cudaSuccess ||
        allow_run_smem<unsigned long long, true, false>(smem_optin) != cudaSuccess ||
        allow_run_smem<unsigned long long, false, true>(smem_optin) != cudaSuccess) {
        cudaGetLastError();
        return GQ_ERR_CUDA;
    }
    if (device >= 0 && device < 64) done[device].store(1, std::memory_order_release);
    return GQ_OK;
}

extern "C" int gq_run(gq_handle h, const gq_run_args* args, void* stream) {
    if (!h || !args || !args->d_counts) return GQ_ERR_INVALID;
    const gq_run_args& g = *args;
    if (g.mode > GQ_RUN_SPLIT || g.threads == 0) return GQ_ERR_INVALID;
    if (g.block == 0 || g.block > 256 || (g.block & 31)) return GQ_ERR_INVALID;
    if (g.mode == GQ_RUN_MIXED && !g.d_sched) return GQ_ERR_INVALID;
    if (g.mode == GQ_RUN_PAIRS && (g.ops & 1)) return GQ_ERR_INVALID;
    if (g.mode == GQ_RUN_SPLIT && (g.producers > g.threads || g.total_ops / g.threads >= (1ull << 32)))
        return GQ_ERR_INVALID;
    if (h->dev.kind != GQ_LFQ && g.threads > h->dev.max_threads) return GQ_ERR_TOO_MANY_THREADS;
    if (h->dev.elem_bytes == 4) {
        const uint64_t per = (g.mode == GQ_RUN_SPLIT) ? (g.total_ops + g.threads - 1) / g.threads : g.ops;
        if (g.threads > 65536 || per > 65536) return GQ_ERR_INVALID;
    }
    RunK a;
    a.mode = g.mode;
    a.threads = g.threads;
    a.ops = g.ops;
    a.producers = g.producers;
    a.delay_ns = g.delay_ns;
    a.total_ops = g.total_ops;
    a.sched = reinterpret_cast<const u64*>(g.d_sched);
    a.status = g.d_status;
    a.val = reinterpret_cast<u64*>(g.d_val);
    a.call = reinterpret_cast<u64*>(g.d_call);
    a.end = reinterpret_cast<u64*>(g.d_end);
    a.counts = g.d_counts;
    a.ticket = reinterpret_cast<u64*>(g.d_ticket);
    a.opcnt = g.d_opcount;
    if (a.ticket && a.opcnt) return GQ_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return h->dev.elem_bytes == 4 ? dispatch_run<unsigned int>(h, a, g.block, st)
                                  : dispatch_run<unsigned long long>(h, a, g.block, st);
}

extern "C" int gq_run_sequence(gq_handle h, const uint8_t* d_kind, const uint64_t* d_val, uint64_t n,
                               int8_t* d_status, uint64_t* d_out, void* stream) {
    if (!h || (n && (!d_kind || !d_val || !d_status || !d_out))) return GQ_ERR_INVALID;
    if (n == 0) return GQ_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const u64* val = reinterpret_cast<const u64*>(d_val);
    u64* out = reinterpret_cast<u64*>(d_out);
    return h->dev.elem_bytes == 4 ? dispatch_seq<unsigned int>(h, d_kind, val, n, d_status, out, st)
                                  : dispatch_seq<unsigned long long>(h, d_kind, val, n, d_status, out, st);
}

extern "C" int gq_drain(gq_handle h, uint64_t* d_out, uint64_t max, unsigned long long* d_count, void* stream) {
    if (!h || !d_count || (max && !d_out)) return GQ_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    u64* out = reinterpret_cast<u64*>(d_out);
    return h->dev.elem_bytes == 4 ? dispatch_drain<unsigned int>(h, out, max, d_count, st)
                                  : dispatch_drain<unsigned long long>(h, out, max, d_count, st);
}
