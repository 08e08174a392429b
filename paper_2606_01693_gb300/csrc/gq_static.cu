// FIFO round trip without any device allocation (include/gq.h,
// gq_fifo_static_roundtrip).
//
// Some callers cannot call cudaMalloc: code that runs while another framework
// owns the device allocator and has reserved all memory, or code that must not
// allocate once a service is up.  This entry point serves them: the queue's
// whole workspace (control lines, both rings, payload array) lives in one
// file-scope static device array of fixed size, so a call allocates nothing;
// the caller passes only its input items and its output buffers.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call re-initialises the part it uses before any queue
// operation.  Calls that overlap on the GPU (different streams, or the same
// device from several host threads without ordering) race on the array.
#include <cuda_runtime.h>

#include <mutex>
#include <string.h>

#include "gq_host.h"
#include "gq_ops.cuh"

using namespace gqd;

namespace {

constexpr uint64_t kStaticMaxItems = 1ull << 16;             // largest n per call
constexpr uint64_t kStaticCtl = 16 * 128;                    // control lines
constexpr uint64_t kStaticRing = 2 * kStaticMaxItems * 8;    // 2n slots of one ring
constexpr uint64_t kStaticBytes = kStaticCtl + 2 * kStaticRing + kStaticMaxItems * 8;   // 2.6 MB

__device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

// Device address of g_static_ws per device, taken once with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

int static_base(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GQ_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) return GQ_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return GQ_OK;
}

// Initialises an empty G-LFQ of capacity n (a power of two) in the array and
// zeroes the caller's output counter.
__global__ void k_static_init(gq_dev q, unsigned long long* num_out) {
    const u64 n = q.capacity;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    const u64 c0 = (2 * n >> (q.log2n + 1)) & ((1ull << q.cycle_bits) - 1);   // cycle of ticket 2n
    const u64 cm1 = (c0 - 1) & ((1ull << q.cycle_bits) - 1);
    for (u64 j = (u64)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * n; j += stride) {
        q.aq.slots[j] = lfq_entry(cm1, kSafe, kBot);
        q.fq.slots[j] = (j < n) ? lfq_entry(c0, kSafe, (u32)j) : lfq_entry(cm1, kSafe, kBot);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *q.err = 0;
        for (int i = 0; i < 16; ++i) q.scratch[i] = 0;
        *q.aq.head = 2 * n;
        *q.aq.tail = 2 * n;
        *q.fq.head = 2 * n;
        *q.fq.tail = 3 * n;
        *q.aq.threshold = -1;
        *q.fq.threshold = (long long)(3 * n) - 1;
        *num_out = 0;
    }
}

__global__ void k_static_enq(const __grid_constant__ gq_dev q, const unsigned long long* __restrict__ items, u64 n) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        queue_enqueue<unsigned long long, GQ_LFQ>(q, items[k], 0);
}

__global__ void k_static_deq(const __grid_constant__ gq_dev q, unsigned long long* __restrict__ out, u64 n, unsigned long long* num_out) {
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        unsigned long long v;
        if (queue_dequeue<unsigned long long, GQ_LFQ>(q, &v, 0) == GQ_OK) {
            const u64 p = warp_faa<false>(reinterpret_cast<u64*>(num_out), 1, 32);
            out[p] = v;
        }
    }
}

}  // namespace

extern "C" int gq_fifo_static_roundtrip(const unsigned long long* d_items, uint64_t n, unsigned long long* d_out,
                                        unsigned long long* d_num_out, void* stream) {
    if (n > kStaticMaxItems) return GQ_ERR_INVALID;
    if (!d_num_out || (n && (!d_items || !d_out))) return GQ_ERR_INVALID;
    void* base = nullptr;
    int s = static_base(&base);
    if (s != GQ_OK) return s;
    uint32_t log2n = 1;
    while ((1ull << log2n) < n) ++log2n;
    const uint64_t cap = 1ull << log2n;
    char* b = static_cast<char*>(base);
    gq_dev q;
    memset(&q, 0, sizeof(q));
    q.kind = GQ_LFQ;
    q.elem_bytes = 8;
    q.log2n = log2n;
    q.cycle_bits = 31;
    q.max_threads = 1;
    q.batch_width = 32;
    q.capacity = cap;
    q.ring_order = log2n + 1;
    q.slot_mask = 2 * cap - 1;
    q.cycle_mask = (1ull << 31) - 1;
    q.cycle_half = 1ull << 30;
    q.thr_reset = (int64_t)(3 * cap) - 1;
    q.err = reinterpret_cast<unsigned int*>(b);
    q.scratch = reinterpret_cast<unsigned long long*>(b + 128);
    q.aq.head = reinterpret_cast<unsigned long long*>(b + 2 * 128);
    q.aq.tail = reinterpret_cast<unsigned long long*>(b + 3 * 128);
    q.aq.threshold = reinterpret_cast<long long*>(b + 4 * 128);
    q.fq.head = reinterpret_cast<unsigned long long*>(b + 5 * 128);
    q.fq.tail = reinterpret_cast<unsigned long long*>(b + 6 * 128);
    q.fq.threshold = reinterpret_cast<long long*>(b + 7 * 128);
    q.aq.slots = reinterpret_cast<unsigned long long*>(b + kStaticCtl);
    q.fq.slots = reinterpret_cast<unsigned long long*>(b + kStaticCtl + kStaticRing);
    q.data = b + kStaticCtl + 2 * kStaticRing;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t grid = (uint32_t)((2 * cap + 255) / 256);
    k_static_init<<<grid, 256, 0, st>>>(q, d_num_out);
    if (n) {
        const uint32_t g2 = (uint32_t)((n + 255) / 256);
        k_static_enq<<<g2, 256, 0, st>>>(q, d_items, n);
        k_static_deq<<<g2, 256, 0, st>>>(q, d_out, n, d_num_out);
    }
    return gq_check_launch();
}
