// Same-box L2 atomic micro-benchmarks (include/gq_drivers.h, gq_atomic_peak).
//
// The queues are bound by L2 atomic throughput, not by HBM bandwidth or tensor
// cores: every operation is a handful of 64-bit RMWs on L2-resident words.  The
// roofline denominators are measured here on the same GPU:
//   * same-address fetch-add: the ceiling of one hot ticket counter;
//   * warp-coalesced CAS: 32 lanes on 32 consecutive 8-byte words, the access
//     shape of a warp's slot CASes after WaveFAA handed it consecutive tickets;
//   * scattered CAS: every lane on an unrelated word (no coalescing);
//   * fetch-add on 16 counters 4 KB apart and on 16 counters 128 B apart: a
//     queue's hot counters only add up their single-address rates when they
//     sit in different L2 slices, which decides the control-line spacing.
#include <cuda_runtime.h>

#include "../../include/gq_drivers.h"
#include "gq_atomics.cuh"
#include "gq_host.h"

using namespace gqd;

namespace {

__device__ __forceinline__ u64 hash64(u64 x) {
    x ^= x >> 33;
    x *= 0xFF51AFD7ED558CCDull;
    x ^= x >> 33;
    x *= 0xC4CEB9FE1A85EC53ull;
    x ^= x >> 33;
    return x;
}

__device__ __forceinline__ u64 atom_add_relaxed(u64* p, u64 v) {
    u64 r;
    asm volatile("atom.relaxed.gpu.global.add.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
    return r;
}
__device__ __forceinline__ u64 atom_cas_relaxed(u64* p, u64 cmp, u64 v) {
    u64 r;
    asm volatile("atom.relaxed.gpu.global.cas.b64 %0, [%1], %2, %3;" : "=l"(r) : "l"(p), "l"(cmp), "l"(v)
                 : "memory");
    return r;
}
__device__ __forceinline__ u64 ld_relaxed_gpu(const u64* p) {
    u64 r;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(r) : "l"(p) : "memory");
    return r;
}

__global__ void k_peak(int pattern, u32 iters, u64* buf, u64 words, unsigned long long* sink) {
    const u64 gtid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 warp = gtid >> 5;
    const u32 lane = threadIdx.x & 31;
    const u64 groups = words >> 5;  // 32-word groups
    u64 acc = 0;
    if (pattern == GQ_PEAK_SAME_ADDR_FAA) {
        if (lane == 0)
            for (u32 i = 0; i < iters; ++i) acc += atom_add_relaxed(buf, 1);
    } else if (pattern == GQ_PEAK_SPREAD_FAA || pattern == GQ_PEAK_PACKED_FAA) {
        u64* c = buf + (warp % 16) * (pattern == GQ_PEAK_SPREAD_FAA ? 512 : 16);
        if (lane == 0)
            for (u32 i = 0; i < iters; ++i) acc += atom_add_relaxed(c, 1);
    } else if (pattern == GQ_PEAK_COALESCED_CAS) {
        for (u32 i = 0; i < iters; ++i) {
            const u64 g = hash64(warp * 0x9E3779B97F4A7C15ull + i) % groups;
            acc += atom_cas_relaxed(buf + g * 32 + lane, acc, acc + i);
        }
    } else if (pattern == GQ_PEAK_SCATTERED_CAS) {
        for (u32 i = 0; i < iters; ++i) {
            const u64 w = hash64(gtid * 0x9E3779B97F4A7C15ull + i) % words;
            acc += atom_cas_relaxed(buf + w, acc, acc + i);
        }
    } else {
        for (u32 i = 0; i < iters; ++i) {
            const u64 g = hash64(warp * 0x9E3779B97F4A7C15ull + i) % groups;
            acc += ld_relaxed_gpu(buf + g * 32 + lane);
        }
    }
    if (acc == 0x5EEDull) atomicAdd(sink, 1ull);
}

__global__ void k_wavefaa_probe(const uint8_t* take, u32 threads, u32 width, u64* counters, u64* tickets) {
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= threads) return;
    u64 ticket = ~0ull;
    if (take[t] == 1 || take[t] == 2) ticket = warp_faa<true>(counters + (take[t] - 1), 1, width);
    tickets[t] = ticket;
}

}  // namespace

extern "C" int gq_wavefaa_probe(const uint8_t* d_take, uint32_t threads, uint32_t width, unsigned long long* d_counters,
                                unsigned long long* d_tickets, void* stream) {
    if (!d_take || !threads || !d_counters || !d_tickets || width == 0 || width > 32 || (width & (width - 1)))
        return GQ_ERR_INVALID;
    k_wavefaa_probe<<<(threads + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_take, threads, width, reinterpret_cast<u64*>(d_counters), reinterpret_cast<u64*>(d_tickets));
    return gq_check_launch();
}

extern "C" int gq_atomic_peak(int pattern, uint32_t blocks, uint32_t threads, uint32_t iters,
                              unsigned long long* d_buf, uint64_t buf_words, unsigned long long* d_sink,
                              void* stream) {
    if (pattern < 0 || pattern > GQ_PEAK_PACKED_FAA || !d_buf || !d_sink) return GQ_ERR_INVALID;
    if (blocks == 0 || threads == 0 || threads > 1024 || (threads & 31) || buf_words < 32) return GQ_ERR_INVALID;
    if (pattern == GQ_PEAK_SPREAD_FAA && buf_words < 16 * 512) return GQ_ERR_INVALID;
    if (pattern == GQ_PEAK_PACKED_FAA && buf_words < 16 * 16) return GQ_ERR_INVALID;
    k_peak<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(pattern, iters, d_buf, buf_words, d_sink);
    return gq_check_launch();
}
