// Applications on the queues (include/gq_apps.h): level-synchronous BFS with
// two alternating frontier queues (Section V-B).
//
// GPU-first structure: one cooperative persistent kernel runs every level; a
// device-wide barrier (bounded wait) separates levels, so no host round trip
// happens per level.  Per level only as many warps dequeue as the frontier
// needs (ceil(F / 32)), which keeps the end-of-level EMPTY dequeues few (a
// G-WFQ-YMC EMPTY dequeue costs a pool cell).  A lane that dequeued a vertex of
// degree < 32 scans it alone; vertices of degree >= 32 are scanned by the whole
// warp with coalesced adjacency loads.  A neighbour is claimed with a CAS on
// its distance word (UNREACHED -> level + 1); distances are unique, so any
// claim order yields the same distances.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/gq_apps.h"
#include "gq_bfs.cuh"
#include "gq_host.h"

using namespace gqd;

namespace {

constexpr u32 kBarrierSpinLimit = 1u << 26;   // x ~100 ns sleeps: a few seconds
constexpr u64 kGridChunkCap = 1u << 21;       // chunk-map positions of a whole-GPU search

// Control words in the first queue's scratch line (words 8..15).
enum { kCtlFront0 = 2, kCtlFront1 = 3, kCtlFront2 = 4, kCtlErr = 5 };

// Device-wide barrier for a cooperative launch: the last block to arrive
// resets the count and bumps the generation; the others wait for it, at most
// kBarrierSpinLimit sleeps, after which they latch an error and go on.  The
// count and the generation sit on different 4 KB lines of the search's table
// (the arrivals' atomics do not queue behind the waiters' loads).
// If `word` is given, thread 0 reads it after the barrier and every thread of
// the block gets the value in *value (one load per block instead of per thread).
__device__ __forceinline__ bool grid_barrier(u64* ctl, u64* table, u32 nblocks, u64* word = nullptr,
                                             u64* value = nullptr) {
    __shared__ int s_ok;
    __shared__ u64 s_val;
    u64* count = table + kTabBarCount * kTabLine;
    u64* generation = table + kTabBarGen * kTabLine;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const u64 gen = ld_acq(generation);
        __threadfence();
        if (atomicAdd(reinterpret_cast<unsigned long long*>(count), 1ull) + 1 == nblocks) {
            st_rlx(count, 0);
            st_rel(generation, gen + 1);
        } else {
            u32 it = 0;
            while (ld_acq(generation) == gen) {
                if (++it > kBarrierSpinLimit) {
                    atomicCAS(reinterpret_cast<unsigned long long*>(ctl + kCtlErr), 0ull, 1ull);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok && ld_acq(ctl + kCtlErr) == 0;
        if (word) s_val = ld_acq(word);
    }
    __syncthreads();
    if (word) *value = s_val;
    return s_ok != 0;
}

template <int KIND>
__global__ void __launch_bounds__(256) k_bfs(const __grid_constant__ gq_dev qa, const __grid_constant__ gq_dev qb, u64 n,
                                             const u64* __restrict__ off, const u32* __restrict__ adj, u32 src,
                                             u32* dist, u64* table, u64 cap, unsigned long long* stats) {
    u64* ctl = reinterpret_cast<u64*>(qa.scratch) + 8;
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 nthreads = gridDim.x * blockDim.x;
    const u32 warp = tid >> 5, nwarps = nthreads >> 5;
    u64 maxdeg = 0;
    for (u64 v = tid; v < n; v += nthreads) {
        dist[v] = kUnreached;
        const u64 d = off[v + 1] - off[v];
        maxdeg = d > maxdeg ? d : maxdeg;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const u64 y = __shfl_xor_sync(0xffffffffu, maxdeg, o);
        maxdeg = y > maxdeg ? y : maxdeg;
    }
    if ((threadIdx.x & 31) == 0 && maxdeg) atomicMax(reinterpret_cast<unsigned long long*>(table + kTabMaxDeg), maxdeg);
    if (tid == 0)
        chunk_reset_all(table);
    if (!grid_barrier(ctl, table, gridDim.x)) return;
    // without a vertex of degree >= kHeavyDeg no chunk is ever published
    const bool chunks = ld_acq(table + kTabMaxDeg) >= kHeavyDeg;
    if (tid == 0) {
        dist[src] = 0;
        if (queue_enqueue<unsigned int, KIND>(qa, src, 0) == GQ_OK) st_rlx(ctl + kCtlFront0, 1);
    }
    u64 frontier = 0;
    if (!grid_barrier(ctl, table, gridDim.x, ctl + kCtlFront0, &frontier)) return;
    u64 edges = 0, reached = 0;
    u32 level = 0;
    for (;; ++level) {
        if (frontier == 0) break;
        reached += (tid == 0) ? frontier : 0;
        if (tid == 0) {
            st_rlx(ctl + kCtlFront0 + (level + 2) % 3, 0);   // read by all during level - 1
            chunk_prepare_next(table, level);
        }
        const u64 want = (frontier + 31) / 32;
        const u64 dq = want < nwarps ? want : nwarps;
        const LevelCtx c = level_ctx(off, adj, dist, level, tid, table, cap, frontier, dq);
        const gq_dev& cur = (level & 1) ? qb : qa;
        const gq_dev& nxt = (level & 1) ? qa : qb;
        u32 cnt = 0;
        if (warp < dq) level_dequeue<KIND>(cur, nxt, c, warp, chunks, &cnt, &edges);
        if (chunks && !level_chunks<KIND>(nxt, c, &cnt, &edges) && (threadIdx.x & 31) == 0)
            atomicCAS(reinterpret_cast<unsigned long long*>(ctl + kCtlErr), 0ull, 2ull);
        warp_add_full(reinterpret_cast<unsigned long long*>(ctl + kCtlFront0 + (level + 1) % 3), cnt);
        if (!grid_barrier(ctl, table, gridDim.x, ctl + kCtlFront0 + (level + 1) % 3, &frontier)) return;
    }
    if (stats) warp_add_full(stats + 2, edges);
    if (tid == 0 && stats) {
        stats[0] = level;
        stats[1] = reached;
        stats[3] = ld_acq(ctl + kCtlErr);
    }
}

template <int KIND>
int bfs_grid_threads(uint64_t* threads) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bfs<KIND>, 256, 0) != cudaSuccess || occ < 1)
        return GQ_ERR_CUDA;
    *threads = (uint64_t)occ * (uint64_t)sms * 256;
    return GQ_OK;
}

template <int KIND>
int launch_bfs(gq_handle ha, gq_handle hb, uint64_t n, const uint64_t* off, const uint32_t* adj, uint32_t src,
               uint32_t* dist, unsigned long long* stats, cudaStream_t st) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bfs<KIND>, 256, 0) != cudaSuccess || occ < 1)
        return GQ_ERR_CUDA;
    uint64_t grid = (uint64_t)occ * (uint64_t)ha->sm_count;
    if (KIND != GQ_LFQ) {
        const uint64_t rec = ha->dev.max_threads < hb->dev.max_threads ? ha->dev.max_threads : hb->dev.max_threads;
        if (grid > rec / 256) grid = rec / 256;
    }
    if (grid < 1) return GQ_ERR_TOO_MANY_THREADS;
    // chunk map, owned by the first queue's handle (made and zeroed once; a
    // search leaves it zeroed)
    u64 cap = kGridChunkCap;
    if (!ha->aux) {
        const u64 bytes = chunk_map_bytes(cap);
        if (cudaMalloc(&ha->aux, bytes) != cudaSuccess) {
            cudaGetLastError();
            ha->aux = nullptr;
            return GQ_ERR_NOMEM;
        }
        if (cudaMemsetAsync(ha->aux, 0, bytes, st) != cudaSuccess) return GQ_ERR_CUDA;
        ha->aux_bytes = bytes;
    }
    u64* table = static_cast<u64*>(ha->aux);
    // a search that ended on an expired barrier wait may have left the count behind;
    // the maximum degree is accumulated afresh by every search
    if (cudaMemsetAsync(table + kTabBarCount * kTabLine, 0, sizeof(u64), st) != cudaSuccess ||
        cudaMemsetAsync(table + kTabMaxDeg, 0, sizeof(u64), st) != cudaSuccess)
        return GQ_ERR_CUDA;
    gq_dev qa = ha->dev, qb = hb->dev;
    const u64* o = reinterpret_cast<const u64*>(off);
    const u32* a = reinterpret_cast<const u32*>(adj);
    void* args[] = {&qa, &qb, &n, (void*)&o, (void*)&a, &src, &dist, &table, &cap, &stats};
    if (cudaLaunchCooperativeKernel((const void*)k_bfs<KIND>, dim3((unsigned)grid), dim3(256), args, 0, st) != cudaSuccess)
        return GQ_ERR_CUDA;
    return gq_check_launch();
}

// ---------------------------------------------------------------------------
// Batched BFS: one instance per thread-block cluster at a time
// ---------------------------------------------------------------------------

constexpr u32 kNoInstance = 0xFFFFFFFFu;

struct BatchK {
    const gq_bfs_instance* inst;
    const u32* order;
    u32 ninst;
    u64* ctl;                  // 8 words per slot: [0] instance, [1..3] frontier counts
    u64* tables;               // chunk map per slot (kClusterChunkCap positions)
    unsigned long long* stats; // instances, edges, levels, errors
};

__global__ void k_bfs_batch_fill(const __grid_constant__ gq_dev idq, const u32* order, u32 ninst, u64* err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (u32 i = 0; i < ninst; ++i)
        if (queue_enqueue<unsigned int, GQ_LFQ>(idq, order[i], 0) != GQ_OK) atomicAdd(reinterpret_cast<unsigned long long*>(err), 1ull);
}

template <int KIND>
__global__ void __launch_bounds__(256) k_bfs_batch(const __grid_constant__ gq_dev idq, const gq_dev* __restrict__ fq,
                                                   const __grid_constant__ BatchK a) {
    cg::cluster_group cluster = cg::this_cluster();
    const u32 cblocks = cluster.num_blocks();
    const u32 slot = blockIdx.x / cblocks;
    const u32 ct = cluster.block_rank() * blockDim.x + threadIdx.x;    // thread id within the cluster
    const u32 nct = cblocks * blockDim.x;
    u64* ctl = a.ctl + 8 * (u64)slot;
    const gq_dev& qa = fq[2 * slot];
    const gq_dev& qb = fq[2 * slot + 1];
    u64 edges = 0, levels_sum = 0, done = 0;
    for (u32 guard = 0; guard < a.ninst + 1; ++guard) {
        if (ct == 0) {
            unsigned int id = 0;
            const int s = queue_dequeue<unsigned int, GQ_LFQ>(idq, &id, slot);
            st_rlx(ctl, s == GQ_OK ? id : kNoInstance);
        }
        cluster.sync();
        const u32 id = (u32)ld_acq(ctl);
        cluster.sync();                      // everyone has read the id before ctl is reused
        if (id == kNoInstance || id >= a.ninst) break;
        const gq_bfs_instance g = a.inst[id];
        const u32 lv = cluster_bfs<KIND>(qa, qb, ctl + 1, a.tables + slot * (chunk_map_bytes(kClusterChunkCap) / 8),
                                         kClusterChunkCap, g, g.d_dist, ct, nct, cluster, &edges,
                                         a.stats ? a.stats + 3 : nullptr);
        if (ct == 0) {
            levels_sum += lv;
            ++done;
        }
    }
    if (a.stats) {
        warp_add_full(a.stats + 1, edges);
        if (ct == 0) {
            atomicAdd(a.stats, done);
            atomicAdd(a.stats + 2, levels_sum);
        }
    }
}

template <int KIND>
int launch_bfs_batch(gq_handle idq, const gq_handle* fr, u32 slots, u32 cb, const gq_bfs_instance* inst,
                     const u32* order, u32 ninst, void* ws, unsigned long long* stats, cudaStream_t st) {
    char* b = static_cast<char*>(ws);
    gq_dev* views = reinterpret_cast<gq_dev*>(b);
    u64* ctl = reinterpret_cast<u64*>(b + (((u64)2 * slots * sizeof(gq_dev) + 255) / 256) * 256);
    std::vector<gq_dev> h(2 * slots);
    for (u32 i = 0; i < 2 * slots; ++i) h[i] = fr[i]->dev;
    if (cudaMemcpyAsync(views, h.data(), h.size() * sizeof(gq_dev), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return GQ_ERR_CUDA;
    u64* tables = ctl + 8 * (u64)slots;
    if (cudaMemsetAsync(ctl, 0, (u64)slots * (64 + chunk_map_bytes(kClusterChunkCap)), st) != cudaSuccess)
        return GQ_ERR_CUDA;
    k_bfs_batch_fill<<<1, 1, 0, st>>>(idq->dev, order, ninst, stats ? reinterpret_cast<u64*>(stats + 3) : ctl);
    BatchK a{inst, order, ninst, ctl, tables, stats};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(slots * cb);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cb;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    gq_dev iq = idq->dev;
    const gq_dev* fv = views;
    if (cudaLaunchKernelEx(&cfg, k_bfs_batch<KIND>, iq, fv, a) != cudaSuccess) return GQ_ERR_CUDA;
    return gq_check_launch();
}

}  // namespace

extern "C" int gq_bfs_batch_workspace_bytes(uint32_t slots, uint64_t* bytes) {
    if (!slots || !bytes) return GQ_ERR_INVALID;
    *bytes = (((uint64_t)2 * slots * sizeof(gq_dev) + 255) / 256) * 256 +
             (uint64_t)slots * (64 + chunk_map_bytes(kClusterChunkCap));
    return GQ_OK;
}

extern "C" int gq_bfs_batch(gq_handle id_queue, const gq_handle* frontier, uint32_t slots, uint32_t cluster_blocks,
                            const gq_bfs_instance* d_instances, const uint32_t* d_order, uint32_t ninst,
                            void* d_workspace, unsigned long long* d_stats, void* stream) {
    if (!id_queue || !frontier || !slots || !d_instances || !d_order || !ninst || !d_workspace) return GQ_ERR_INVALID;
    if (cluster_blocks != 1 && cluster_blocks != 2 && cluster_blocks != 4 && cluster_blocks != 8) return GQ_ERR_INVALID;
    if (id_queue->dev.kind != GQ_LFQ || id_queue->dev.elem_bytes != 4 || id_queue->dev.capacity < ninst)
        return GQ_ERR_INVALID;
    const int kind = frontier[0]->dev.kind;
    for (uint32_t i = 0; i < 2 * slots; ++i) {
        if (!frontier[i] || frontier[i]->dev.kind != kind || frontier[i]->dev.elem_bytes != 4 ||
            frontier[i]->device != id_queue->device)
            return GQ_ERR_INVALID;
        if (kind != GQ_LFQ && frontier[i]->dev.max_threads < cluster_blocks * 256) return GQ_ERR_TOO_MANY_THREADS;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d_stats && cudaMemsetAsync(d_stats, 0, 4 * sizeof(unsigned long long), st) != cudaSuccess) return GQ_ERR_CUDA;
    switch (kind) {
        case GQ_LFQ: return launch_bfs_batch<GQ_LFQ>(id_queue, frontier, slots, cluster_blocks, d_instances, d_order, ninst, d_workspace, d_stats, st);
        case GQ_WFQ: return launch_bfs_batch<GQ_WFQ>(id_queue, frontier, slots, cluster_blocks, d_instances, d_order, ninst, d_workspace, d_stats, st);
        default: return launch_bfs_batch<GQ_YMC>(id_queue, frontier, slots, cluster_blocks, d_instances, d_order, ninst, d_workspace, d_stats, st);
    }
}

int gq_bfs_grid_threads(int kind, uint64_t* threads) {
    switch (kind) {
        case GQ_LFQ: return bfs_grid_threads<GQ_LFQ>(threads);
        case GQ_WFQ: return bfs_grid_threads<GQ_WFQ>(threads);
        case GQ_YMC: return bfs_grid_threads<GQ_YMC>(threads);
        default: return GQ_ERR_INVALID;
    }
}

extern "C" int gq_bfs(gq_handle q_a, gq_handle q_b, uint64_t n, const uint64_t* d_offsets, const uint32_t* d_adj,
                      uint32_t src, uint32_t* d_dist, unsigned long long* d_stats, void* stream) {
    if (!q_a || !q_b || q_a == q_b || !d_offsets || !d_dist || n == 0 || n >= 0xFFFFFFFFull || src >= n)
        return GQ_ERR_INVALID;
    if (q_a->dev.kind != q_b->dev.kind || q_a->dev.elem_bytes != 4 || q_b->dev.elem_bytes != 4 ||
        q_a->device != q_b->device)
        return GQ_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(q_a->dev.scratch + 8, 0, 8 * sizeof(unsigned long long), st) != cudaSuccess) return GQ_ERR_CUDA;
    if (d_stats && cudaMemsetAsync(d_stats, 0, 4 * sizeof(unsigned long long), st) != cudaSuccess) return GQ_ERR_CUDA;
    switch (q_a->dev.kind) {
        case GQ_LFQ: return launch_bfs<GQ_LFQ>(q_a, q_b, n, d_offsets, d_adj, src, d_dist, d_stats, st);
        case GQ_WFQ: return launch_bfs<GQ_WFQ>(q_a, q_b, n, d_offsets, d_adj, src, d_dist, d_stats, st);
        default: return launch_bfs<GQ_YMC>(q_a, q_b, n, d_offsets, d_adj, src, d_dist, d_stats, st);
    }
}
