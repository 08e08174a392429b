// BFS serving runtime (include/gq_serve.h): a persistent device scheduler fed
// by a host request ring in mapped pinned memory, and the per-request-launch
// form it is measured against.
//
// Device side.  One persistent launch of `slots` thread-block clusters.  Each
// cluster's thread 0 takes the next request ticket with a fetch-add on a
// device counter and polls the ring entry of that ticket (system-scope
// acquire) until the host has published it, sleeping between polls; the wait
// is bounded by %globaltimer and a host stop word.  It hands the request to the
// cluster through device-memory control words, the cluster runs the
// level-synchronous BFS on its own two frontier queues (hardware cluster
// barrier between levels), and thread 0 marks the entry done with a
// system-scope release after a system fence.  Tickets >= the request count end
// the cluster.
//
// Host side (native, in this file).  One thread runs arrivals, admission and
// completion: it publishes each request once its arrival time has passed, its
// ring entry is free (the request one ring-length earlier is done) and its
// state fits in the budget (first come first served); scratch distance arrays
// come from a first-fit arena with coalescing.  It polls the done words of the
// requests in flight and records latencies.  If the scheduler kernel ends
// before every request is done, or nothing progresses for the wait limit, it
// raises the stop word and reports the error.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <deque>
#include <algorithm>
#include <iterator>
#include <map>
#include <vector>

#include "../../include/gq_serve.h"
#include "gq_bfs.cuh"
#include "gq_host.h"

using namespace gqd;

namespace {

// One 64-byte ring entry in mapped pinned memory.
struct ServeEntry {
    u64 seq;      // host: ticket + 1 once the fields below are valid (release)
    u64 done;     // device: ticket + 1 once the distances are written (release, system scope)
    u64 req;      // host: graph id | source << 32
    u64 dist;     // host: device address of the request's distance array
    u64 levels;   // device: levels of the search
    u64 pad[3];
};
static_assert(sizeof(ServeEntry) == 64, "ring entries are one 64-byte line");

// Words the host writes in mapped pinned memory (the device only loads them:
// no atomic read-modify-write touches host memory).
struct ServeShared {
    u64 stop;     // 1 = every cluster leaves at its next wait
    u64 pad[15];
};

constexpr u64 kNoTicket = ~0ull;
constexpr u64 kMember = ~0ull - 1;      // ctl[0]: the cluster joined another cluster's gang
constexpr u64 kSealed = 1ull << 63;     // gang join word: closed
constexpr u64 kGangWaitNs = 20000;      // a gang leader waits this long for idle clusters to join
// Chunk-map positions of one slot's table.  A gang uses all 2^18 (chunks of 128
// edges for the heavy vertices of any level of the pool's largest graphs,
// scale 20: about 3.3 * 10^7 directed edges), so no hub falls back to one
// warp's gather, which the gang's other warps could not share (with 2^14 a
// 12-cluster gang took 17-22 ms on a scale-20 graph instead of 1 ms).  One
// cluster alone keeps the cluster search's 2^14 (one scale-20 search: 16 ms
// with it, 21 ms with the full map, G-WFQ-YMC).
constexpr u64 kServeChunkCap = 1u << 18;

// Gang record of a slot (8 words in device memory).  A gang is one request
// served by several clusters: the cluster that took the ticket (the leader)
// offers the gang, idle clusters join, and all of them run one BFS on the
// leader's queues with a barrier of their own between levels.
enum {
    kGJoin = 0,     // <epoch 31 | joined count 32>, kSealed once the leader closed the gang
    kGGo = 1,       // <epoch | member count> once closed (members wait for it)
    kGBarCnt = 2,   // barrier arrivals of the current phase
    kGBarGen = 3    // barrier generation
};

struct ServeK {
    ServeEntry* ring;            // device view of the mapped ring
    ServeShared* sh;             // device view of the mapped shared words
    const gq_bfs_instance* graphs;
    u32 ngraphs, ring_mask;
    u64 nreq;
    u64* claim;                  // next ticket (device memory)
    u64* ctl;                    // 8 words per slot (device memory)
    u64* tables;                 // chunk map per slot (device memory)
    unsigned long long* stats;   // edges scanned, requests served, first error (1 = wait limit, 2 = bad
                                 // request), requests served by gangs
    u64 wait_ns;
    u64* gang;                   // 8 words per slot (device memory)
    u64* gang_open;              // <epoch | leader slot + 1> of the gang open for joining, 0 = none
    u32 gang_max;                // most clusters per request (1 = no gangs)
    u32 gang_min_n;              // requests on graphs of at least this many vertices form gangs
};

using sys_ref = cuda::atomic_ref<u64, cuda::thread_scope_system>;

__device__ __forceinline__ u64 ld_acq_sys(u64* p) { return sys_ref(*p).load(kAcq); }
__device__ __forceinline__ u64 ld_rlx_sys(u64* p) { return sys_ref(*p).load(kRlx); }
__device__ __forceinline__ void st_rel_sys(u64* p, u64 v) { sys_ref(*p).store(v, kRel); }
__device__ __forceinline__ void st_rlx_sys(u64* p, u64 v) { sys_ref(*p).store(v, kRlx); }

// Thread 0 of a cluster that took ticket t (entry e): checks the request,
// copies its fields into ctl[4..5] and, for a large graph, forms a gang.
// ctl[0] = t, ctl[7] = <members 16 | rank 24 | leader slot 24> (rank 0, leader
// = own slot); ctl[0] = kNoTicket for a bad request (the cluster leaves).
__device__ void take_request(const ServeK& a, u32 slot, u64* ctl, u64 t, ServeEntry* e) {
    const u64 req = ld_rlx_sys(&e->req);
    const u32 g = (u32)req, s = (u32)(req >> 32);
    if (g >= a.ngraphs || s >= a.graphs[g].n) {
        atomicCAS(a.stats + 2, 0ull, 2ull);
        st_rlx_sys(&e->levels, ~0ull);
        st_rel_sys(&e->done, t + 1);
        st_rlx(ctl, kNoTicket);
        return;
    }
    st_rlx(ctl + 4, ((u64)s << 32) | g);
    st_rlx(ctl + 5, ld_rlx_sys(&e->dist));
    u64 members = 1;
    if (a.gang_max > 1 && a.graphs[g].n >= a.gang_min_n) {
        u64* gr = a.gang + 8 * (u64)slot;
        const u64 ep = ((t + 1) & 0x7FFFFFFFull) | ((t + 1) & 0x7FFFFFFFull ? 0 : 1);
        st_rlx(gr + kGGo, 0);
        st_rlx(gr + kGBarCnt, 0);
        st_rel(gr + kGJoin, ep << 32);
        const u64 offer = (ep << 32) | (slot + 1);
        if (atomicCAS(reinterpret_cast<unsigned long long*>(a.gang_open), 0ull, offer) == 0ull) {
            // wait (boundedly) for idle clusters, then close the gang
            const u64 t0 = globaltimer();
            while ((u32)ld_acq(gr + kGJoin) + 1 < a.gang_max && globaltimer() - t0 < kGangWaitNs) __nanosleep(64);
            atomicCAS(reinterpret_cast<unsigned long long*>(a.gang_open), offer, 0ull);
            const u64 j = atomicOr(reinterpret_cast<unsigned long long*>(gr + kGJoin), kSealed);
            members = 1 + (u32)j;
        }
        // the member count (and, before it, ctl[4..5]) is released to the members
        st_rel(gr + kGGo, (ep << 32) | members);
    }
    st_rlx(ctl + 7, (members << 48) | slot);
    st_rlx(ctl, t);
}

// Thread 0 of an idle cluster: joins the open gang if there is one and it has
// room.  On success ctl[0] = kMember and ctl[7] describes the gang.
__device__ bool try_join(const ServeK& a, u32 slot, u64* ctl) {
    const u64 o = ld_acq(a.gang_open);
    if (o == 0) return false;
    const u32 lead = (u32)o - 1;
    const u64 ep = o >> 32;
    if (lead == slot) return false;
    u64* gr = a.gang + 8 * (u64)lead;
    u64 j = ld_acq(gr + kGJoin);
    u32 rank = 0;
    for (u32 it = 0; it < 64 && rank == 0; ++it) {
        if ((j >> 32) != ep || (u32)j + 1 >= a.gang_max) return false;   // another gang, closed, or full
        const u64 w = atomicCAS(reinterpret_cast<unsigned long long*>(gr + kGJoin), j, j + 1);
        if (w == j) rank = (u32)j + 1;
        else j = w;
    }
    if (rank == 0) return false;
    const u64 t0 = globaltimer();
    u64 go = ld_acq(gr + kGGo);
    for (u32 polls = 0; (go >> 32) != ep; ++polls) {
        if (globaltimer() - t0 > a.wait_ns) {
            atomicCAS(a.stats + 2, 0ull, 1ull);
            st_rlx(ctl, kNoTicket);
            return true;
        }
        __nanosleep(32);
        go = ld_acq(gr + kGGo);
    }
    st_rlx(ctl + 7, ((go & 0xFFFFull) << 48) | ((u64)rank << 24) | lead);
    st_rlx(ctl, kMember);
    return true;
}

// Thread 0 of a cluster: the next piece of work, in ctl[0] (a ticket, kMember,
// or kNoTicket when there is none left, the host asked to stop, or the wait
// limit expired with no ticket published, error latched).  A ticket is taken
// only once the host has published it (a CAS on the claim counter from the
// ticket it read), so an idle cluster holds no ticket and can join a gang.
__device__ void next_work(const ServeK& a, u32 slot, u64* ctl) {
    u64 last = ~0ull, t0 = 0;
    for (u32 polls = 0;; ++polls) {
        const u64 c = ld_acq(a.claim);
        if (c >= a.nreq) break;
        ServeEntry* e = a.ring + (c & a.ring_mask);
        if (ld_acq_sys(&e->seq) == c + 1) {
            if (atomicCAS(reinterpret_cast<unsigned long long*>(a.claim), c, c + 1) == c) {
                take_request(a, slot, ctl, c, e);
                return;
            }
            continue;                       // another cluster took it: look at the next ticket
        }
        if (a.gang_max > 1 && try_join(a, slot, ctl)) return;
        if (ld_rlx_sys(&a.sh->stop)) break;
        if (c != last) {
            last = c;
            t0 = globaltimer();
        } else if (globaltimer() - t0 > a.wait_ns) {
            atomicCAS(a.stats + 2, 0ull, 1ull);
            break;
        }
        __nanosleep(polls < 256 ? 64 : 256);
    }
    st_rlx(ctl, kNoTicket);
}

// Barrier of the clusters that serve one request.  One cluster: the cluster
// barrier.  A gang: the cluster barrier, then thread 0 of each cluster meets
// the others on the leader's counter (arrive with a fetch-add after a fence,
// wait boundedly for the generation to move), then the cluster barrier again.
// Returns false in every thread of the cluster once a wait expired (latched).
// The gang part is a call out of line, so that one search body (the
// one-cluster search with a call in its barrier) is inlined into the scheduler
// kernel, not one per barrier type.
struct ServeSync {
    cg::cluster_group& cluster;
    u64* gr;                     // the leader's gang record
    u64* flag;                   // this cluster's broadcast word
    u32 members;
    bool lead;                   // thread 0 of this cluster
    u64 wait_ns;
    unsigned long long* err;
    __device__ bool operator()() const {
        if (members <= 1) {
            cluster.sync();
            return true;
        }
        return gang_sync(cluster, gr, flag, members, lead, wait_ns, err);
    }
    static __device__ __noinline__ bool gang_sync(cg::cluster_group& cluster, u64* gr, u64* flag, u32 members,
                                                  bool lead, u64 wait_ns, unsigned long long* err) {
        cluster.sync();
        if (lead) {
            bool ok = true;
            const u64 g0 = ld_acq(gr + kGBarGen);
            __threadfence();
            if (atomicAdd(reinterpret_cast<unsigned long long*>(gr + kGBarCnt), 1ull) + 1 == members) {
                st_rlx(gr + kGBarCnt, 0);
                st_rel(gr + kGBarGen, g0 + 1);
            } else {
                const u64 t0 = globaltimer();
                while (ld_acq(gr + kGBarGen) == g0) {
                    if (globaltimer() - t0 > wait_ns) {
                        atomicCAS(err, 0ull, 1ull);
                        ok = false;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
            st_rlx(flag, ok ? 0 : 1);
        }
        cluster.sync();
        return ld_rlx(flag) == 0;
    }
};

// Registers: G-LFQ's and G-WFQ-YMC's kernels are held to 64 (four 256-thread
// blocks per SM: 74 eight-block clusters on the GPU; unbounded, the compiler
// takes 115 and 80, and 36 and 51 clusters fit).  G-WFQ's takes 64 unbounded,
// and bounding it anyway cost it 30 % of its requests per second at
// saturation (3.2 against 4.6 k req/s at 10,000 req/s offered).
template <int KIND>
__global__ void __launch_bounds__(256, KIND == GQ_WFQ ? 0 : 4) k_serve(const gq_dev* __restrict__ fq, const __grid_constant__ ServeK a) {
    cg::cluster_group cluster = cg::this_cluster();
    const u32 cblocks = cluster.num_blocks();
    const u32 slot = blockIdx.x / cblocks;
    const u32 ct = cluster.block_rank() * blockDim.x + threadIdx.x;
    const u32 nct = cblocks * blockDim.x;
    // [0] ticket / kMember / kNoTicket, [1..3] frontier counts, [4] src|graph,
    // [5] dist, [6] gang barrier flag, [7] gang <members | rank | leader>
    u64* ctl = a.ctl + 8 * (u64)slot;
    u64 edges = 0, served = 0, ganged = 0;
    // every iteration takes a ticket or joins a gang that took one
    for (u64 guard = 0; guard <= 2 * a.nreq; ++guard) {
        if (ct == 0) next_work(a, slot, ctl);
        cluster.sync();
        const u64 t = ld_acq(ctl);
        const u64 gd = ld_acq(ctl + 7);
        if (t == kNoTicket) break;
        const u32 lead = (u32)(gd & 0xFFFFFFull), rank = (u32)((gd >> 24) & 0xFFFFFFull);
        const u32 members = (u32)(gd >> 48);
        u64* lctl = a.ctl + 8 * (u64)lead;
        const u64 gs = ld_acq(lctl + 4);
        u32* dist = reinterpret_cast<u32*>(ld_acq(lctl + 5));
        cluster.sync();                      // every thread has read ctl before it is reused
        gq_bfs_instance g = a.graphs[(u32)gs];
        g.src = (u32)(gs >> 32);
        u64* table = a.tables + lead * (chunk_map_bytes(kServeChunkCap) / 8);
        const gq_dev& qa = fq[2 * lead];
        const gq_dev& qb = fq[2 * lead + 1];
        // a gang shares the leader's chunk map at full size; one cluster uses
        // the cluster search's (its warps are busy with their own gathers)
        const ServeSync sync{cluster, a.gang + 8 * (u64)lead, ctl + 6, members, ct == 0, a.wait_ns, a.stats + 2};
        const u32 levels = group_bfs<KIND>(qa, qb, lctl + 1, table, members > 1 ? kServeChunkCap : kClusterChunkCap,
                                           g, dist, rank * nct + ct, members * nct, sync, &edges, a.stats + 2);
        if (ct == 0 && t != kMember) {
            ServeEntry* e = a.ring + (t & a.ring_mask);
            __threadfence_system();
            st_rlx_sys(&e->levels, levels == kBfsAborted ? ~0ull : (u64)levels);
            st_rel_sys(&e->done, t + 1);
            ++served;
            ganged += members > 1;
        }
        if (levels == kBfsAborted) break;
    }
    warp_add_full(a.stats, edges);
    if (ct == 0 && served) atomicAdd(a.stats + 1, served);
    if (ct == 0 && ganged) atomicAdd(a.stats + 3, ganged);
}

// ---------------------------------------------------------------------------
// Host runtime
// ---------------------------------------------------------------------------

typedef std::chrono::steady_clock Clock;

// First-fit allocator over [0, size) with coalescing of freed neighbours.
class Arena {
  public:
    explicit Arena(u64 size) {
        if (size) free_[0] = size;
    }
    bool alloc(u64 bytes, u64* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const u64 rest = it->second - bytes, at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            return true;
        }
        return false;
    }
    void release(u64 off, u64 bytes) {
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + bytes == nx->first) {
            bytes += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }

  private:
    std::map<u64, u64> free_;
};

u64 round256(u64 b) { return (b + 255) / 256 * 256; }

u64 ring_capacity_for(u64 n) {
    u64 c = 4096;
    while (c < n) c <<= 1;
    return c;
}
u64 ymc_pool_for(u64 n) { return 4 * n + (1ull << 18); }

// Queue capacity and thread count used for a graph of n vertices.
u64 queue_capacity(int kind, u64 n) { return kind == GQ_YMC ? ymc_pool_for(n) : ring_capacity_for(n); }

struct Runtime {
    const gq_serve_config& c;
    gq_serve_result& r;
    std::vector<u64> charge, dist_bytes, arena_off;
    std::vector<char> finished, waited;
    Arena arena;
    u64 charged = 0;
    char* d_arena = nullptr;
    Clock::time_point t0;

    Runtime(const gq_serve_config& cfg, gq_serve_result& res, u64 arena_size)
        : c(cfg), r(res), arena(arena_size) {}

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    // Admits request i (charges the budget, places its distance array);
    // false if it must wait.
    bool admit(u64 i, u32** dist) {
        if (charged + charge[i] > c.budget_bytes) return false;
        uint32_t* out = c.req_out ? c.req_out[i] : nullptr;
        if (!out) {
            u64 off = 0;
            if (!arena.alloc(dist_bytes[i], &off)) return false;
            arena_off[i] = off;
            out = reinterpret_cast<uint32_t*>(d_arena + off);
        }
        charged += charge[i];
        if (charged > r.peak_state_bytes) r.peak_state_bytes = charged;
        *dist = out;
        return true;
    }
    void complete(u64 i, double t) {
        r.latency_s[i] = t - c.req_arrival_s[i];
        charged -= charge[i];
        if (arena_off[i] != ~0ull) arena.release(arena_off[i], dist_bytes[i]);
        finished[i] = 1;
    }
};

struct Queues {
    std::vector<gq_handle> h;
    ~Queues() {
        for (gq_handle q : h)
            if (q) gq_destroy(q);
    }
    int create(u64 count, int kind, u64 cap, u32 max_threads, cudaStream_t st) {
        h.assign(count, nullptr);
        for (u64 i = 0; i < count; ++i) {
            const int s = gq_create(kind, cap, 4, max_threads, nullptr, nullptr, st, &h[i]);
            if (s != GQ_OK) return s;
        }
        return GQ_OK;
    }
    int status(cudaStream_t st) {
        for (gq_handle q : h) {
            const int s = gq_sync_status(q, st);
            if (s != GQ_OK) return s;
        }
        return GQ_OK;
    }
};

template <int KIND>
cudaError_t launch_serve(u32 slots, u32 cb, const gq_dev* views, const ServeK& a, cudaStream_t st) {
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
    return cudaLaunchKernelEx(&cfg, k_serve<KIND>, views, a);
}

template <int KIND>
cudaError_t max_clusters(u32 cb, int* out) {
    // 16-block clusters exceed the portable cluster size and must be allowed
    cudaError_t e = cudaFuncSetAttribute(k_serve<KIND>, cudaFuncAttributeNonPortableClusterSizeAllowed, cb > 8 ? 1 : 0);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cb);
    cfg.blockDim = dim3(256);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cb;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, k_serve<KIND>, &cfg);
}

// The stream and the distance arena of one gq_serve call.
struct Buffers {
    char* arena = nullptr;
    cudaStream_t st = nullptr;
    ~Buffers() {
        if (st) cudaStreamSynchronize(st);
        if (arena) cudaFree(arena);
        if (st) cudaStreamDestroy(st);
    }
};

// One persistent scheduler launch and everything it uses: 2 * slots frontier
// queues, the mapped request ring and shared words, and a device block (ticket
// counter | 64 B control per slot | stats | chunk maps | queue views | graph
// table).  A run of the scheduler is an "episode": tickets restart at 0, the
// host publishes requests in ticket order, and the clusters leave when their
// ticket reaches the episode's limit or the host raises the stop word.
struct Persistent {
    const gq_serve_config& c;
    u32 slots = 0;
    Queues fr;
    void* dev = nullptr;
    void* mapped = nullptr;
    ServeEntry* ring = nullptr;
    ServeShared* sh = nullptr;
    u64 ring_n = 0;
    char* d = nullptr;
    u64 o_stats = 0;
    ServeK a;
    const gq_dev* dv = nullptr;
    cudaEvent_t ended = nullptr;
    bool running = false, stopping = false;
    u64 next_ticket = 0;
    std::vector<u64> entry_req;     // ring entry -> request whose ticket it holds
    std::vector<char> entry_busy;   // ring entry holds a ticket not yet seen done
    std::vector<u64> inflight;      // published tickets not yet seen done

    explicit Persistent(const gq_serve_config& cfg) : c(cfg) {}
    ~Persistent() {
        if (ended) cudaEventDestroy(ended);
        if (dev) cudaFree(dev);
        if (mapped) cudaFreeHost(mapped);
    }

    int init(u64 nmax, cudaStream_t st) {
        const u32 cb = c.cluster_blocks;
        int fit = 0;
        cudaError_t e = c.kind == GQ_LFQ ? max_clusters<GQ_LFQ>(cb, &fit)
                        : c.kind == GQ_WFQ ? max_clusters<GQ_WFQ>(cb, &fit)
                                           : max_clusters<GQ_YMC>(cb, &fit);
        if (e != cudaSuccess || fit < 1) return GQ_ERR_CUDA;
        slots = c.slots ? c.slots : (u32)fit;
        if (slots > (u32)fit) slots = (u32)fit;
        if ((u64)slots > c.nrequests) slots = c.nrequests;
        u32 gang = c.gang_clusters ? c.gang_clusters : 16;
        if (gang > slots) gang = slots;
        // a gang runs on its leader's queues: records for every thread of a gang
        int s = fr.create(2ull * slots, c.kind, queue_capacity(c.kind, nmax), cb * 256 * gang, st);
        if (s != GQ_OK) return s;

        ring_n = 1;
        while (ring_n < c.nrequests && ring_n < 4096) ring_n <<= 1;
        const u64 ring_bytes = ring_n * sizeof(ServeEntry);
        if (cudaHostAlloc(&mapped, ring_bytes + sizeof(ServeShared), cudaHostAllocMapped) != cudaSuccess) {
            mapped = nullptr;
            return GQ_ERR_NOMEM;
        }
        std::memset(mapped, 0, ring_bytes + sizeof(ServeShared));
        ring = static_cast<ServeEntry*>(mapped);
        sh = reinterpret_cast<ServeShared*>(static_cast<char*>(mapped) + ring_bytes);
        void* d_mapped = nullptr;
        if (cudaHostGetDevicePointer(&d_mapped, mapped, 0) != cudaSuccess) return GQ_ERR_CUDA;
        entry_req.assign(ring_n, 0);
        entry_busy.assign(ring_n, 0);

        const u64 o_ctl = 256;                       // claim counter at 0, open gang word at 128
        const u64 o_gang = round256(o_ctl + 64ull * slots);
        o_stats = round256(o_gang + 64ull * slots);
        const u64 o_tables = o_stats + 256,
                  o_views = round256(o_tables + slots * chunk_map_bytes(kServeChunkCap)),
                  o_graphs = round256(o_views + 2ull * slots * sizeof(gq_dev)),
                  total = round256(o_graphs + (u64)c.ngraphs * sizeof(gq_bfs_instance));
        if (cudaMalloc(&dev, total) != cudaSuccess) {
            dev = nullptr;
            return GQ_ERR_NOMEM;
        }
        d = static_cast<char*>(dev);
        std::vector<gq_dev> views(2ull * slots);
        for (u64 i = 0; i < views.size(); ++i) views[i] = fr.h[i]->dev;
        if (cudaMemsetAsync(d, 0, o_views, st) != cudaSuccess ||
            cudaMemcpyAsync(d + o_views, views.data(), views.size() * sizeof(gq_dev), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(d + o_graphs, c.graphs, (u64)c.ngraphs * sizeof(gq_bfs_instance),
                            cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return GQ_ERR_CUDA;
        if (cudaEventCreateWithFlags(&ended, cudaEventDisableTiming) != cudaSuccess) return GQ_ERR_CUDA;
        a.ring = static_cast<ServeEntry*>(d_mapped);
        a.sh = reinterpret_cast<ServeShared*>(static_cast<char*>(d_mapped) + ring_bytes);
        a.graphs = reinterpret_cast<const gq_bfs_instance*>(d + o_graphs);
        a.ngraphs = c.ngraphs;
        a.ring_mask = (u32)(ring_n - 1);
        a.nreq = 0;
        a.claim = reinterpret_cast<u64*>(d);
        a.ctl = reinterpret_cast<u64*>(d + o_ctl);
        a.stats = reinterpret_cast<unsigned long long*>(d + o_stats);
        a.tables = reinterpret_cast<u64*>(d + o_tables);
        a.wait_ns = (u64)((c.wait_limit_s > 0 ? c.wait_limit_s : 30.0) * 1e9);
        a.gang = reinterpret_cast<u64*>(d + o_gang);
        a.gang_open = reinterpret_cast<u64*>(d + 128);
        a.gang_max = gang;
        a.gang_min_n = c.gang_min_vertices ? c.gang_min_vertices : (1u << 17);
        dv = reinterpret_cast<const gq_dev*>(d + o_views);
        return GQ_OK;
    }

    // Launches an episode whose clusters leave once `limit` tickets are claimed.
    int start(u64 limit, cudaStream_t st) {
        for (u64 e = 0; e < ring_n; ++e) {
            ring[e].seq = 0;
            ring[e].done = 0;
        }
        __atomic_store_n(&sh->stop, 0ull, __ATOMIC_RELEASE);
        if (cudaMemsetAsync(a.claim, 0, 256, st) != cudaSuccess) return GQ_ERR_CUDA;   // claim, open gang
        a.nreq = limit;
        const cudaError_t e = c.kind == GQ_LFQ ? launch_serve<GQ_LFQ>(slots, c.cluster_blocks, dv, a, st)
                              : c.kind == GQ_WFQ ? launch_serve<GQ_WFQ>(slots, c.cluster_blocks, dv, a, st)
                                                 : launch_serve<GQ_YMC>(slots, c.cluster_blocks, dv, a, st);
        if (e != cudaSuccess || cudaEventRecord(ended, st) != cudaSuccess) return GQ_ERR_CUDA;
        running = true;
        stopping = false;
        next_ticket = 0;
        std::fill(entry_busy.begin(), entry_busy.end(), 0);
        return GQ_OK;
    }

    bool can_publish() const { return running && !stopping && !entry_busy[next_ticket & (ring_n - 1)]; }

    // Publishes request i (distances to dist) as the next ticket.
    void publish(u64 i, u32* dist) {
        const u64 t = next_ticket++;
        const u64 e = t & (ring_n - 1);
        ServeEntry* en = ring + e;
        en->req = (u64)c.req_graph[i] | ((u64)c.req_src[i] << 32);
        en->dist = reinterpret_cast<u64>(dist);
        en->levels = 0;
        entry_req[e] = i;
        entry_busy[e] = 1;
        __atomic_store_n(&en->seq, t + 1, __ATOMIC_RELEASE);
        inflight.push_back(t);
    }

    // Reports every published ticket now done (done(request, bad) for each).
    template <class F>
    void poll(F done) {
        for (u64 k = 0; k < inflight.size();) {
            const u64 t = inflight[k];
            ServeEntry* en = ring + (t & (ring_n - 1));
            if (__atomic_load_n(&en->done, __ATOMIC_ACQUIRE) == t + 1) {
                entry_busy[t & (ring_n - 1)] = 0;
                done(entry_req[t & (ring_n - 1)], en->levels == ~0ull);
                inflight[k] = inflight.back();
                inflight.pop_back();
            } else {
                ++k;
            }
        }
    }

    // Asks the clusters to leave at their next wait (only with nothing in flight,
    // so that no published ticket is left unclaimed).
    void stop() {
        __atomic_store_n(&sh->stop, 1ull, __ATOMIC_RELEASE);
        stopping = true;
    }

    // 1 if the episode's kernel has ended, 0 if it runs, < 0 on a CUDA error.
    int ended_yet() {
        const cudaError_t q = cudaEventQuery(ended);
        if (q == cudaErrorNotReady) return 0;
        if (q != cudaSuccess) return GQ_ERR_CUDA;
        running = stopping = false;
        return 1;
    }

    // Device error word and edge count (after the last episode ended).
    int finish(gq_serve_result& r, cudaStream_t st) {
        unsigned long long st3[4] = {0, 0, 0, 0};
        if (cudaStreamSynchronize(st) != cudaSuccess ||
            cudaMemcpy(st3, d + o_stats, sizeof(st3), cudaMemcpyDeviceToHost) != cudaSuccess)
            return GQ_ERR_CUDA;
        r.edges_scanned = st3[0];
        r.persistent_requests = st3[1];
        r.gang_requests = st3[3];
        if (st3[2]) return st3[2] == 2 ? GQ_ERR_INVALID : GQ_ERR_TIMEOUT;
        return fr.status(st);
    }
};

// One gq_bfs launch per request (the whole GPU), in order on one stream.
struct PerRequest {
    const gq_serve_config& c;
    Queues fr;
    std::vector<cudaEvent_t> ev;
    std::deque<u64> pending;        // launched requests, in launch (= completion) order
    u64 launched = 0;

    explicit PerRequest(const gq_serve_config& cfg) : c(cfg) {}
    ~PerRequest() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    int init(u64 nmax, cudaStream_t st) {
        // gq_bfs runs one thread per resident slot of the GPU: one record each
        uint64_t bt = 0;
        int s = gq_bfs_grid_threads(c.kind, &bt);
        if (s != GQ_OK) return s;
        s = fr.create(2, c.kind, queue_capacity(c.kind, nmax), (uint32_t)(bt < (1u << 20) ? bt : (1u << 20)), st);
        if (s != GQ_OK) return s;
        const u64 nev = c.nrequests < 1024 ? c.nrequests : 1024;
        ev.assign(nev, nullptr);
        for (u64 i = 0; i < nev; ++i)
            if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) return GQ_ERR_CUDA;
        return cudaStreamSynchronize(st) == cudaSuccess ? GQ_OK : GQ_ERR_CUDA;
    }
    bool can_launch() const { return pending.size() < ev.size(); }
    int launch(u64 i, u32* dist, cudaStream_t st) {
        const gq_bfs_instance& g = c.graphs[c.req_graph[i]];
        if (c.kind == GQ_YMC && (gq_reset(fr.h[0], st) != GQ_OK || gq_reset(fr.h[1], st) != GQ_OK))
            return GQ_ERR_CUDA;
        const int s = gq_bfs(fr.h[0], fr.h[1], g.n, g.d_offsets, g.d_adj, c.req_src[i], dist, nullptr, st);
        if (s != GQ_OK) return s;
        if (cudaEventRecord(ev[launched % ev.size()], st) != cudaSuccess) return GQ_ERR_CUDA;
        ++launched;
        pending.push_back(i);
        return GQ_OK;
    }
    // Reports requests now done, in order; < 0 on a CUDA error.
    template <class F>
    int poll(F done) {
        while (!pending.empty()) {
            const cudaError_t q = cudaEventQuery(ev[(launched - pending.size()) % ev.size()]);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) return GQ_ERR_CUDA;
            const u64 i = pending.front();
            pending.pop_front();
            done(i);
        }
        return GQ_OK;
    }
};

// The host loop shared by the three modes.  Requests are started in arrival
// order (first come, first served) once admitted; `route` says where the next
// one goes.
int serve_loop(Runtime& rt, cudaStream_t st, u64 nmax) {
    const gq_serve_config& c = rt.c;
    const u64 n = c.nrequests;
    const double limit = c.wait_limit_s > 0 ? c.wait_limit_s : 30.0;
    const bool use_p = c.mode != GQ_SERVE_PER_REQUEST, use_r = c.mode != GQ_SERVE_PERSISTENT;
    Persistent P(c);
    PerRequest R(c);
    int s = GQ_OK;
    if (use_p && (s = P.init(nmax, st)) != GQ_OK) return s;
    if (use_r && (s = R.init(nmax, st)) != GQ_OK) return s;
    rt.r.slots_used = use_p ? P.slots : 0;
    // adaptive: the persistent scheduler takes over when this many launched
    // requests are still waiting on the stream, and hands back after idling
    const u64 switch_backlog = c.switch_backlog ? c.switch_backlog : 8;
    const double idle_s = 0.5e-3;

    rt.t0 = Clock::now();
    if (c.mode == GQ_SERVE_PERSISTENT && (s = P.start(n, st)) != GQ_OK) return s;
    u64 next = 0, done = 0;
    double last_progress = 0, idle_since = 0;
    int err = GQ_OK;
    auto finished = [&](u64 i) {
        rt.complete(i, rt.now());
        ++done;
        last_progress = rt.now();
    };
    for (u64 iter = 0; done < n && err == GQ_OK; ++iter) {
        const double t = rt.now();
        // start arrived requests in order
        while (next < n && c.req_arrival_s[next] <= t) {
            bool to_p = c.mode == GQ_SERVE_PERSISTENT;
            if (c.mode == GQ_SERVE_ADAPTIVE) {
                if (P.running && !P.stopping) to_p = true;
                else if (!P.running && R.pending.size() >= switch_backlog) {
                    if ((err = P.start(~0ull, st)) != GQ_OK) break;
                    to_p = true;
                } else if (P.running) {
                    break;                                 // stopping: wait for the scheduler to leave
                }
            }
            if (to_p ? !P.can_publish() : !R.can_launch()) break;
            u32* dist = nullptr;
            if (!rt.admit(next, &dist)) {
                if (!rt.waited[next]) {
                    rt.waited[next] = 1;
                    ++rt.r.admission_waits;
                }
                break;
            }
            if (to_p) {
                P.publish(next, dist);
            } else if ((err = R.launch(next, dist, st)) != GQ_OK) {
                break;
            }
            ++next;
        }
        if (err != GQ_OK) break;
        // completions
        if (use_p)
            P.poll([&](u64 i, bool bad) {
                if (bad && err == GQ_OK) err = GQ_ERR_INVALID;
                finished(i);
            });
        if (use_r && (s = R.poll(finished)) != GQ_OK) {
            err = s;
            break;
        }
        // adaptive: an idle scheduler hands back to per-request launches
        if (c.mode == GQ_SERVE_ADAPTIVE && P.running) {
            if (!P.stopping) {
                const bool idle = P.inflight.empty() && (next == n || c.req_arrival_s[next] > rt.now());
                if (!idle) {
                    idle_since = rt.now();
                } else if (rt.now() - idle_since > idle_s) {
                    P.stop();
                }
            }
            if (P.stopping && (s = P.ended_yet()) < 0) err = s;
        }
        if ((iter & 1023) == 1023 && c.mode == GQ_SERVE_PERSISTENT && P.running) {
            const int e = P.ended_yet();
            if (e < 0) {
                err = e;
            } else if (e == 1) {             // ended: every request it served is done now
                P.poll([&](u64 i, bool bad) {
                    if (bad && err == GQ_OK) err = GQ_ERR_INVALID;
                    finished(i);
                });
                if (done < n && err == GQ_OK) err = GQ_ERR_TIMEOUT;
            }
        }
        if ((iter & 1023) == 1023 && done < next) {
            const double now = rt.now();
            if (now - last_progress > limit + 5.0 && now - c.req_arrival_s[done < n ? done : n - 1] > limit + 5.0)
                err = GQ_ERR_TIMEOUT;
        }
    }
    if (use_p) {
        if (P.running) P.stop();
        const int f = P.finish(rt.r, st);
        if (err == GQ_OK && f != GQ_OK) err = f;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && err == GQ_OK) err = GQ_ERR_CUDA;
    if (use_r && err == GQ_OK) err = R.fr.status(st);
    return err;
}

int validate(const gq_serve_config* c, const gq_serve_result* r) {
    if (!c || !r || !r->latency_s) return GQ_ERR_INVALID;
    if (c->kind != GQ_LFQ && c->kind != GQ_WFQ && c->kind != GQ_YMC) return GQ_ERR_INVALID;
    if (c->mode != GQ_SERVE_PERSISTENT && c->mode != GQ_SERVE_PER_REQUEST && c->mode != GQ_SERVE_ADAPTIVE)
        return GQ_ERR_INVALID;
    if (c->mode != GQ_SERVE_PER_REQUEST && c->cluster_blocks != 1 && c->cluster_blocks != 2 &&
        c->cluster_blocks != 4 && c->cluster_blocks != 8 && c->cluster_blocks != 16)
        return GQ_ERR_INVALID;
    if (!c->ngraphs || !c->nrequests || !c->graphs || !c->req_graph || !c->req_src || !c->req_arrival_s)
        return GQ_ERR_INVALID;
    if (!(c->wait_limit_s >= 0) || c->budget_bytes == 0) return GQ_ERR_INVALID;
    if (c->gang_clusters > 64 || c->reserved != 0) return GQ_ERR_INVALID;
    for (u32 g = 0; g < c->ngraphs; ++g) {
        const gq_bfs_instance& x = c->graphs[g];
        if (x.n == 0 || x.n >= 0xFFFFFFFFull || !x.d_offsets || !x.d_adj) return GQ_ERR_INVALID;
    }
    for (u32 i = 0; i < c->nrequests; ++i) {
        if (c->req_graph[i] >= c->ngraphs || c->req_src[i] >= c->graphs[c->req_graph[i]].n) return GQ_ERR_INVALID;
        if (!(c->req_arrival_s[i] >= 0) || (i && c->req_arrival_s[i] < c->req_arrival_s[i - 1]))
            return GQ_ERR_INVALID;
    }
    return GQ_OK;
}

}  // namespace

extern "C" int gq_serve(const gq_serve_config* cfg, gq_serve_result* res) {
    int s = validate(cfg, res);
    if (s != GQ_OK) return s;
    const gq_serve_config& c = *cfg;
    res->wall_s = 0;
    res->peak_state_bytes = res->admission_waits = res->edges_scanned = res->persistent_requests = 0;
    res->slots_used = 0;
    res->gang_requests = 0;
    res->status = GQ_OK;
    for (u32 i = 0; i < c.nrequests; ++i) res->latency_s[i] = -1.0;

    // per-graph state: CSR bytes need m = offsets[n], read once from the device
    std::vector<u64> graph_charge(c.ngraphs), graph_dist(c.ngraphs);
    u64 nmax = 1;
    // Per-thread queue records (G-WFQ, G-WFQ-YMC) are counted for the threads
    // that run a request: a cluster in the persistent scheduler (a gang of
    // clusters for a graph large enough to form one), the whole cooperative
    // grid of one gq_bfs launch otherwise (adaptive mode may run a request
    // either way and counts the larger).
    u32 mt = c.cluster_blocks * 256;
    if (c.mode != GQ_SERVE_PERSISTENT) {
        uint64_t bt = 0;
        if ((s = gq_bfs_grid_threads(c.kind, &bt)) != GQ_OK) return res->status = s;
        mt = (u32)(bt < (1u << 20) ? bt : (1u << 20));
    }
    for (u32 g = 0; g < c.ngraphs; ++g) {
        const gq_bfs_instance& x = c.graphs[g];
        u64 m = 0;
        if (cudaMemcpy(&m, x.d_offsets + x.n, sizeof(u64), cudaMemcpyDeviceToHost) != cudaSuccess)
            return res->status = GQ_ERR_CUDA;
        // a request that may be served by a gang counts a gang's threads
        u32 mtg = mt;
        const u32 gang = c.gang_clusters ? c.gang_clusters : 16;
        const u64 gmin = c.gang_min_vertices ? c.gang_min_vertices : (1u << 17);
        if (c.mode != GQ_SERVE_PER_REQUEST && gang > 1 && x.n >= gmin && c.cluster_blocks * 256 * gang > mtg)
            mtg = c.cluster_blocks * 256 * gang;
        uint64_t qb = 0;
        s = gq_workspace_bytes(c.kind, queue_capacity(c.kind, x.n), 4, mtg, nullptr, &qb);
        if (s != GQ_OK) return res->status = s;
        graph_dist[g] = round256(4 * x.n);
        graph_charge[g] = 8 * (x.n + 1) + 4 * m + graph_dist[g] + 2 * qb;
        if (x.n > nmax) nmax = x.n;
    }
    u64 arena_need = 0;
    for (u32 i = 0; i < c.nrequests; ++i) {
        const u32 g = c.req_graph[i];
        if (graph_charge[g] > c.budget_bytes) return res->status = GQ_ERR_INVALID;
        if (!c.req_out || !c.req_out[i]) arena_need += graph_dist[g];
    }
    const u64 arena_size = arena_need < c.budget_bytes ? arena_need : c.budget_bytes;
    Runtime rt(c, *res, arena_size);
    rt.charge.resize(c.nrequests);
    rt.dist_bytes.resize(c.nrequests);
    rt.arena_off.assign(c.nrequests, ~0ull);
    rt.finished.assign(c.nrequests, 0);
    rt.waited.assign(c.nrequests, 0);
    for (u32 i = 0; i < c.nrequests; ++i) {
        rt.charge[i] = graph_charge[c.req_graph[i]];
        rt.dist_bytes[i] = graph_dist[c.req_graph[i]];
    }

    Buffers b;
    if (cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking) != cudaSuccess) return res->status = GQ_ERR_CUDA;
    if (arena_size && cudaMalloc(&b.arena, arena_size) != cudaSuccess) {
        b.arena = nullptr;
        return res->status = GQ_ERR_NOMEM;
    }
    rt.d_arena = b.arena;
    s = serve_loop(rt, b.st, nmax);
    double last = 0;
    for (u32 i = 0; i < c.nrequests; ++i)
        if (rt.finished[i] && c.req_arrival_s[i] + res->latency_s[i] > last)
            last = c.req_arrival_s[i] + res->latency_s[i];
    res->wall_s = last - c.req_arrival_s[0];
    return res->status = s;
}
