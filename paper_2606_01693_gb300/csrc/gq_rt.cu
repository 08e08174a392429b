// Tile-based wavefront ray tracer on the queues (include/gq_apps.h, gq_render).
//
// Compiled with -fmad=false: every multiply and add is rounded on its own, in
// the order written, so the radiance matches a sequential CPU trace bit for
// bit (IEEE division and square root are nvcc's defaults).
//
// Work distribution: each tile has a queue of pixel indices and a count of the
// items in it that no warp has reserved yet.  A warp picks a tile, reserves up
// to 32 items from its count (so every dequeue it then issues finds an item:
// the queue is linearizable and the reserved items are in it), traces one
// segment per item, and re-enqueues the scattered rays into the same tile
// before adding them back to the count.  Warps that find a tile empty move on
// to the next one; all exit when the device work counter (pixels not yet
// finished) reaches zero.  Idle waiting is bounded.
#include <cuda_runtime.h>

#include <string.h>
#include <vector>

#include "../../include/gq_apps.h"
#include "gq_host.h"
#include "gq_ops.cuh"

using namespace gqd;

namespace {

constexpr u32 kMaxSpheres = 8192;
constexpr u32 kIdleLimit = 1u << 24;

struct RtWs {            // device workspace layout (byte offsets)
    u64 devs, pending, ctl, state, total;
};

RtWs rt_layout(const gq_rt_scene& s) {
    RtWs w;
    const u64 ntiles = (u64)s.tiles_x * s.tiles_y;
    const u64 npix = (u64)s.width * s.height;
    u64 off = 0;
    w.devs = off;    off += (ntiles * sizeof(gq_dev) + 255) / 256 * 256;
    w.pending = off; off += (ntiles * 8 + 255) / 256 * 256;
    w.ctl = off;     off += 256;
    w.state = off;   off += 10 * npix * 4;   // ox oy oz dx dy dz tr tg tb bounce
    w.total = (off + 255) / 256 * 256;
    return w;
}

struct RtK {
    u32 width, height, tiles_x, tiles_y, tile_w, tile_h, max_bounces, nspheres;
    float cam_x, cam_y, cam_z, scale_x, scale_y;
    u64 seed;
    const float* centre;
    const float* radius;
    const float* albedo;
    const gq_dev* tq;       // per-tile queue views (device copy)
    long long* pending;     // per-tile unreserved items
    u64* ctl;               // [0] pixels left, [1] segments, [2] errors
    float* st;              // ray state, structure of arrays
    float* image;
};

__device__ __forceinline__ u64 rt_sm64(u64 seed, u64 k) {
    u64 z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float rt_uni(u64 seed, u64 key) {
    return (float)(rt_sm64(seed, key) >> 40) * (1.0f / 16777216.0f);
}
__device__ __forceinline__ float rt_dot(float ax, float ay, float az, float bx, float by, float bz) {
    float s = ax * bx;
    s = s + ay * by;
    s = s + az * bz;
    return s;
}

__device__ __forceinline__ u32 tile_of(const RtK& k, u32 pix) {
    const u32 px = pix % k.width, py = pix / k.width;
    return (py / k.tile_h) * k.tiles_x + px / k.tile_w;
}

// Primary rays: state of every pixel, then its index into the tile's queue.
template <int KIND>
__global__ void __launch_bounds__(256) k_rt_primary(const __grid_constant__ RtK k) {
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    const u64 npix = (u64)k.width * k.height;
    for (u64 p = tid; p < npix; p += (u64)gridDim.x * blockDim.x) {
        const u32 px = (u32)(p % k.width), py = (u32)(p / k.width);
        const float fx = ((float)px + 0.5f) / (float)k.width;
        const float fy = ((float)py + 0.5f) / (float)k.height;
        const float u = (2.0f * fx - 1.0f) * k.scale_x;
        const float v = (1.0f - 2.0f * fy) * k.scale_y;
        const float len0 = sqrtf(u * u + v * v + 1.0f);
        float* st = k.st;
        st[0 * npix + p] = k.cam_x;
        st[1 * npix + p] = k.cam_y;
        st[2 * npix + p] = k.cam_z;
        st[3 * npix + p] = u / len0;
        st[4 * npix + p] = v / len0;
        st[5 * npix + p] = 1.0f / len0;
        st[6 * npix + p] = 1.0f;
        st[7 * npix + p] = 1.0f;
        st[8 * npix + p] = 1.0f;
        reinterpret_cast<u32*>(st)[9 * npix + p] = 0;
        const u32 t = tile_of(k, (u32)p);
        if (queue_enqueue<unsigned int, KIND, true>(k.tq[t], (unsigned)p, tid) == GQ_OK)
            atomicAdd(reinterpret_cast<unsigned long long*>(k.pending + t), 1ull);
        else
            atomicOr(reinterpret_cast<unsigned long long*>(k.ctl + 2), 4ull);
    }
}

// Reserves up to 32 unreserved items of tile t (lane 0 does the atomics).
__device__ __forceinline__ u32 rt_reserve(long long* pending, u32 t) {
    u32 got = 0;
    if (lane_id() == 0) {
        long long p = aref<long long>(pending[t]).load(kRlx);
        for (int a = 0; a < 8 && p > 0; ++a) {
            const long long want = p < 32 ? p : 32;
            if (aref<long long>(pending[t]).compare_exchange_strong(p, p - want, kAR, kRlx)) {
                got = (u32)want;
                break;
            }
        }
    }
    return __shfl_sync(0xffffffffu, got, 0);
}

template <int KIND>
__global__ void __launch_bounds__(256) k_rt_trace(const __grid_constant__ RtK k) {
    extern __shared__ float4 sph[];
    for (u32 i = threadIdx.x; i < k.nspheres; i += blockDim.x)
        sph[i] = make_float4(k.centre[3 * i], k.centre[3 * i + 1], k.centre[3 * i + 2], k.radius[i] * k.radius[i]);
    __syncthreads();
    const u32 tid = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 lane = threadIdx.x & 31;
    const u32 ntiles = k.tiles_x * k.tiles_y;
    const u64 npix = (u64)k.width * k.height;
    u32 tile = (tid >> 5) % ntiles;
    u32 idle = 0;
    u64 segs = 0;
    float* st = k.st;
    u32* bnc = reinterpret_cast<u32*>(st) + 9 * npix;
    for (;;) {
        const u32 nres = rt_reserve(k.pending, tile);
        if (nres == 0) {
            if (ld_acq(k.ctl) == 0) break;                      // every pixel finished
            tile = (tile + 1) % ntiles;
            if (++idle > kIdleLimit) {
                if (lane == 0) atomicOr(reinterpret_cast<unsigned long long*>(k.ctl + 2), 1ull);
                break;
            }
            if (idle % ntiles == 0) __nanosleep(256);
            continue;
        }
        idle = 0;
        unsigned int pix = 0;
        bool have = false;
        if (lane < nres) {
            have = queue_dequeue<unsigned int, KIND>(k.tq[tile], &pix, tid) == GQ_OK;
            if (!have) atomicOr(reinterpret_cast<unsigned long long*>(k.ctl + 2), 2ull);
        }
        bool again = false, done = false;
        if (have) {
            ++segs;
            const u64 p = pix;
            float ox = st[0 * npix + p], oy = st[1 * npix + p], oz = st[2 * npix + p];
            float dx = st[3 * npix + p], dy = st[4 * npix + p], dz = st[5 * npix + p];
            float tr = st[6 * npix + p], tg = st[7 * npix + p], tb = st[8 * npix + p];
            const u32 bounce = bnc[p];
            float best = __int_as_float(0x7f800000);   // +infinity
            int hit = -1;
            // sph[s].w holds r * r (the same fp32 product the test would form)
#pragma unroll 4
            for (u32 s = 0; s < k.nspheres; ++s) {
                const float4 c = sph[s];
                const float ocx = ox - c.x, ocy = oy - c.y, ocz = oz - c.z;
                const float b = rt_dot(ocx, ocy, ocz, dx, dy, dz);
                const float cc = rt_dot(ocx, ocy, ocz, ocx, ocy, ocz) - c.w;
                const float disc = b * b - cc;
                if (disc < 0.0f) continue;
                const float sq = sqrtf(disc);
                float t = -b - sq;
                if (!(t > 1e-4f)) t = -b + sq;
                if (t > 1e-4f && t < best) {
                    best = t;
                    hit = (int)s;
                }
            }
            float* img = k.image + 3 * p;
            if (hit < 0) {
                const float sk = 0.5f * (dy + 1.0f);
                img[0] = tr * ((1.0f - sk) + sk * 0.5f);
                img[1] = tg * ((1.0f - sk) + sk * 0.7f);
                img[2] = tb * ((1.0f - sk) + sk * 1.0f);
                done = true;
            } else if (bounce == k.max_bounces) {
                img[0] = 0.0f;
                img[1] = 0.0f;
                img[2] = 0.0f;
                done = true;
            } else {
                const float4 c = sph[hit];
                const float hx = ox + best * dx, hy = oy + best * dy, hz = oz + best * dz;
                const float rad = k.radius[hit];     // sph[].w holds the squared radius
                const float nx = (hx - c.x) / rad, ny = (hy - c.y) / rad, nz = (hz - c.z) / rad;
                tr = tr * k.albedo[3 * hit];
                tg = tg * k.albedo[3 * hit + 1];
                tb = tb * k.albedo[3 * hit + 2];
                float qx = 0.0f, qy = 0.0f, qz = 0.0f;
                for (u32 a = 0; a < 32; ++a) {
                    const u64 key = ((p * 16 + (u64)bounce) * 64 + (u64)a) * 4;
                    const float cx = 2.0f * rt_uni(k.seed, key) - 1.0f;
                    const float cy = 2.0f * rt_uni(k.seed, key + 1) - 1.0f;
                    const float cz = 2.0f * rt_uni(k.seed, key + 2) - 1.0f;
                    if (rt_dot(cx, cy, cz, cx, cy, cz) < 1.0f) {
                        qx = cx;
                        qy = cy;
                        qz = cz;
                        break;
                    }
                }
                const float wx = nx + qx, wy = ny + qy, wz = nz + qz;
                const float l2 = rt_dot(wx, wy, wz, wx, wy, wz);
                if (l2 <= 1e-12f) {
                    dx = nx;
                    dy = ny;
                    dz = nz;
                } else {
                    const float l = sqrtf(l2);
                    dx = wx / l;
                    dy = wy / l;
                    dz = wz / l;
                }
                st[0 * npix + p] = hx;
                st[1 * npix + p] = hy;
                st[2 * npix + p] = hz;
                st[3 * npix + p] = dx;
                st[4 * npix + p] = dy;
                st[5 * npix + p] = dz;
                st[6 * npix + p] = tr;
                st[7 * npix + p] = tg;
                st[8 * npix + p] = tb;
                bnc[p] = bounce + 1;
                again = true;
            }
        }
        if (again) {
            if (queue_enqueue<unsigned int, KIND>(k.tq[tile], pix, tid) == GQ_OK) {
                const u64 base = warp_faa<false>(reinterpret_cast<u64*>(k.pending + tile), 1, 32);
                (void)base;
            } else {
                atomicOr(reinterpret_cast<unsigned long long*>(k.ctl + 2), 4ull);
            }
        }
        if (done) warp_faa<false>(k.ctl, ~0ull, 32);          // pixels left -= 1 per finished lane
        __syncwarp();
    }
    warp_add_full(reinterpret_cast<unsigned long long*>(k.ctl + 1), segs);
}

__global__ void k_rt_stats(const u64* ctl, u64 npix, u32 ntiles, unsigned long long* stats) {
    stats[0] = ctl[1];
    stats[1] = npix - ctl[0];
    stats[2] = ctl[2];
    stats[3] = ntiles;
}

template <int KIND>
int launch_rt(const gq_handle* tiles, const gq_rt_scene& s, void* ws, float* image, unsigned long long* stats,
              cudaStream_t st) {
    const RtWs w = rt_layout(s);
    const u32 ntiles = s.tiles_x * s.tiles_y;
    char* b = static_cast<char*>(ws);
    std::vector<gq_dev> devs(ntiles);
    u32 rec = 0xFFFFFFFFu;
    for (u32 t = 0; t < ntiles; ++t) {
        devs[t] = tiles[t]->dev;
        if (tiles[t]->dev.max_threads < rec) rec = tiles[t]->dev.max_threads;
    }
    if (cudaMemcpyAsync(b + w.devs, devs.data(), ntiles * sizeof(gq_dev), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return GQ_ERR_CUDA;
    if (cudaMemsetAsync(b + w.pending, 0, ntiles * 8, st) != cudaSuccess) return GQ_ERR_CUDA;
    const u64 npix = (u64)s.width * s.height;
    if (cudaMemcpyAsync(b + w.ctl, &npix, 8, cudaMemcpyHostToDevice, st) != cudaSuccess) return GQ_ERR_CUDA;
    if (cudaMemsetAsync(b + w.ctl + 8, 0, 16, st) != cudaSuccess) return GQ_ERR_CUDA;
    RtK k;
    memset(&k, 0, sizeof(k));
    k.width = s.width;
    k.height = s.height;
    k.tiles_x = s.tiles_x;
    k.tiles_y = s.tiles_y;
    k.tile_w = (s.width + s.tiles_x - 1) / s.tiles_x;
    k.tile_h = (s.height + s.tiles_y - 1) / s.tiles_y;
    k.max_bounces = s.max_bounces;
    k.nspheres = s.nspheres;
    k.cam_x = s.cam_x;
    k.cam_y = s.cam_y;
    k.cam_z = s.cam_z;
    k.scale_x = s.scale_x;
    k.scale_y = s.scale_y;
    k.seed = s.seed;
    k.centre = s.d_centre;
    k.radius = s.d_radius;
    k.albedo = s.d_albedo;
    k.tq = reinterpret_cast<const gq_dev*>(b + w.devs);
    k.pending = reinterpret_cast<long long*>(b + w.pending);
    k.ctl = reinterpret_cast<u64*>(b + w.ctl);
    k.st = reinterpret_cast<float*>(b + w.state);
    k.image = image;
    const size_t smem = (size_t)s.nspheres * sizeof(float4);
    if (cudaFuncSetAttribute(k_rt_trace<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GQ_ERR_CUDA;
    int sms = 0, occ = 0, occp = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, tiles[0]->device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rt_trace<KIND>, 256, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occp, k_rt_primary<KIND>, 256, 0) != cudaSuccess)
        return GQ_ERR_CUDA;
    u64 grid = (u64)(occ > 0 ? occ : 1) * sms;
    u64 gridp = (u64)(occp > 0 ? occp : 1) * sms;
    if (KIND != GQ_LFQ) {
        if (grid > rec / 256) grid = rec / 256;
        if (gridp > rec / 256) gridp = rec / 256;
    }
    if (grid < 1 || gridp < 1) return GQ_ERR_TOO_MANY_THREADS;
    k_rt_primary<KIND><<<(unsigned)gridp, 256, 0, st>>>(k);
    k_rt_trace<KIND><<<(unsigned)grid, 256, smem, st>>>(k);
    if (stats) k_rt_stats<<<1, 1, 0, st>>>(k.ctl, npix, ntiles, stats);
    return gq_check_launch();
}

bool scene_ok(const gq_rt_scene* s) {
    return s && s->width > 0 && s->height > 0 && s->tiles_x > 0 && s->tiles_y > 0 && s->tiles_x <= s->width &&
           s->tiles_y <= s->height && (u64)s->width * s->height < (1ull << 32) && s->nspheres <= kMaxSpheres &&
           s->max_bounces <= 15 && (s->nspheres == 0 || (s->d_centre && s->d_radius && s->d_albedo));
}

}  // namespace

extern "C" int gq_render_workspace_bytes(const gq_rt_scene* scene, uint64_t* bytes) {
    if (!scene_ok(scene) || !bytes) return GQ_ERR_INVALID;
    *bytes = rt_layout(*scene).total;
    return GQ_OK;
}

extern "C" int gq_render(const gq_handle* tiles, const gq_rt_scene* scene, void* d_workspace, float* d_image,
                         unsigned long long* d_stats, void* stream) {
    if (!scene_ok(scene) || !tiles || !d_workspace || !d_image) return GQ_ERR_INVALID;
    const u32 ntiles = scene->tiles_x * scene->tiles_y;
    for (u32 t = 0; t < ntiles; ++t) {
        if (!tiles[t] || tiles[t]->dev.elem_bytes != 4 || tiles[t]->dev.kind != tiles[0]->dev.kind ||
            tiles[t]->device != tiles[0]->device)
            return GQ_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (tiles[0]->dev.kind) {
        case GQ_LFQ: return launch_rt<GQ_LFQ>(tiles, *scene, d_workspace, d_image, d_stats, st);
        case GQ_WFQ: return launch_rt<GQ_WFQ>(tiles, *scene, d_workspace, d_image, d_stats, st);
        default: return launch_rt<GQ_YMC>(tiles, *scene, d_workspace, d_image, d_stats, st);
    }
}
