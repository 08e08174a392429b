// Sequential CPU ray tracer: the per-pixel radiance that the wavefront GPU
// ray tracer must reproduce.  Test infrastructure only (see oracle.h).
// Built with -ffp-contract=off: every multiply and add below is rounded on
// its own, in the order written.
#include "oracle.h"

#include <math.h>

#include <thread>
#include <vector>

namespace {

inline uint64_t sm64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

inline float uni(uint64_t seed, uint64_t key) {
    return (float)(sm64(seed, key) >> 40) * (1.0f / 16777216.0f);
}

struct V3 {
    float x, y, z;
};

inline float dot3(V3 a, V3 b) {
    float s = a.x * b.x;
    s = s + a.y * b.y;
    s = s + a.z * b.z;
    return s;
}

// radiance of one pixel; counts traced segments
void trace_pixel(const orc_rt_scene& S, int64_t pix, float* out, int32_t* segs) {
    const int px = (int)(pix % S.width), py = (int)(pix / S.width);
    const float fx = ((float)px + 0.5f) / (float)S.width;
    const float fy = ((float)py + 0.5f) / (float)S.height;
    const float u = (2.0f * fx - 1.0f) * S.scale_x;
    const float v = (1.0f - 2.0f * fy) * S.scale_y;
    const float len0 = sqrtf(u * u + v * v + 1.0f);
    V3 o = {S.cam_x, S.cam_y, S.cam_z};
    V3 d = {u / len0, v / len0, 1.0f / len0};
    V3 tp = {1.0f, 1.0f, 1.0f};
    int nseg = 0;
    for (int bounce = 0;; ++bounce) {
        ++nseg;
        float best = INFINITY;
        int hit = -1;
        for (int k = 0; k < S.nspheres; ++k) {
            const V3 oc = {o.x - S.centre[3 * k], o.y - S.centre[3 * k + 1], o.z - S.centre[3 * k + 2]};
            const float b = dot3(oc, d);
            const float r = S.radius[k];
            const float cc = dot3(oc, oc) - r * r;
            const float disc = b * b - cc;
            if (disc < 0.0f) continue;
            const float sq = sqrtf(disc);
            float t = -b - sq;
            if (!(t > 1e-4f)) t = -b + sq;
            if (t > 1e-4f && t < best) {
                best = t;
                hit = k;
            }
        }
        if (hit < 0) {
            const float s = 0.5f * (d.y + 1.0f);
            out[0] = tp.x * ((1.0f - s) + s * 0.5f);
            out[1] = tp.y * ((1.0f - s) + s * 0.7f);
            out[2] = tp.z * ((1.0f - s) + s * 1.0f);
            break;
        }
        if (bounce == S.max_bounces) {
            out[0] = out[1] = out[2] = 0.0f;
            break;
        }
        const V3 p = {o.x + best * d.x, o.y + best * d.y, o.z + best * d.z};
        const float r = S.radius[hit];
        const V3 n = {(p.x - S.centre[3 * hit]) / r, (p.y - S.centre[3 * hit + 1]) / r,
                      (p.z - S.centre[3 * hit + 2]) / r};
        tp = {tp.x * S.albedo[3 * hit], tp.y * S.albedo[3 * hit + 1], tp.z * S.albedo[3 * hit + 2]};
        V3 q = {0.0f, 0.0f, 0.0f};
        for (int a = 0; a < 32; ++a) {
            const uint64_t key = (((uint64_t)pix * 16 + (uint64_t)bounce) * 64 + (uint64_t)a) * 4;
            const V3 c = {2.0f * uni(S.seed, key) - 1.0f, 2.0f * uni(S.seed, key + 1) - 1.0f,
                          2.0f * uni(S.seed, key + 2) - 1.0f};
            if (dot3(c, c) < 1.0f) {
                q = c;
                break;
            }
        }
        const V3 w = {n.x + q.x, n.y + q.y, n.z + q.z};
        const float l2 = dot3(w, w);
        if (l2 <= 1e-12f) {
            d = n;
        } else {
            const float l = sqrtf(l2);
            d = {w.x / l, w.y / l, w.z / l};
        }
        o = p;
    }
    if (segs) *segs = nseg;
}

}  // namespace

extern "C" void orc_render_pixels(const orc_rt_scene* scene, const int64_t* pixels, int64_t m, float* rgb,
                                  int32_t* segments, int32_t threads) {
    if (threads < 1) threads = 1;
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([=] {
            for (int64_t i = t; i < m; i += threads)
                trace_pixel(*scene, pixels[i], rgb + 3 * i, segments ? segments + i : nullptr);
        });
    for (auto& th : pool) th.join();
}
