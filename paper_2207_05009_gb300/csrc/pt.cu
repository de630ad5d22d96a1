// The luminaire as an emitter inside a small path tracer (paper Sec. 3,
// Eq. 2: what leaves the proxy is L_o = L_e + T L_i; Sec. 5, "Sampling": the
// proxy surface is sampled uniformly for next-event estimation).
//
// Scene: a closed room (an axis-aligned box with diffuse walls, seen from
// inside) holding the luminaire, whose proxy is the tree's bounding box.
// Paths are traced as a wavefront.  Per bounce every path queries the
// luminaire twice through plo_render_rays:
//   along its own ray: camera rays add the L_e they see, and every ray's
//     throughput is multiplied by T (light from behind the luminaire passes
//     through it attenuated, the second term of Eq. 2);
//   along the next-event ray from its wall point x toward a point y drawn
//     uniformly on the proxy surface: when y lies on a face that faces x it
//     is where that ray enters the proxy, and the luminaire's emission along
//     it arrives at x; the estimate is
//       thr * (rho / pi) * L_e(x -> y) * cos_x * cos_y / |y - x|^2 * A,
//     A the proxy's surface area.
// Then a cosine-weighted bounce off the wall (throughput *= rho).  Light
// reaches the camera only through the luminaire (the walls do not emit), so
// indirect rays do not add L_e (next-event estimation counted it).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "plo_internal.h"

using namespace plo;

namespace {

constexpr float PI_F = 3.14159265358979323846f;

__device__ __forceinline__ uint64_t pt_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

struct PtArgs {
    plo_pt_scene sc;
    float bmin[3], bmax[3];  // proxy box (world)
    float face_cdf[6];       // cumulative face areas / total
    float area;              // total proxy surface area
    const float* uni;        // [paths][dims] or NULL
    uint64_t seed;
    int dims;
    int64_t base;            // first global path index of this chunk
    int64_t n;               // paths in this chunk
    float* ray;              // [n][6] current ray (query A input)
    float* thr;              // [n][3]
    float* L;                // [n][3]
    float* nee_ray;          // [n][6] (query B input)
    float* nee_w;            // [n][3]
    const float* rgbA;
    const float* TA;
    const float* rgbB;
};

__device__ __forceinline__ float pt_u(const PtArgs& a, int64_t p, int k) {
    if (a.uni) return __ldg(a.uni + p * a.dims + k);
    const uint64_t z = pt_mix(pt_mix(a.seed ^ 0x7A7E57ULL) ^ ((uint64_t)p * 0x9E3779B97F4A7C15ULL + (uint64_t)k));
    return (float)(z >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ void normalize3(float* v) {
    const float s = rsqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] *= s;
    v[1] *= s;
    v[2] *= s;
}

// Camera rays: pixel (px + u0, py + u1) of a pinhole camera.
__global__ void k_pt_camera(PtArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int64_t p = a.base + i;
    const int64_t pix = p % ((int64_t)a.sc.width * a.sc.height);
    const int px = (int)(pix % a.sc.width), py = (int)(pix / a.sc.width);
    float fwd[3], right[3], up[3];
    for (int k = 0; k < 3; ++k) fwd[k] = a.sc.cam_target[k] - a.sc.cam_pos[k];
    normalize3(fwd);
    right[0] = fwd[1] * a.sc.cam_up[2] - fwd[2] * a.sc.cam_up[1];
    right[1] = fwd[2] * a.sc.cam_up[0] - fwd[0] * a.sc.cam_up[2];
    right[2] = fwd[0] * a.sc.cam_up[1] - fwd[1] * a.sc.cam_up[0];
    normalize3(right);
    up[0] = right[1] * fwd[2] - right[2] * fwd[1];
    up[1] = right[2] * fwd[0] - right[0] * fwd[2];
    up[2] = right[0] * fwd[1] - right[1] * fwd[0];
    const float th = tanf(0.5f * a.sc.fov_y);
    const float sx = (2.0f * ((float)px + pt_u(a, p, 0)) / (float)a.sc.width - 1.0f) * th * (float)a.sc.width /
                     (float)a.sc.height;
    const float sy = (1.0f - 2.0f * ((float)py + pt_u(a, p, 1)) / (float)a.sc.height) * th;
    float d[3];
    for (int k = 0; k < 3; ++k) d[k] = fwd[k] + sx * right[k] + sy * up[k];
    normalize3(d);
    for (int k = 0; k < 3; ++k) {
        a.ray[6 * i + k] = a.sc.cam_pos[k];
        a.ray[6 * i + 3 + k] = d[k];
        a.thr[3 * i + k] = 1.0f;
        a.L[3 * i + k] = 0.0f;
    }
}

// The "explicitly handled" emitter of the overhead comparison: an opaque box
// of constant radiance in place of the luminaire.
__global__ void k_pt_box_query(PtArgs a, const float* rays, float* rgb, float* T) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    float tn = -INFINITY, tf = INFINITY;
    bool miss = false;
    for (int k = 0; k < 3; ++k) {
        const float o = rays[6 * i + k], d = rays[6 * i + 3 + k];
        if (d == 0.0f) {
            miss |= o < a.bmin[k] || o > a.bmax[k];
            continue;
        }
        const float t0 = (a.bmin[k] - o) / d, t1 = (a.bmax[k] - o) / d;
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
    const bool hit = !miss && tn < tf && tf > 0.0f;
    for (int k = 0; k < 3; ++k) rgb[3 * i + k] = hit ? a.sc.box_radiance[k] : 0.0f;
    T[i] = hit ? 0.0f : 1.0f;
}

// After query A: direct emission (camera rays), pass-through, wall hit,
// next-event ray and weight, cosine-weighted bounce.
__global__ void k_pt_wall(PtArgs a, int bounce) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int64_t p = a.base + i;
    float o[3], d[3], thr[3];
    for (int k = 0; k < 3; ++k) {
        o[k] = a.ray[6 * i + k];
        d[k] = a.ray[6 * i + 3 + k];
        thr[k] = a.thr[3 * i + k];
    }
    const float T = a.TA[i];
    for (int k = 0; k < 3; ++k) {
        if (bounce == 0) a.L[3 * i + k] += thr[k] * a.rgbA[3 * i + k];
        thr[k] *= T;
    }
    // wall: the room is seen from inside
    float tw = INFINITY;
    int ax = 0;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0f) continue;
        const float t = ((d[k] > 0.0f ? a.sc.room_max[k] : a.sc.room_min[k]) - o[k]) / d[k];
        if (t < tw) {
            tw = t;
            ax = k;
        }
    }
    const int wall = 2 * ax + (d[ax] > 0.0f ? 1 : 0);
    float x[3], n[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < 3; ++k) x[k] = o[k] + tw * d[k];
    x[ax] = d[ax] > 0.0f ? a.sc.room_max[ax] : a.sc.room_min[ax];
    n[ax] = d[ax] > 0.0f ? -1.0f : 1.0f;
    const int dim0 = 2 + 5 * bounce;
    // next-event estimation: y uniform on the proxy surface
    const float u2 = pt_u(a, p, dim0), u3 = pt_u(a, p, dim0 + 1), u4 = pt_u(a, p, dim0 + 2);
    int f = 0;
    while (f < 5 && u2 >= a.face_cdf[f]) ++f;
    const int fa = f >> 1, fb = (fa + 1) % 3, fc = (fa + 2) % 3;
    float y[3];
    y[fa] = (f & 1) ? a.bmax[fa] : a.bmin[fa];
    y[fb] = a.bmin[fb] + u3 * (a.bmax[fb] - a.bmin[fb]);
    y[fc] = a.bmin[fc] + u4 * (a.bmax[fc] - a.bmin[fc]);
    float w[3];
    for (int k = 0; k < 3; ++k) w[k] = y[k] - x[k];
    const float dist2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    normalize3(w);
    const bool faces = (f & 1) ? x[fa] > y[fa] : x[fa] < y[fa];
    const float cos_x = n[0] * w[0] + n[1] * w[1] + n[2] * w[2];
    const float cos_y = fabsf(w[fa]);
    const float g = (faces && cos_x > 0.0f) ? cos_x * cos_y / dist2 * a.area / PI_F : 0.0f;
    const float* rho = a.sc.albedo[wall];
    for (int k = 0; k < 3; ++k) {
        a.nee_ray[6 * i + k] = x[k];
        a.nee_ray[6 * i + 3 + k] = w[k];
        a.nee_w[3 * i + k] = thr[k] * rho[k] * g;
    }
    // cosine-weighted bounce about the inward normal
    const float u5 = pt_u(a, p, dim0 + 3), u6 = pt_u(a, p, dim0 + 4);
    const float r = sqrtf(u5), phi = 2.0f * PI_F * u6;
    float sp, cp;
    sincosf(phi, &sp, &cp);
    float nd[3];
    nd[ax] = n[ax] * sqrtf(fmaxf(0.0f, 1.0f - u5));
    nd[(ax + 1) % 3] = r * cp;
    nd[(ax + 2) % 3] = r * sp;
    for (int k = 0; k < 3; ++k) {
        a.ray[6 * i + k] = x[k];
        a.ray[6 * i + 3 + k] = nd[k];
        a.thr[3 * i + k] = thr[k] * rho[k];
    }
}

__global__ void k_pt_nee(PtArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    for (int k = 0; k < 3; ++k) a.L[3 * i + k] += a.nee_w[3 * i + k] * a.rgbB[3 * i + k];
}

__global__ void k_pt_store(PtArgs a, float* samples) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    for (int k = 0; k < 3; ++k) samples[3 * (a.base + i) + k] = a.L[3 * i + k];
}

// image[pixel] = mean over the samples, summed in sample order
__global__ void k_pt_resolve(const float* samples, int64_t pixels, int spp, float* image) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pixels) return;
    float s[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < spp; ++k)
        for (int c = 0; c < 3; ++c) s[c] += samples[3 * ((int64_t)k * pixels + i) + c];
    for (int c = 0; c < 3; ++c) image[3 * i + c] = s[c] / (float)spp;
}

plo_status check_scene(const plo_pt_scene* s) {
    if (!s) return set_error(PLO_ERR_INVALID_ARG, "scene is NULL");
    if (s->width <= 0 || s->height <= 0) return set_error(PLO_ERR_INVALID_ARG, "width and height must be > 0");
    if (s->max_bounces < 1 || s->max_bounces > 16) return set_error(PLO_ERR_INVALID_ARG, "max_bounces in [1, 16]");
    if (!(s->fov_y > 0.0f && s->fov_y < 3.1f)) return set_error(PLO_ERR_INVALID_ARG, "fov_y in (0, 3.1)");
    if (s->emitter != PLO_PT_OCTREE && s->emitter != PLO_PT_CONSTANT_BOX)
        return set_error(PLO_ERR_INVALID_ARG, "unknown emitter");
    for (int k = 0; k < 3; ++k)
        if (!(s->room_min[k] < s->room_max[k])) return set_error(PLO_ERR_INVALID_ARG, "room_min < room_max");
    return PLO_OK;
}

}  // namespace

extern "C" plo_status plo_pt_render(const plo_tree* lum, const plo_render_params* params, const plo_pt_scene* scene,
                                    int32_t spp, uint64_t seed, const float* d_uniforms, float* d_image,
                                    float* d_samples, void* stream) {
    if (!lum || !params || !d_image) return set_error(PLO_ERR_INVALID_ARG, "tree, params or image is NULL");
    plo_status st = check_scene(scene);
    if (st != PLO_OK) return st;
    if (spp < 1) return set_error(PLO_ERR_INVALID_ARG, "spp must be >= 1");
    if (params->proxy != PLO_PROXY_BOX)
        return set_error(PLO_ERR_UNSUPPORTED, "the path tracer samples the proxy box (PLO_PROXY_BOX only)");
    PtArgs a{};
    a.sc = *scene;
    float ext[3];
    for (int k = 0; k < 3; ++k) {
        a.bmin[k] = lum->bbox_min[k];
        ext[k] = 1.0f / lum->inv_ext[k];
        a.bmax[k] = a.bmin[k] + ext[k];
        if (!(a.bmin[k] >= scene->room_min[k] && a.bmax[k] <= scene->room_max[k]))
            return set_error(PLO_ERR_INVALID_ARG, "the luminaire's box must lie inside the room");
    }
    float fa[6];
    for (int f = 0; f < 6; ++f) fa[f] = ext[((f >> 1) + 1) % 3] * ext[((f >> 1) + 2) % 3];
    a.area = fa[0] + fa[1] + fa[2] + fa[3] + fa[4] + fa[5];
    float c = 0.0f;
    for (int f = 0; f < 6; ++f) a.face_cdf[f] = (c += fa[f]) / a.area;
    a.uni = d_uniforms;
    a.seed = seed;
    a.dims = 2 + 5 * scene->max_bounces;
    const int64_t pixels = (int64_t)scene->width * scene->height;
    const int64_t total = pixels * spp;
    const int64_t chunk = total < ((int64_t)1 << 22) ? total : ((int64_t)1 << 22);
    cudaStream_t s = (cudaStream_t)stream;
    // workspace: ray, thr, L, nee_ray, nee_w, rgbA, TA, rgbB, TB (+ samples)
    const size_t per = 6 + 3 + 3 + 6 + 3 + 3 + 1 + 3 + 1;
    float* ws = nullptr;
    float* own_samples = nullptr;
    cudaError_t e = (cudaError_t)dev_malloc_async((void**)&ws, (size_t)chunk * per * 4, s);
    if (e == cudaSuccess && !d_samples) e = (cudaError_t)dev_malloc_async((void**)&own_samples, (size_t)total * 12, s);
    if (e != cudaSuccess) {
        if (ws) cudaFreeAsync(ws, s);
        return cuda_error(e, "path tracer workspace");
    }
    float* samples = d_samples ? d_samples : own_samples;
    a.ray = ws;
    a.thr = a.ray + 6 * chunk;
    a.L = a.thr + 3 * chunk;
    a.nee_ray = a.L + 3 * chunk;
    a.nee_w = a.nee_ray + 6 * chunk;
    float* rgbA = a.nee_w + 3 * chunk;
    float* TA = rgbA + 3 * chunk;
    float* rgbB = TA + chunk;
    float* TB = rgbB + 3 * chunk;
    a.rgbA = rgbA;
    a.TA = TA;
    a.rgbB = rgbB;
    for (int64_t base = 0; st == PLO_OK && base < total; base += chunk) {
        a.base = base;
        a.n = total - base < chunk ? total - base : chunk;
        const unsigned blocks = (unsigned)((a.n + 255) / 256);
        k_pt_camera<<<blocks, 256, 0, s>>>(a);
        for (int b = 0; st == PLO_OK && b < scene->max_bounces; ++b) {
            if (scene->emitter == PLO_PT_OCTREE)
                st = plo_render_rays(lum, a.ray, a.n, params, rgbA, TA, nullptr, stream);
            else
                k_pt_box_query<<<blocks, 256, 0, s>>>(a, a.ray, rgbA, TA);
            if (st != PLO_OK) break;
            k_pt_wall<<<blocks, 256, 0, s>>>(a, b);
            if (scene->emitter == PLO_PT_OCTREE)
                st = plo_render_rays(lum, a.nee_ray, a.n, params, rgbB, TB, nullptr, stream);
            else
                k_pt_box_query<<<blocks, 256, 0, s>>>(a, a.nee_ray, rgbB, TB);
            if (st != PLO_OK) break;
            k_pt_nee<<<blocks, 256, 0, s>>>(a);
        }
        if (st == PLO_OK) k_pt_store<<<blocks, 256, 0, s>>>(a, samples);
    }
    if (st == PLO_OK) k_pt_resolve<<<(unsigned)((pixels + 255) / 256), 256, 0, s>>>(samples, pixels, spp, d_image);
    e = cudaGetLastError();
    cudaFreeAsync(ws, s);
    if (own_samples) cudaFreeAsync(own_samples, s);
    if (st != PLO_OK) return st;
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "path tracer launch");
}
