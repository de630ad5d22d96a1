// Error reporting, version, and the host-buffer render entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>

#include "plo_internal.h"

namespace plo {

namespace {
thread_local std::string g_last_error;
}

plo_status set_error(plo_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

namespace {
std::atomic<int> g_fail_after{-1};
}

namespace {
// true when the failure hook makes this allocation fail
bool hook_fails() {
    int n = g_fail_after.load();
    while (n >= 0) {
        if (g_fail_after.compare_exchange_weak(n, n - 1)) return n == 0;
    }
    return false;
}
}  // namespace

int dev_malloc(void** p, size_t bytes) {
    if (hook_fails()) {
        *p = nullptr;
        return (int)cudaErrorMemoryAllocation;
    }
    return (int)cudaMalloc(p, bytes);
}

int dev_malloc_async(void** p, size_t bytes, cudaStream_t s) {
    if (hook_fails()) {
        *p = nullptr;
        return (int)cudaErrorMemoryAllocation;
    }
    return (int)cudaMallocAsync(p, bytes, s);
}

plo_status cuda_error(int err, const char* what) {
    cudaError_t e = static_cast<cudaError_t>(err);
    return set_error(e == cudaErrorMemoryAllocation ? PLO_ERR_OOM : PLO_ERR_CUDA,
                     std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

}  // namespace plo

using namespace plo;

extern "C" const char* plo_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* plo_version(void) { return "plo 0.1.0 (sm_103a)"; }

extern "C" void plo_debug_fail_alloc_after(int32_t n) { g_fail_after.store(n < 0 ? -1 : n); }

// Host-buffer render: chunks of rays alternate between two internal streams,
// so the host->device copy of one chunk overlaps the render and the
// device->host copy of the previous one.  A quarter of the rays per chunk,
// within [2^20, 2^22]: fewer, larger chunks keep the per-launch tails few,
// while four of them still hide most of the copies (measured on 16M rays:
// 2^20 rays per chunk 238, 2^21 264, 2^22 276, 2^23 263 Mrays/s).
extern "C" plo_status plo_render_rays_host(const plo_tree* tree, const float* h_rays, int64_t n,
                                           const plo_render_params* params, float* h_rgb, float* h_T,
                                           void* stream) {
    if (!tree) return set_error(PLO_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0) return set_error(PLO_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return PLO_OK;
    if (!h_rays || !h_rgb || !h_T) return set_error(PLO_ERR_INVALID_ARG, "rays, rgb or T is NULL");
    const int64_t chunk =
        std::min<int64_t>(n, std::max<int64_t>((int64_t)1 << 20, std::min<int64_t>((int64_t)1 << 22, (n + 3) / 4)));
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t s[2] = {nullptr, nullptr};
    cudaEvent_t ready = nullptr;
    float* buf[2] = {nullptr, nullptr};
    plo_status st = PLO_OK;
    cudaError_t e = cudaSuccess;
    const size_t per = (size_t)chunk * (6 + 3 + 1) * sizeof(float);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&s[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ready, user);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(s[k], ready, 0);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = (cudaError_t)dev_malloc_async((void**)&buf[k], per, s[k]);
    if (e != cudaSuccess) st = cuda_error(e, "plo_render_rays_host setup");
    for (int64_t off = 0, c = 0; st == PLO_OK && off < n; off += chunk, ++c) {
        const int64_t m = std::min(chunk, n - off);
        cudaStream_t cs = s[c & 1];
        float* d_rays = buf[c & 1];
        float* d_rgb = d_rays + 6 * chunk;
        float* d_T = d_rgb + 3 * chunk;
        e = cudaMemcpyAsync(d_rays, h_rays + 6 * off, (size_t)m * 6 * sizeof(float), cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) { st = cuda_error(e, "host-to-device ray copy"); break; }
        st = plo_render_rays(tree, d_rays, m, params, d_rgb, d_T, nullptr, cs);
        if (st != PLO_OK) break;
        e = cudaMemcpyAsync(h_rgb + 3 * off, d_rgb, (size_t)m * 3 * sizeof(float), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_T + off, d_T, (size_t)m * sizeof(float), cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) { st = cuda_error(e, "device-to-host result copy"); break; }
    }
    for (int k = 0; k < 2; ++k) {
        if (buf[k]) cudaFreeAsync(buf[k], s[k]);
        if (s[k]) {
            cudaError_t se = cudaStreamSynchronize(s[k]);
            if (se != cudaSuccess && st == PLO_OK) st = cuda_error(se, "plo_render_rays_host");
            cudaStreamDestroy(s[k]);
        }
    }
    if (ready) cudaEventDestroy(ready);
    return st;
}
