// Learned part (paper Sec. 4.2-4.4): the NeRF-SH network trained by the
// library's own kernels on rays rendered from a ground-truth octree.
//
//   sampling + positional encoding  k_pe        (Sec. 4.1 ray marching, Sec. 4.2 PE)
//   8 x 256 ReLU layers + SH head   k_gemm      (tcgen05, gemm.cuh)
//   quadrature, loss, d loss/d raw  k_quad      (Eq. 3-6, Eq. 7-9)
//   weight and bias gradients       k_wgrad (bias: an extra MMA against ones)
//   data gradients through ReLU     k_gemm (mask epilogue; the forward keeps the masks as bits)
//   Adam + exponential lr decay     k_adam      (Sec. 4.4)
//
// Activations are bf16 [samples][features] row-major; weights are kept as
// FP32 masters plus bf16 copies W [out][in] (forward B operand) and W^T
// [in][out] (data-gradient B operand), zero-padded to the GEMM tile shapes:
// layer 1 input 63 -> 64 columns, head output 1 + 3K -> 64 rows.
//
// Two output architectures (Sec. 4.2):
//   PLO_ARCH_LINEAR_HEAD  trunk -> linear 256 -> 1 + 3K (sigma, SH);
//   PLO_ARCH_PAPER        trunk -> [ReLU(W_f h + b_f) (128) | sigma (1)] as
//                         one 192-row layer with a split epilogue, then the
//                         128 -> 3K SH layer whose output row 0 is a zero row
//                         that carries sigma, so both architectures leave
//                         raw[:, 0] = sigma_raw, raw[:, 1 + ch K + k] = SH.
// The coarse/fine step (Sec. 4.3-4.4) runs a coarse network on stratified
// samples, places fine samples by its weights (k_fine) and trains a fine
// network on the union.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gemm.cuh"
#include "trunk.cuh"
#include "plo_internal.h"
#include "sh.cuh"

using namespace plo;

namespace plo {
namespace {

constexpr int WIDTH = 256;
constexpr int DEPTH = 8;
constexpr int N_FREQ = 10;
constexpr int PE_DIM = 3 + 6 * N_FREQ;  // 63
constexpr int PE_PAD = 64;
constexpr int OUT_PAD = 64;
constexpr int N_LAYERS = DEPTH + 1;      // linear-head architecture
constexpr int MAX_LAYERS = DEPTH + 2;    // paper architecture: + combined layer, + SH layer
constexpr int FEAT = 128;                // width of the layer before the SH outputs (Sec. 4.2)
constexpr int COMB_PAD = 192;            // combined layer rows: 128 features, sigma, zero padding

// ---------------------------------------------------------------- TMA maps
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

// bf16 matrix [rows][cols] (cols contiguous) read in boxes of 64 columns x
// box_rows rows with the 128-byte swizzle.
plo_status make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    EncodeFn fn = encoder();
    if (!fn) return set_error(PLO_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PLO_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
    return PLO_OK;
}

// bf16 matrix [rows][cols] written by TMA stores in boxes of 32 columns x 32
// rows, unswizzled (the epilogue stages each box row-major in shared memory).
plo_status make_store_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols) {
    EncodeFn fn = encoder();
    if (!fn) return set_error(PLO_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PLO_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
    return PLO_OK;
}

int sm_count_of_current() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------- GEMM launchers
// O: tensor map of the bf16 output (boxes of 32 x 32) for TMA stores, or
// NULL for direct stores from the epilogue threads.
template <int N, int K>
cudaError_t launch_gemm(const CUtensorMap& A, const CUtensorMap& B, const CUtensorMap* O, gemm::EpiArgs ep, int epi,
                        int M, int sms, cudaStream_t s) {
    ep.tma_out = O ? 1 : 0;
    const size_t smem = gemm::gemm_smem_bytes(N, K);
    cudaError_t e = cudaFuncSetAttribute(gemm::k_gemm<N, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int tiles = (M + gemm::BM - 1) / gemm::BM;
    int grid = tiles < sms ? tiles : sms;
    if (grid < 1) return cudaSuccess;
    gemm::k_gemm<N, K><<<grid, gemm::GEMM_THREADS, smem, s>>>(A, B, O ? *O : A, ep, epi, M);
    return cudaGetLastError();
}

template <int NIN>
cudaError_t launch_wgrad(const CUtensorMap& dZ, const CUtensorMap& H, float* dW, int n_out, int M, int sms,
                         unsigned int* err, cudaStream_t s, float* db = nullptr) {
    const size_t smem = gemm::wgrad_smem_bytes<NIN>();
    cudaError_t e = cudaFuncSetAttribute(gemm::k_wgrad<NIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int out_tiles = (n_out + gemm::BM - 1) / gemm::BM;
    int n_chunks = (2 * sms) / out_tiles;
    const int blocks64 = M / 64;
    if (n_chunks > blocks64) n_chunks = blocks64;
    if (n_chunks < 1) n_chunks = 1;
    const int chunk = ((blocks64 + n_chunks - 1) / n_chunks) * 64;
    n_chunks = (M + chunk - 1) / chunk;
    dim3 grid(out_tiles, n_chunks);
    gemm::k_wgrad<NIN><<<grid, gemm::THREADS, smem, s>>>(dZ, H, dW, n_out, M, chunk, err, db);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- small kernels
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// Stratification jitter in [0,1): SplitMix64 (Steele, Lea, Flood 2014)
// finaliser applied to a key of (seed, step, ray, sample).
__device__ __forceinline__ float jitter_u(uint64_t seed, uint64_t step, uint64_t ray, uint64_t j) {
    uint64_t k = mix64(seed ^ mix64(step + 0x51ED2701ULL));
    k = mix64(k ^ (ray * 0x9E3779B97F4A7C15ULL + j));
    return (float)(k >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ void unit_cube_clip(const float* o, const float* d, float& t0, float& t1, bool& hit) {
    float tn = -INFINITY, tf = INFINITY;
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            miss |= o[a] < 0.0f || o[a] > 1.0f;
            continue;
        }
        float inv = 1.0f / d[a];
        float ta = (0.0f - o[a]) * inv, tb = (1.0f - o[a]) * inv;
        tn = fmaxf(tn, fminf(ta, tb));
        tf = fminf(tf, fmaxf(ta, tb));
    }
    hit = !miss && tn < tf && tf > 0.0f;
    t0 = hit ? fmaxf(tn, 0.0f) : 0.0f;
    t1 = hit ? tf : 0.0f;
}

// Stratified samples t_j = t0 + (j + u_j)(t1 - t0)/N along each ray, segment
// lengths delta_j = t_{j+1} - t_j (the last ends at t1), and the positional
// encoding of x_j = o + t_j d -> X[ray*N + j][0..63] (column 63 is zero).
__global__ void k_pe(const float* rays, int n_rays, int N, const float* jitter, uint64_t seed, uint64_t step,
                     __nv_bfloat16* X, float* delta, float* t_out) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_rays * N) return;
    const int r = (int)(idx / N), j = (int)(idx % N);
    float o[3], d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = __ldg(rays + 6 * (int64_t)r + a);
        d[a] = __ldg(rays + 6 * (int64_t)r + 3 + a);
    }
    float t0, t1;
    bool hit;
    unit_cube_clip(o, d, t0, t1, hit);
    const float span = t1 - t0;
    const float u = jitter ? __ldg(jitter + idx) : jitter_u(seed, step, r, j);
    const float t = t0 + ((float)j + u) * span / (float)N;
    float tn = t1;
    if (j + 1 < N) {
        const float un = jitter ? __ldg(jitter + idx + 1) : jitter_u(seed, step, r, j + 1);
        tn = t0 + ((float)(j + 1) + un) * span / (float)N;
    }
    delta[idx] = hit ? tn - t : 0.0f;
    if (t_out) t_out[idx] = t;
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = fminf(fmaxf(o[a] + t * d[a], 0.0f), 1.0f);
    __nv_bfloat16* row = X + idx * PE_PAD;
    float f[PE_PAD];
    f[0] = x[0];
    f[1] = x[1];
    f[2] = x[2];
#pragma unroll
    for (int k = 0; k < N_FREQ; ++k) {
        const float sc = (float)(1 << k);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float sv, cv;
            sincospif(sc * x[a], &sv, &cv);
            f[3 + 6 * k + a] = sv;
            f[6 + 6 * k + a] = cv;
        }
    }
    f[63] = 0.0f;
    uint4* dst = reinterpret_cast<uint4*>(row);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int u2 = 0; u2 < 4; ++u2) {
            __nv_bfloat162 h = __floats2bfloat162_rn(f[8 * q + 2 * u2], f[8 * q + 2 * u2 + 1]);
            w[u2] = *reinterpret_cast<uint32_t*>(&h);
        }
        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Positional encoding of one point (unit-cube coordinates) into a bf16 row.
__device__ __forceinline__ void encode_point(const float* x, __nv_bfloat16* row) {
    float f[PE_PAD];
    f[0] = x[0];
    f[1] = x[1];
    f[2] = x[2];
#pragma unroll
    for (int k = 0; k < N_FREQ; ++k) {
        const float sc = (float)(1 << k);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float sv, cv;
            sincospif(sc * x[a], &sv, &cv);
            f[3 + 6 * k + a] = sv;
            f[6 + 6 * k + a] = cv;
        }
    }
    f[63] = 0.0f;
    uint4* dst = reinterpret_cast<uint4*>(row);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int u2 = 0; u2 < 4; ++u2) {
            __nv_bfloat162 h = __floats2bfloat162_rn(f[8 * q + 2 * u2], f[8 * q + 2 * u2 + 1]);
            w[u2] = *reinterpret_cast<uint32_t*>(&h);
        }
        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Positional encoding of given points (unit-cube coordinates) -> X.
__global__ void k_pe_points(const float* pts, int64_t n, __nv_bfloat16* X) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = __ldg(pts + 3 * idx + a);
    encode_point(x, X + idx * PE_PAD);
}

// ---- distillation (Sec. 5, "Creating the plenoctree") ----
// Voxels at depth D are addressed by their Morton code: the child slot
// (bx | by << 1 | bz << 2) of every level from the root, most significant
// first.
__device__ __forceinline__ void morton_decode(uint64_t m, int D, uint32_t* c) {
    c[0] = c[1] = c[2] = 0;
    for (int l = 0; l < D; ++l) {
        const uint32_t slot = (uint32_t)(m >> (3 * (D - 1 - l))) & 7u;
        c[0] = 2u * c[0] + (slot & 1u);
        c[1] = 2u * c[1] + ((slot >> 1) & 1u);
        c[2] = 2u * c[2] + (slot >> 2);
    }
}

// Centre of voxels base .. base+n-1 (Morton order) -> X.
__global__ void k_pe_centres(uint64_t base, int64_t n, int D, __nv_bfloat16* X) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    uint32_t c[3];
    morton_decode(base + (uint64_t)idx, D, c);
    const float inv_g = 1.0f / (float)(1u << D);
    float x[3] = {((float)c[0] + 0.5f) * inv_g, ((float)c[1] + 0.5f) * inv_g, ((float)c[2] + 0.5f) * inv_g};
    encode_point(x, X + idx * PE_PAD);
}

// S jittered samples in each listed voxel -> X (row i*S + s).  Offsets come
// from SplitMix64 (Steele, Lea, Flood 2014): key = mix(mix(seed ^ 0xD15711)
// ^ (code * 0x9E3779B97F4A7C15 + 3 s + a)), u = (key >> 40) / 2^24.
__global__ void k_pe_jitter(const uint32_t* codes, int64_t nv, int S, int D, uint64_t seed, __nv_bfloat16* X) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nv * S) return;
    const int64_t i = idx / S;
    const int s = (int)(idx % S);
    const uint64_t code = __ldg(codes + i);
    uint32_t c[3];
    morton_decode(code, D, c);
    const uint64_t k0 = mix64(seed ^ 0xD15711ULL);
    const uint64_t base = code * 0x9E3779B97F4A7C15ULL;
    const float inv_g = 1.0f / (float)(1u << D);
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const uint64_t key = mix64(k0 ^ (base + (uint64_t)(3 * s + a)));
        const float u = (float)(key >> 40) * (1.0f / 16777216.0f);
        x[a] = ((float)c[a] + u) * inv_g;
    }
    encode_point(x, X + idx * PE_PAD);
}

__global__ void k_keep(const float* raw, int64_t n, float thresh, uint32_t* flags) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    flags[idx] = fmaxf(__ldg(raw + idx * OUT_PAD), 0.0f) >= thresh ? 1u : 0u;
}

// Appends the kept voxels of a chunk (codes base + i, Morton order) at the
// running count *count; the last thread advances the count.
__global__ void k_compact_kept(uint64_t base, int64_t n, const uint32_t* flag, const uint32_t* pos, uint32_t* count,
                               uint32_t* codes) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c0 = *count;
    if (flag[i]) codes[c0 + pos[i]] = (uint32_t)(base + (uint64_t)i);
}
__global__ void k_advance_count(const uint32_t* flag, const uint32_t* pos, int64_t n, uint32_t* count) {
    *count += pos[n - 1] + flag[n - 1];
}

// sigma >= 0 as a 24-bit float (the 16-bit trees' density word): FP32
// without its sign, mantissa rounded to nearest even at 16 bits, kept finite.
__device__ __forceinline__ uint32_t sigma24(float v) {
    const uint32_t b = __float_as_uint(v) & 0x7FFFFFFFu;
    uint32_t r = (b + 0x3Fu + ((b >> 7) & 1u)) >> 7;
    return r >= 0xFF0000u ? 0xFEFFFFu : r;
}

// One distilled leaf per thread: the mean over its S jittered samples of
// ReLU(sigma_raw) and of each raw SH coefficient, packed as plo_build_tree
// packs a leaf: the record (FP32 coefficients, or 16-bit ones times a
// power-of-two scale 2^e that puts the largest |coefficient| in [2^14, 2^15)
// for FP16 and in [0.5, 1) for BF16) and the entry word.
template <int PREC>
__global__ void k_pack_leaves(const float* raw, int64_t nv, int S, int K, int stride, uint32_t* yword, uint8_t* emits,
                              uint8_t* records) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    float sig = 0.0f;
    for (int s = 0; s < S; ++s) sig += fmaxf(__ldg(raw + (i * S + s) * OUT_PAD), 0.0f);
    sig /= (float)S;
    const int nc = 3 * K;
    uint8_t* rec = records + (size_t)i * stride;
    // the means (written at once for FP32 records; for 16-bit ones this pass
    // finds the largest |mean| and the next recomputes the same values)
    float m = 0.0f;
    bool any = false;
    for (int k = 0; k < nc; ++k) {
        float acc = 0.0f;
        for (int s = 0; s < S; ++s) acc += __ldg(raw + (i * S + s) * OUT_PAD + 1 + k);
        const float c = acc / (float)S;
        any |= c != 0.0f;
        m = fmaxf(m, fabsf(c));
        if (PREC == PLO_PREC_FP32) reinterpret_cast<float*>(rec)[k] = c;
    }
    emits[i] = any ? 1 : 0;
    if (PREC == PLO_PREC_FP32) {
        for (int b = 4 * nc; b < stride; ++b) rec[b] = 0;
        yword[i] = __float_as_uint(sig);
        return;
    }
    int e;
    frexpf(m, &e);
    if (PREC == PLO_PREC_FP16) e -= 15;
    e = max(-126, min(127, e));
    const float inv = ldexpf(1.0f, -e);
    uint16_t* h = reinterpret_cast<uint16_t*>(rec);
    for (int k = 0; k < nc; ++k) {
        float acc = 0.0f;
        for (int s = 0; s < S; ++s) acc += __ldg(raw + (i * S + s) * OUT_PAD + 1 + k);
        const float v = (acc / (float)S) * inv;
        h[k] = PREC == PLO_PREC_FP16 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    for (int b = 2 * nc; b < stride; ++b) rec[b] = 0;
    yword[i] = sigma24(sig) | (any ? (uint32_t)(e + 127) << 24 : 0u);
}

// Quadrature render of Eq. 3 from the head outputs, the loss of Eq. 7-9 and
// its gradient w.r.t. the head outputs.  One warp per ray; lane l owns the
// samples [l*S, (l+1)*S).  raw: fp32 [ray*N + j][64] (0: sigma, 1 + ch*K + k:
// SH); dO: bf16, same layout; ray_loss [n_rays].
template <int K, int S>
__global__ void k_quad(const float* raw, const float* delta, const float* rays, const float* rgb_gt,
                       const float* alpha_gt, int n_rays, float l_max, float eps, int transmittance, int loss_kind,
                       float inv_rays, __nv_bfloat16* dO, float* ray_loss, __nv_bfloat16* dsig_out, int dsig_ld,
                       float* w_out, float* ray_out) {
    const int r = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n_rays) return;
    constexpr int N = 32 * S;
    float dn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) dn[a] = __ldg(rays + 6 * (int64_t)r + 3 + a);
    const float inv_len = rsqrtf(dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2]);
    float Y[K];
    sh_basis<K>(dn[0] * inv_len, dn[1] * inv_len, dn[2] * inv_len, Y);

    float sig[S][3], c[S][3], a[S], dl[S];
    bool pos[S];
    float local = 0.0f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t row = (int64_t)r * N + lane * S + s;
        const float* q = raw + row * OUT_PAD;
        const float sr = __ldg(q);
        pos[s] = sr > 0.0f;
        dl[s] = __ldg(delta + row);
        a[s] = fmaxf(sr, 0.0f) * dl[s];
        local += a[s];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = __fmaf_rn(__ldg(q + 1 + ch * K + k), Y[k], acc);
            const float sg = 1.0f / (1.0f + expf(-acc));
            sig[s][ch] = sg;
            c[s][ch] = l_max * sg;
        }
    }
    // exclusive prefix of optical depth across lanes
    float incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        float v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    float cum = incl - local;
    float T[S + 1], w[S];
    const bool lin = transmittance != PLO_TRANS_EXP;
    T[0] = lin ? fmaxf(0.0f, 1.0f - cum) : expf(-cum);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        cum += a[s];
        T[s + 1] = lin ? fmaxf(0.0f, 1.0f - cum) : expf(-cum);
        // w = T_j - T_{j+1} in a form that does not cancel when sigma delta
        // is small: T_j (1 - e^{-a_j}) (exponential), min(T_j, a_j) (linear)
        w[s] = lin ? fminf(T[s], a[s]) : T[s] * -expm1f(-a[s]);
    }
    float C[3] = {0.0f, 0.0f, 0.0f}, alpha = 0.0f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        alpha += w[s];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) C[ch] = __fmaf_rn(w[s], c[s][ch], C[ch]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        alpha += __shfl_xor_sync(0xffffffffu, alpha, off);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) C[ch] += __shfl_xor_sync(0xffffffffu, C[ch], off);
    }
    // loss (values divided by l_max; the denominator is held constant)
    float dC[3], loss = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float cn = C[ch] / l_max, gn = __ldg(rgb_gt + 3 * (int64_t)r + ch) / l_max;
        const float den = loss_kind == 2 ? 1.0f : cn + eps;
        const float res = (cn - gn) / den;
        loss += res * res;
        dC[ch] = 2.0f * res / den / l_max * inv_rays;
    }
    float dA = 0.0f;
    if (loss_kind == 0) {
        const float da = alpha - __ldg(alpha_gt + r);
        loss += da * da;
        dA = 2.0f * da * inv_rays;
    }
    if (lane == 0) ray_loss[r] = loss;
    if (ray_out && lane == 0) {  // per-ray C^, alpha^ and loss (test hook)
        float* o = ray_out + 5 * (int64_t)r;
        o[0] = C[0];
        o[1] = C[1];
        o[2] = C[2];
        o[3] = alpha;
        o[4] = loss;
    }
    // d loss / d w_j, then d loss / d a_j
    float g[S], wg_local = 0.0f, actg_local = 0.0f, actnext_local = 0.0f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        g[s] = dA;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) g[s] = __fmaf_rn(c[s][ch], dC[ch], g[s]);
        wg_local += w[s] * g[s];
        actg_local += (T[s] > 0.0f ? g[s] : 0.0f);
        actnext_local += (T[s + 1] > 0.0f ? g[s] : 0.0f);
    }
    // suffix sums over later lanes (exclusive of this lane)
    float suf_wg = wg_local, suf_actg = actg_local, suf_actnext = actnext_local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        float v1 = __shfl_down_sync(0xffffffffu, suf_wg, off);
        float v2 = __shfl_down_sync(0xffffffffu, suf_actg, off);
        float v3 = __shfl_down_sync(0xffffffffu, suf_actnext, off);
        if (lane + off < 32) {
            suf_wg += v1;
            suf_actg += v2;
            suf_actnext += v3;
        }
    }
    float after_wg = suf_wg - wg_local;          // sum over later lanes
    float after_actg = suf_actg - actg_local;
    float after_actnext = suf_actnext - actnext_local;
    float da[S];
#pragma unroll
    for (int s = S - 1; s >= 0; --s) {
        if (!lin) {
            // da_j = T_{j+1} g_j - sum_{k>j} w_k g_k
            da[s] = T[s + 1] * g[s] - after_wg;
            after_wg += w[s] * g[s];
        } else {
            // da_j = sum_{k>=j} g_k [T_{k+1} > 0] - sum_{k>j} g_k [T_k > 0]
            after_actnext += (T[s + 1] > 0.0f ? g[s] : 0.0f);
            da[s] = after_actnext - after_actg;
            after_actg += (T[s] > 0.0f ? g[s] : 0.0f);
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t row = (int64_t)r * N + lane * S + s;
        float out[OUT_PAD];
#pragma unroll
        for (int k = 0; k < OUT_PAD; ++k) out[k] = 0.0f;
        const float dsig = pos[s] ? da[s] * dl[s] : 0.0f;
        out[0] = dsig_out ? 0.0f : dsig;
        if (dsig_out) dsig_out[row * dsig_ld] = __float2bfloat16_rn(dsig);
        if (w_out) w_out[row] = w[s];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float ds = w[s] * dC[ch] * l_max * sig[s][ch] * (1.0f - sig[s][ch]);
#pragma unroll
            for (int k = 0; k < K; ++k) out[1 + ch * K + k] = ds * Y[k];
        }
        uint4* dst = reinterpret_cast<uint4*>(dO + row * OUT_PAD);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                __nv_bfloat162 h = __floats2bfloat162_rn(out[8 * q + 2 * u], out[8 * q + 2 * u + 1]);
                wv[u] = *reinterpret_cast<uint32_t*>(&h);
            }
            dst[q] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
    }
}

// Fine samples of the coarse/fine scheme (Sec. 4.3-4.4) and the merged
// sample set; one warp per ray.  Coarse sample i owns [t_i, t_i + delta_i);
// the density is constant there with mass proportional to w_i + 1e-5, and
// stratified u_j = (j + xi_j) / Nf goes through the inverse CDF.  The merged
// set lists the coarse and fine parameters in ascending order (a coarse
// sample first at equal t): fine sample j of segment b has rank j + b + 1,
// coarse sample i has rank i + (fine samples in segments before i).  Then
// delta_k = t_{k+1} - t_k (the last ends at the exit of the unit cube) and X
// gets the encoding of o + t_k d in row ray * (Nc + Nf) + k.
constexpr int HIER_WARPS = 4;
constexpr int HIER_MAX_NC = 128;
constexpr int HIER_MAX_N = 256;
constexpr float FINE_FLOOR = 1e-5f;

__device__ __forceinline__ float fine_u(uint64_t seed, uint64_t step, uint64_t ray, uint64_t j) {
    return jitter_u(seed ^ 0xF17E5A3B1E000000ULL, step, ray, j);
}

__global__ void __launch_bounds__(32 * HIER_WARPS)
    k_fine(const float* rays, int n_rays, int Nc, int Nf, const float* t_c, const float* delta_c, const float* w_c,
           const float* xi, uint64_t seed, uint64_t step, __nv_bfloat16* X, float* delta_out, float* t_out) {
    __shared__ float sC[HIER_WARPS][HIER_MAX_NC + 1];
    __shared__ float sT[HIER_WARPS][HIER_MAX_NC];
    __shared__ float sD[HIER_WARPS][HIER_MAX_NC];
    __shared__ int sCnt[HIER_WARPS][HIER_MAX_NC];
    __shared__ float sM[HIER_WARPS][HIER_MAX_N];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * HIER_WARPS + wid;
    if (r >= n_rays) return;  // the whole warp leaves together
    const int N = Nc + Nf, PB = Nc / 32, QF = Nf / 32;
    float* C = sC[wid];
    float* T = sT[wid];
    float* D = sD[wid];
    int* cnt = sCnt[wid];
    float* Mg = sM[wid];
    const int64_t base = (int64_t)r * Nc;
    float local = 0.0f;
    for (int q = 0; q < PB; ++q) {
        const int i = lane * PB + q;
        T[i] = __ldg(t_c + base + i);
        D[i] = __ldg(delta_c + base + i);
        local += __ldg(w_c + base + i) + FINE_FLOOR;
        cnt[i] = 0;
    }
    float incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    float run = incl - local;
    for (int q = 0; q < PB; ++q) {
        const int i = lane * PB + q;
        C[i] = run;
        run += __ldg(w_c + base + i) + FINE_FLOOR;
    }
    if (lane == 31) C[Nc] = run;
    __syncwarp();
    const float total = C[Nc];
    float tf[HIER_MAX_N / 32];
    int bf[HIER_MAX_N / 32];
    for (int q = 0; q < QF; ++q) {
        const int j = lane * QF + q;
        const float x = xi ? __ldg(xi + (int64_t)r * Nf + j) : fine_u(seed, step, (uint64_t)r, (uint64_t)j);
        const float u = ((float)j + x) / (float)Nf * total;
        int lo = 0, hi = Nc - 1;  // the last segment i with C[i] <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (C[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        const float span = C[lo + 1] - C[lo];
        const float frac = span > 0.0f ? fminf(fmaxf((u - C[lo]) / span, 0.0f), 1.0f) : 0.0f;
        // inside the segment, also after rounding, so the ranks below give an
        // ascending list
        const float hi_t = lo + 1 < Nc ? T[lo + 1] : T[lo] + D[lo];
        tf[q] = fminf(fmaxf(T[lo] + frac * D[lo], T[lo]), hi_t);
        bf[q] = lo;
        atomicAdd(&cnt[lo], 1);
    }
    __syncwarp();
    // exclusive prefix of the per-segment counts
    int lc = 0;
    for (int q = 0; q < PB; ++q) lc += cnt[lane * PB + q];
    int ic = lc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, ic, off);
        if (lane >= off) ic += v;
    }
    int before = ic - lc;
    for (int q = 0; q < PB; ++q) {
        const int i = lane * PB + q;
        const int c = cnt[i];
        Mg[i + before] = T[i];
        before += c;
    }
    for (int q = 0; q < QF; ++q) Mg[lane * QF + q + bf[q] + 1] = tf[q];
    __syncwarp();
    float o[3], d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = __ldg(rays + 6 * (int64_t)r + a);
        d[a] = __ldg(rays + 6 * (int64_t)r + 3 + a);
    }
    float t0, t1;
    bool hit;
    unit_cube_clip(o, d, t0, t1, hit);
    for (int k = lane; k < N; k += 32) {
        const float t = Mg[k];
        const float tn = k + 1 < N ? Mg[k + 1] : t1;
        const int64_t row = (int64_t)r * N + k;
        delta_out[row] = hit ? tn - t : 0.0f;
        if (t_out) t_out[row] = t;
        if (X) {
            float x[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) x[a] = fminf(fmaxf(o[a] + t * d[a], 0.0f), 1.0f);
            encode_point(x, X + row * PE_PAD);
        }
    }
}

struct LayerGeom {
    int n_layers;
    int64_t off[MAX_LAYERS + 1];  // offset of layer l's W in the padded flat array; bias follows W
    int out_real[MAX_LAYERS], in_real[MAX_LAYERS], out_pad[MAX_LAYERS], in_pad[MAX_LAYERS];
    int out_first[MAX_LAYERS];    // first trained row (the paper SH layer's row 0 carries sigma)
};

__device__ __forceinline__ int find_layer(const LayerGeom& g, int64_t i) {
    int l = 0;
#pragma unroll
    for (int k = 1; k < MAX_LAYERS; ++k)
        if (k < g.n_layers && i >= g.off[k]) l = k;
    return l;
}

// Adam (Kingma & Ba) with bias correction on the FP32 masters, then the bf16
// copies W [out][in] and W^T [in][out].  Padding entries stay zero.
__global__ void k_adam(LayerGeom g, float* master, float* m, float* v, const float* grad, int64_t n, float lr,
                       float b1, float b2, float eps, float bc1, float bc2, int update, __nv_bfloat16* const* W,
                       __nv_bfloat16* const* WT) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = find_layer(g, i);
    const int64_t loc = i - g.off[l];
    const int64_t wsz = (int64_t)g.out_pad[l] * g.in_pad[l];
    const bool is_w = loc < wsz;
    const int o = is_w ? (int)(loc / g.in_pad[l]) : (int)(loc - wsz);
    const int in = is_w ? (int)(loc % g.in_pad[l]) : 0;
    const bool real = o >= g.out_first[l] && o < g.out_real[l] && (!is_w || in < g.in_real[l]);
    float p = master[i];
    if (update && real) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        master[i] = p;
    }
    if (!real) p = 0.0f;
    if (is_w) {
        const __nv_bfloat16 h = __float2bfloat16_rn(p);
        W[l][(int64_t)o * g.in_pad[l] + in] = h;
        if (WT[l]) WT[l][(int64_t)in * g.out_pad[l] + o] = h;
    }
}

__global__ void k_mean(const float* x, int n, float* out, const float* y = nullptr) {
    __shared__ float red[256];
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i] + (y ? y[i] : 0.0f);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / (float)n;
}

}  // namespace
}  // namespace plo

// ---------------------------------------------------------------- the handle
struct plo_mlp {
    plo_mlp_desc desc;
    int K, n_out;
    int arch, n_layers;
    int device, sms;
    LayerGeom geom;
    int64_t n_params_pad;
    float *master = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
    __nv_bfloat16* W[MAX_LAYERS] = {};
    __nv_bfloat16* WT[MAX_LAYERS] = {};
    __nv_bfloat16** d_W = nullptr;
    __nv_bfloat16** d_WT = nullptr;
    CUtensorMap mapW[MAX_LAYERS], mapWT[MAX_LAYERS];
    int64_t step = 0;
    unsigned int* d_err = nullptr;
    // workspace (samples capacity)
    int64_t cap = 0;
    int cap_rays = 0;
    __nv_bfloat16* H[MAX_LAYERS] = {};  // H[0] = X [cap][64], H[1..8] [cap][256], H[9] [cap][128] (paper)
    uint32_t* HB[MAX_LAYERS] = {};      // H[l] > 0 as bits, [cap][in_pad[l] / 32] words (l >= 1; training)
    float* raw = nullptr;               // [cap][64]
    float* sraw = nullptr;              // [cap][64] fp32 half of the paper combined layer (column 0: sigma)
    __nv_bfloat16* dO = nullptr;        // [cap][64]
    __nv_bfloat16* dZ[DEPTH] = {};      // [cap][256]: d loss / d Z_l (pre-activation of trunk layer l)
    __nv_bfloat16* dZc = nullptr;       // [cap][192] gradient of the paper combined layer's output
    float* delta = nullptr;
    float* tsamp = nullptr;             // [cap] sample parameters (coarse pass)
    float* wts = nullptr;               // [cap] quadrature weights (coarse pass)
    float* ray_loss = nullptr;
    CUtensorMap mapA_H[MAX_LAYERS], mapA_dO, mapA_dZ[DEPTH], mapA_dZc;  // A operand boxes (128 rows)
    CUtensorMap mapW_H[MAX_LAYERS], mapW_dO, mapW_dZ[DEPTH], mapW_dZc;  // wgrad boxes (64 rows)
    CUtensorMap mapO_H[MAX_LAYERS], mapO_dZ7, mapO_dZc;           // TMA-store boxes (32 x 32)
};

namespace {

void free_workspace(plo_mlp* m) {
    for (int l = 0; l < MAX_LAYERS; ++l) cudaFree(m->H[l]), m->H[l] = nullptr;
    for (int l = 0; l < MAX_LAYERS; ++l) cudaFree(m->HB[l]), m->HB[l] = nullptr;
    cudaFree(m->raw);
    cudaFree(m->sraw);
    cudaFree(m->dO);
    for (int l = 0; l < DEPTH; ++l) cudaFree(m->dZ[l]), m->dZ[l] = nullptr;
    cudaFree(m->dZc);
    cudaFree(m->delta);
    cudaFree(m->tsamp);
    cudaFree(m->wts);
    cudaFree(m->ray_loss);
    m->raw = m->sraw = m->delta = m->tsamp = m->wts = m->ray_loss = nullptr;
    m->dO = m->dZc = nullptr;
    m->cap = 0;
    m->cap_rays = 0;
}

plo_status ensure_workspace(plo_mlp* m, int64_t samples, int rays) {
    if (samples <= m->cap && rays <= m->cap_rays) return PLO_OK;
    cudaDeviceSynchronize();
    free_workspace(m);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = (cudaError_t)dev_malloc(p, bytes);
    };
    const bool paper = m->arch == PLO_ARCH_PAPER;
    alloc((void**)&m->H[0], (size_t)samples * PE_PAD * 2);
    for (int l = 1; l <= DEPTH; ++l) alloc((void**)&m->H[l], (size_t)samples * WIDTH * 2);
    if (paper) alloc((void**)&m->H[DEPTH + 1], (size_t)samples * FEAT * 2);
    for (int l = 1; l <= DEPTH; ++l) alloc((void**)&m->HB[l], (size_t)samples * (WIDTH / 32) * 4);
    if (paper) alloc((void**)&m->HB[DEPTH + 1], (size_t)samples * (FEAT / 32) * 4);
    alloc((void**)&m->raw, (size_t)samples * OUT_PAD * 4);
    if (paper) alloc((void**)&m->sraw, (size_t)samples * OUT_PAD * 4);
    alloc((void**)&m->dO, (size_t)samples * OUT_PAD * 2);
    for (int l = 0; l < DEPTH; ++l) alloc((void**)&m->dZ[l], (size_t)samples * WIDTH * 2);
    if (paper) alloc((void**)&m->dZc, (size_t)samples * COMB_PAD * 2);
    alloc((void**)&m->delta, (size_t)samples * 4);
    alloc((void**)&m->tsamp, (size_t)samples * 4);
    alloc((void**)&m->wts, (size_t)samples * 4);
    alloc((void**)&m->ray_loss, (size_t)(rays > 0 ? rays : 1) * 4);
    // columns of dZc that no kernel writes (sigma's padding) stay zero
    if (e == cudaSuccess && paper) e = cudaMemset(m->dZc, 0, (size_t)samples * COMB_PAD * 2);
    if (e != cudaSuccess) {
        free_workspace(m);
        cudaGetLastError();
        return set_error(PLO_ERR_OOM, "device allocation of the training workspace failed");
    }
    m->cap = samples;
    m->cap_rays = rays;
    plo_status st = PLO_OK;
    for (int l = 0; l < m->n_layers && st == PLO_OK; ++l) {
        const int cols = m->geom.in_pad[l];
        st = make_map(&m->mapA_H[l], m->H[l], samples, cols, 128);
        if (st == PLO_OK) st = make_map(&m->mapW_H[l], m->H[l], samples, cols, 64);
    }
    if (st == PLO_OK && paper) st = make_map(&m->mapA_dZc, m->dZc, samples, COMB_PAD, 128);
    if (st == PLO_OK && paper) st = make_map(&m->mapW_dZc, m->dZc, samples, COMB_PAD, 64);
    if (st == PLO_OK && paper) st = make_store_map(&m->mapO_dZc, m->dZc, samples, COMB_PAD);
    for (int l = 1; l < m->n_layers && st == PLO_OK; ++l)
        st = make_store_map(&m->mapO_H[l], m->H[l], samples, m->geom.in_pad[l]);
    if (st == PLO_OK) st = make_store_map(&m->mapO_dZ7, m->dZ[DEPTH - 1], samples, WIDTH);
    if (st == PLO_OK) st = make_map(&m->mapA_dO, m->dO, samples, OUT_PAD, 128);
    if (st == PLO_OK) st = make_map(&m->mapW_dO, m->dO, samples, OUT_PAD, 64);
    for (int k = 0; k < DEPTH && st == PLO_OK; ++k) {
        st = make_map(&m->mapA_dZ[k], m->dZ[k], samples, WIDTH, 128);
        if (st == PLO_OK) st = make_map(&m->mapW_dZ[k], m->dZ[k], samples, WIDTH, 64);
    }
    return st;
}

void init_geom(plo_mlp* m) {
    int64_t off = 0;
    LayerGeom& g = m->geom;
    g = LayerGeom{};
    g.n_layers = m->n_layers;
    for (int l = 0; l < m->n_layers; ++l) {
        g.in_real[l] = l == 0 ? PE_DIM : WIDTH;
        g.in_pad[l] = l == 0 ? PE_PAD : WIDTH;
        g.out_real[l] = WIDTH;
        g.out_pad[l] = WIDTH;
        g.out_first[l] = 0;
        if (l == DEPTH && m->arch == PLO_ARCH_LINEAR_HEAD) {
            g.out_real[l] = m->n_out;
            g.out_pad[l] = OUT_PAD;
        } else if (l == DEPTH) {  // paper: [features (128) | sigma | padding]
            g.out_real[l] = FEAT + 1;
            g.out_pad[l] = COMB_PAD;
        } else if (l == DEPTH + 1) {  // paper: SH layer, row 0 carries sigma
            g.in_real[l] = g.in_pad[l] = FEAT;
            g.out_real[l] = m->n_out;
            g.out_pad[l] = OUT_PAD;
            g.out_first[l] = 1;
        }
        g.off[l] = off;
        off += (int64_t)g.out_pad[l] * g.in_pad[l] + g.out_pad[l];
    }
    g.off[m->n_layers] = off;
    m->n_params_pad = off;
}

// The canonical flat parameter order (the oracle's): blocks of (W [rows][cols]
// then b [rows]); each block lands at `row0` of padded layer `layer`.
struct Block {
    int layer, row0, rows, cols;
    float init_scale;  // multiplier of the He-uniform bound
};
int canonical_blocks(int arch, int n_out, Block* b) {
    int n = 0;
    for (int l = 0; l < DEPTH; ++l) b[n++] = {l, 0, WIDTH, l == 0 ? PE_DIM : WIDTH, 1.0f};
    if (arch == PLO_ARCH_LINEAR_HEAD) {
        b[n++] = {DEPTH, 0, n_out, WIDTH, 0.1f};
    } else {
        b[n++] = {DEPTH, FEAT, 1, WIDTH, 0.1f};          // sigma
        b[n++] = {DEPTH, 0, FEAT, WIDTH, 1.0f};          // the 128-wide layer
        b[n++] = {DEPTH + 1, 1, n_out - 1, FEAT, 0.1f};  // SH coefficients
    }
    return n;
}

float* bias_ptr(plo_mlp* m, float* base, int l) {
    return base + m->geom.off[l] + (int64_t)m->geom.out_pad[l] * m->geom.in_pad[l];
}

plo_status refresh_bf16(plo_mlp* m, cudaStream_t s) {
    const int64_t n = m->n_params_pad;
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m->geom, m->master, m->adam_m, m->adam_v, m->grad, n, 0.0f,
                                                       0.9f, 0.999f, 1e-8f, 1.0f, 1.0f, 0, m->d_W, m->d_WT);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "weight cast kernel");
}

int64_t canonical_count(int arch, int n_out) {
    Block bl[MAX_LAYERS + 2];
    const int nb = canonical_blocks(arch, n_out, bl);
    int64_t c = 0;
    for (int k = 0; k < nb; ++k) c += (int64_t)bl[k].rows * bl[k].cols + bl[k].rows;
    return c;
}

void canonical_to_padded(const plo_mlp* m, const float* c, std::vector<float>& p) {
    p.assign(m->n_params_pad, 0.0f);
    Block bl[MAX_LAYERS + 2];
    const int nb = canonical_blocks(m->arch, m->n_out, bl);
    const LayerGeom& g = m->geom;
    int64_t ci = 0;
    for (int k = 0; k < nb; ++k) {
        const Block& B = bl[k];
        const int64_t w0 = g.off[B.layer], b0 = w0 + (int64_t)g.out_pad[B.layer] * g.in_pad[B.layer];
        for (int o = 0; o < B.rows; ++o)
            for (int i = 0; i < B.cols; ++i) p[w0 + (int64_t)(B.row0 + o) * g.in_pad[B.layer] + i] = c[ci++];
        for (int o = 0; o < B.rows; ++o) p[b0 + B.row0 + o] = c[ci++];
    }
}
void padded_to_canonical(const plo_mlp* m, const std::vector<float>& p, float* c) {
    Block bl[MAX_LAYERS + 2];
    const int nb = canonical_blocks(m->arch, m->n_out, bl);
    const LayerGeom& g = m->geom;
    int64_t ci = 0;
    for (int k = 0; k < nb; ++k) {
        const Block& B = bl[k];
        const int64_t w0 = g.off[B.layer], b0 = w0 + (int64_t)g.out_pad[B.layer] * g.in_pad[B.layer];
        for (int o = 0; o < B.rows; ++o)
            for (int i = 0; i < B.cols; ++i) c[ci++] = p[w0 + (int64_t)(B.row0 + o) * g.in_pad[B.layer] + i];
        for (int o = 0; o < B.rows; ++o) c[ci++] = p[b0 + B.row0 + o];
    }
}

// Forward of the MLP over H[0] (already encoded) for `samples` rows; the head
// writes fp32 raw outputs.  For training (`masks`), each ReLU layer also
// writes which of its outputs are positive as bits (HB), the backward pass's
// ReLU masks at 1/16 of the bytes of the activations.
// The trunk (layers 0..7) runs as one layer-fused kernel (k_trunk): each
// 128-row tile stays in shared memory from the encoding to H[8]; the layers'
// outputs H[1..8] are stored for the backward pass and the activation hook
// (`keep` false: only H[8], which the head reads).
template <bool BWD>
cudaError_t launch_trunk_kernel(const gemm::TrunkMaps& maps, const gemm::TrunkArgs& a, int sms, cudaStream_t s) {
    const size_t smem = gemm::trunk_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(gemm::k_trunk<BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = (a.M + gemm::BM - 1) / gemm::BM;
    const int grid = tiles < sms ? tiles : sms;
    if (grid < 1) return cudaSuccess;
    gemm::k_trunk<BWD><<<grid, gemm::TR_THREADS, smem, s>>>(maps, a);
    return cudaGetLastError();
}

cudaError_t launch_trunk(plo_mlp* m, int64_t samples, bool masks, bool keep, cudaStream_t s) {
    static_assert(gemm::TR_LAYERS == DEPTH && gemm::TR_N == WIDTH, "trunk shape");
    gemm::TrunkMaps maps;
    maps.x = m->mapA_H[0];
    gemm::TrunkArgs a{};
    for (int l = 0; l < DEPTH; ++l) {
        maps.w[l] = m->mapW[l];
        maps.h[l] = m->mapA_H[l + 1];
        a.bias[l] = bias_ptr(m, m->master, l);
        a.bits[l] = masks ? m->HB[l + 1] : nullptr;
    }
    a.store = keep ? 0xFFu : 0x80u;
    a.err = m->d_err;
    a.M = (int)samples;
    return launch_trunk_kernel<false>(maps, a, m->sms, s);
}

// The trunk's data-gradient chain (job j: layer l = 7 - j): dZ[l-1] =
// (dZ[l] W_l) masked by the forward's ReLU bits of H[l], from dZ[7].
cudaError_t launch_trunk_bwd(plo_mlp* m, int64_t samples, cudaStream_t s) {
    gemm::TrunkMaps maps;
    maps.x = m->mapA_dZ[DEPTH - 1];
    gemm::TrunkArgs a{};
    for (int j = 0; j < DEPTH - 1; ++j) {
        const int l = DEPTH - 1 - j;
        maps.w[j] = m->mapWT[l];
        maps.h[j] = m->mapA_dZ[l - 1];
        a.bits[j] = m->HB[l];
    }
    a.store = (1u << (DEPTH - 1)) - 1u;
    a.err = m->d_err;
    a.M = (int)samples;
    return launch_trunk_kernel<true>(maps, a, m->sms, s);
}

plo_status forward_layers(plo_mlp* m, int64_t samples, cudaStream_t s, bool masks = false, bool keep = true) {
    gemm::EpiArgs ep{};
    ep.err = m->d_err;
    cudaError_t e = launch_trunk(m, samples, masks, keep, s);
    ep.bits_out = nullptr;  // no ReLU after the head
    if (e == cudaSuccess && m->arch == PLO_ARCH_LINEAR_HEAD) {
        ep.bias = bias_ptr(m, m->master, DEPTH);
        ep.out_f32 = m->raw;
        ep.ldo = OUT_PAD;
        e = launch_gemm<OUT_PAD, WIDTH>(m->mapA_H[DEPTH], m->mapW[DEPTH], nullptr, ep, gemm::EPI_BIAS_F32, (int)samples, m->sms,
                                        s);
    } else if (e == cudaSuccess) {
        // [ReLU features -> H[9] (bf16) | sigma block -> sraw (fp32)], then the
        // SH layer, whose zero row 0 picks up sigma from sraw
        ep.bias = bias_ptr(m, m->master, DEPTH);
        ep.out_bf16 = m->H[DEPTH + 1];
        ep.ldo = FEAT;
        ep.bits_out = masks ? m->HB[DEPTH + 1] : nullptr;
        ep.ldb = FEAT / 32;
        ep.split = FEAT;
        ep.out_f32 = m->sraw;
        ep.ldo2 = OUT_PAD;
        e = launch_gemm<COMB_PAD, WIDTH>(m->mapA_H[DEPTH], m->mapW[DEPTH], &m->mapO_H[DEPTH + 1], ep, gemm::EPI_SPLIT, (int)samples, m->sms,
                                         s);
        gemm::EpiArgs eh{};
        eh.err = m->d_err;
        eh.bias = bias_ptr(m, m->master, DEPTH + 1);
        eh.out_f32 = m->raw;
        eh.ldo = OUT_PAD;
        eh.col0_add = m->sraw;
        eh.ld_col0 = OUT_PAD;
        if (e == cudaSuccess)
            e = launch_gemm<OUT_PAD, FEAT>(m->mapA_H[DEPTH + 1], m->mapW[DEPTH + 1], nullptr, eh, gemm::EPI_BIAS_F32,
                                           (int)samples, m->sms, s);
    }
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "MLP forward GEMM launch");
}

// k_quad for N samples per ray (one warp per ray, N / 32 samples per lane).
// The paper architecture takes d loss / d sigma_raw in column 128 of dZc.
cudaError_t launch_quad(plo_mlp* m, int N, const float* d_rays, const float* d_rgb_gt, const float* d_alpha_gt,
                        int n_rays, int loss_kind, float* w_out, cudaStream_t s, float* ray_out = nullptr) {
    const plo_mlp_desc& D = m->desc;
    const float inv_rays = 1.0f / (float)n_rays;
    const unsigned qblocks = (unsigned)((n_rays + 3) / 4);
    __nv_bfloat16* dsig = m->arch == PLO_ARCH_PAPER ? m->dZc + FEAT : nullptr;
#define PLO_QUAD(SS)                                                                                               \
    k_quad<16, SS><<<qblocks, 128, 0, s>>>(m->raw, m->delta, d_rays, d_rgb_gt, d_alpha_gt, n_rays, D.l_max, D.eps, \
                                           D.transmittance, loss_kind, inv_rays, m->dO, m->ray_loss, dsig, COMB_PAD, \
                                           w_out, ray_out)
    switch (N) {
        case 32: PLO_QUAD(1); break;
        case 64: PLO_QUAD(2); break;
        case 96: PLO_QUAD(3); break;
        case 128: PLO_QUAD(4); break;
        case 192: PLO_QUAD(6); break;
        case 256: PLO_QUAD(8); break;
        default: return cudaErrorInvalidValue;
    }
#undef PLO_QUAD
    return cudaGetLastError();
}

// Backward from dO (d loss / d raw, and for the paper architecture d loss /
// d sigma_raw in dZc) through every layer, then one Adam step with the
// exponentially decaying learning rate.
plo_status backward_update(plo_mlp* m, int64_t M, cudaStream_t s) {
    const plo_mlp_desc& D = m->desc;
    gemm::EpiArgs ep{};
    ep.err = m->d_err;
    cudaError_t e;
    if (m->arch == PLO_ARCH_LINEAR_HEAD) {
        e = launch_wgrad<WIDTH>(m->mapW_dO, m->mapW_H[DEPTH], m->grad + m->geom.off[DEPTH], OUT_PAD, (int)M, m->sms,
                                m->d_err, s, bias_ptr(m, m->grad, DEPTH));
        ep.out_bf16 = m->dZ[DEPTH - 1];
        ep.ldo = WIDTH;
        ep.bits = m->HB[DEPTH];
        ep.ldb = WIDTH / 32;
        if (e == cudaSuccess)
            e = launch_gemm<WIDTH, OUT_PAD>(m->mapA_dO, m->mapWT[DEPTH], &m->mapO_dZ7, ep, gemm::EPI_MASKBITS_BF16, (int)M, m->sms, s);
    } else {
        const int SH = DEPTH + 1;
        // SH layer: dW = dO^T feat, db = column sums; d feat -> dZc[:, 0:128]
        e = launch_wgrad<FEAT>(m->mapW_dO, m->mapW_H[SH], m->grad + m->geom.off[SH], OUT_PAD, (int)M, m->sms,
                               m->d_err, s, bias_ptr(m, m->grad, SH));
        ep.out_bf16 = m->dZc;
        ep.ldo = COMB_PAD;
        ep.bits = m->HB[SH];
        ep.ldb = FEAT / 32;
        if (e == cudaSuccess)
            e = launch_gemm<FEAT, OUT_PAD>(m->mapA_dO, m->mapWT[SH], &m->mapO_dZc, ep, gemm::EPI_MASKBITS_BF16, (int)M, m->sms, s);
        // combined layer [features | sigma]: dW = dZc^T h8; d h8 -> dZ[7]
        if (e == cudaSuccess)
            e = launch_wgrad<WIDTH>(m->mapW_dZc, m->mapW_H[DEPTH], m->grad + m->geom.off[DEPTH], COMB_PAD, (int)M,
                                    m->sms, m->d_err, s, bias_ptr(m, m->grad, DEPTH));
        ep.out_bf16 = m->dZ[DEPTH - 1];
        ep.ldo = WIDTH;
        ep.bits = m->HB[DEPTH];
        ep.ldb = WIDTH / 32;
        if (e == cudaSuccess)
            e = launch_gemm<WIDTH, COMB_PAD>(m->mapA_dZc, m->mapWT[DEPTH], &m->mapO_dZ7, ep, gemm::EPI_MASKBITS_BF16, (int)M, m->sms, s);
    }
    // the trunk: the data gradients dZ[6] .. dZ[0] in one layer-fused chain
    // from dZ[7], then every layer's weight gradient (each launch also sums
    // the layer's bias gradient), reading dZ[l] and the layer's input H[l]
    if (e == cudaSuccess) e = launch_trunk_bwd(m, M, s);
    for (int l = DEPTH - 1; l >= 0 && e == cudaSuccess; --l) {
        if (l == 0)
            e = launch_wgrad<PE_PAD>(m->mapW_dZ[0], m->mapW_H[0], m->grad + m->geom.off[0], WIDTH, (int)M, m->sms,
                                     m->d_err, s, bias_ptr(m, m->grad, 0));
        else
            e = launch_wgrad<WIDTH>(m->mapW_dZ[l], m->mapW_H[l], m->grad + m->geom.off[l], WIDTH, (int)M, m->sms,
                                    m->d_err, s, bias_ptr(m, m->grad, l));
    }
    if (e != cudaSuccess) return cuda_error(e, "MLP backward launch");
    // Adam with exponential decay lr0 -> lr1 over total_steps
    const double frac = std::fmin((double)(m->step - 1), (double)D.total_steps) / (double)D.total_steps;
    const float lr = (float)(D.lr0 * std::pow((double)D.lr1 / D.lr0, frac));
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)m->step));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)m->step));
    const int64_t n = m->n_params_pad;
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m->geom, m->master, m->adam_m, m->adam_v, m->grad, n, lr, 0.9f,
                                                       0.999f, 1e-8f, bc1, bc2, 1, m->d_W, m->d_WT);
    e = cudaGetLastError();
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "Adam launch");
}

plo_status check_mlp_desc(const plo_mlp_desc* d) {
    if (!d) return set_error(PLO_ERR_INVALID_ARG, "desc is NULL");
    if (d->sh_degree != 3) return set_error(PLO_ERR_UNSUPPORTED, "the network is built for SH degree 3 (48 coefficients)");
    if (d->transmittance < PLO_TRANS_EXP || d->transmittance > PLO_TRANS_LINEAR)
        return set_error(PLO_ERR_INVALID_ARG, "transmittance must be PLO_TRANS_EXP or PLO_TRANS_LINEAR");
    if (d->loss < PLO_LOSS_PAPER || d->loss > PLO_LOSS_MSE) return set_error(PLO_ERR_INVALID_ARG, "unknown loss");
    if (!(d->l_max > 0.0f) || !(d->lr0 > 0.0f) || !(d->lr1 > 0.0f) || d->total_steps < 1 || !(d->eps > 0.0f))
        return set_error(PLO_ERR_INVALID_ARG, "l_max, lr0, lr1, eps must be > 0 and total_steps >= 1");
    if (!(d->init_radiance >= 0.0f)) return set_error(PLO_ERR_INVALID_ARG, "init_radiance must be >= 0");
    if (d->arch != PLO_ARCH_LINEAR_HEAD && d->arch != PLO_ARCH_PAPER)
        return set_error(PLO_ERR_INVALID_ARG, "arch must be PLO_ARCH_LINEAR_HEAD or PLO_ARCH_PAPER");
    return PLO_OK;
}

}  // namespace

extern "C" int64_t plo_mlp_param_count(int32_t sh_degree) {
    return canonical_count(PLO_ARCH_LINEAR_HEAD, 1 + 3 * (sh_degree + 1) * (sh_degree + 1));
}

extern "C" int64_t plo_mlp_param_count_arch(int32_t sh_degree, int32_t arch) {
    if (arch != PLO_ARCH_LINEAR_HEAD && arch != PLO_ARCH_PAPER) return -1;
    return canonical_count(arch, 1 + 3 * (sh_degree + 1) * (sh_degree + 1));
}

extern "C" plo_status plo_mlp_create(const plo_mlp_desc* desc, uint64_t seed, plo_mlp** out) {
    if (!out) return set_error(PLO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    plo_status st = check_mlp_desc(desc);
    if (st != PLO_OK) return st;
    plo_mlp* m = new (std::nothrow) plo_mlp();
    if (!m) return set_error(PLO_ERR_OOM, "host allocation failed");
    m->desc = *desc;
    m->K = (desc->sh_degree + 1) * (desc->sh_degree + 1);
    m->n_out = 1 + 3 * m->K;
    m->arch = desc->arch;
    m->n_layers = m->arch == PLO_ARCH_PAPER ? MAX_LAYERS : N_LAYERS;
    cudaGetDevice(&m->device);
    m->sms = sm_count_of_current();
    init_geom(m);
    const size_t pbytes = (size_t)m->n_params_pad * 4;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = (cudaError_t)dev_malloc(p, bytes);
    };
    alloc((void**)&m->master, pbytes);
    alloc((void**)&m->adam_m, pbytes);
    alloc((void**)&m->adam_v, pbytes);
    alloc((void**)&m->grad, pbytes);
    alloc((void**)&m->d_err, 256);
    for (int l = 0; l < m->n_layers; ++l) {
        alloc((void**)&m->W[l], (size_t)m->geom.out_pad[l] * m->geom.in_pad[l] * 2);
        if (l >= 1) alloc((void**)&m->WT[l], (size_t)m->geom.out_pad[l] * m->geom.in_pad[l] * 2);
    }
    alloc((void**)&m->d_W, sizeof(void*) * MAX_LAYERS);
    alloc((void**)&m->d_WT, sizeof(void*) * MAX_LAYERS);
    if (e != cudaSuccess) {
        plo_mlp_free(m);
        cudaGetLastError();
        return set_error(PLO_ERR_OOM, "device allocation of the network failed");
    }
    cudaMemcpy(m->d_W, m->W, sizeof(void*) * MAX_LAYERS, cudaMemcpyHostToDevice);
    cudaMemcpy(m->d_WT, m->WT, sizeof(void*) * MAX_LAYERS, cudaMemcpyHostToDevice);
    cudaMemset(m->adam_m, 0, pbytes);
    cudaMemset(m->adam_v, 0, pbytes);
    cudaMemset(m->grad, 0, pbytes);
    cudaMemset(m->d_err, 0, 256);
    for (int l = 0; l < m->n_layers && st == PLO_OK; ++l) {
        st = make_map(&m->mapW[l], m->W[l], m->geom.out_pad[l], m->geom.in_pad[l], (uint32_t)m->geom.out_pad[l]);
        if (st == PLO_OK && l >= 1)
            st = make_map(&m->mapWT[l], m->WT[l], m->geom.in_pad[l], m->geom.out_pad[l], (uint32_t)m->geom.in_pad[l]);
    }
    if (st != PLO_OK) {
        plo_mlp_free(m);
        return st;
    }
    // He-uniform initial weights, zero biases; counter-based (SplitMix64).
    std::vector<float> canon(canonical_count(m->arch, m->n_out));
    int64_t ci = 0;
    uint64_t ctr = 0;
    auto unif = [&]() {
        uint64_t z = seed + 0x9E3779B97F4A7C15ULL * (++ctr);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    Block bl[MAX_LAYERS + 2];
    const int nb = canonical_blocks(m->arch, m->n_out, bl);
    std::vector<int64_t> bias_at(nb);
    for (int k = 0; k < nb; ++k) {
        const double lim = std::sqrt(6.0 / bl[k].cols) * bl[k].init_scale;
        for (int q = 0; q < bl[k].rows * bl[k].cols; ++q) canon[ci++] = (float)((2 * unif() - 1) * lim);
        bias_at[k] = ci;
        for (int q = 0; q < bl[k].rows; ++q) canon[ci++] = 0.0f;
    }
    // output biases: sigma starts positive, the DC coefficient sets the emission
    const double p0 = desc->init_radiance > 0.0f ? std::fmin(std::fmax(desc->init_radiance / desc->l_max, 1e-6), 0.5)
                                                 : 0.5;
    const double dc = std::log(p0 / (1.0 - p0)) / 0.28209479177387814;  // logit / Y_0^0
    if (m->arch == PLO_ARCH_LINEAR_HEAD) {
        float* head_b = canon.data() + bias_at[nb - 1];
        head_b[0] = 0.5f;
        for (int ch = 0; ch < 3; ++ch) head_b[1 + ch * m->K] = (float)dc;
    } else {
        canon[bias_at[nb - 3]] = 0.5f;  // sigma
        for (int ch = 0; ch < 3; ++ch) canon[bias_at[nb - 1] + ch * m->K] = (float)dc;
    }
    *out = m;
    st = plo_mlp_set_params(m, canon.data(), (int64_t)canon.size());
    if (st != PLO_OK) {
        plo_mlp_free(m);
        *out = nullptr;
    }
    return st;
}

extern "C" void plo_mlp_free(plo_mlp* m) {
    if (!m) return;
    cudaDeviceSynchronize();
    free_workspace(m);
    cudaFree(m->master);
    cudaFree(m->adam_m);
    cudaFree(m->adam_v);
    cudaFree(m->grad);
    cudaFree(m->d_err);
    for (int l = 0; l < MAX_LAYERS; ++l) {
        cudaFree(m->W[l]);
        cudaFree(m->WT[l]);
    }
    cudaFree(m->d_W);
    cudaFree(m->d_WT);
    delete m;
}

extern "C" plo_status plo_mlp_set_params(plo_mlp* m, const float* h_params, int64_t n) {
    if (!m || !h_params) return set_error(PLO_ERR_INVALID_ARG, "mlp or params is NULL");
    if (n != canonical_count(m->arch, m->n_out)) return set_error(PLO_ERR_INVALID_ARG, "wrong parameter count");
    std::vector<float> pad;
    try {
        canonical_to_padded(m, h_params, pad);
    } catch (const std::bad_alloc&) {
        return set_error(PLO_ERR_OOM, "host allocation for the parameters failed");
    }
    cudaError_t e = cudaMemcpy(m->master, pad.data(), pad.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "parameter upload");
    plo_status st = refresh_bf16(m, nullptr);
    if (st != PLO_OK) return st;
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "plo_mlp_set_params");
}

static plo_status download_canonical(const plo_mlp* m, const float* dev, float* h, int64_t n) {
    if (!m || !h) return set_error(PLO_ERR_INVALID_ARG, "mlp or output is NULL");
    if (n != canonical_count(m->arch, m->n_out)) return set_error(PLO_ERR_INVALID_ARG, "wrong parameter count");
    std::vector<float> pad;
    try {
        pad.resize(m->n_params_pad);
    } catch (const std::bad_alloc&) {
        return set_error(PLO_ERR_OOM, "host allocation for the parameters failed");
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(pad.data(), dev, pad.size() * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "parameter download");
    padded_to_canonical(m, pad, h);
    return PLO_OK;
}

extern "C" plo_status plo_mlp_get_params(const plo_mlp* m, float* h_params, int64_t n) {
    return download_canonical(m, m ? m->master : nullptr, h_params, n);
}
extern "C" plo_status plo_mlp_get_grads(const plo_mlp* m, float* h_grads, int64_t n) {
    return download_canonical(m, m ? m->grad : nullptr, h_grads, n);
}

extern "C" plo_status plo_mlp_forward(plo_mlp* m, const float* d_points, int64_t n, float* d_raw, void* stream) {
    if (!m) return set_error(PLO_ERR_INVALID_ARG, "mlp is NULL");
    if (n < 0) return set_error(PLO_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return PLO_OK;
    if (!d_points || !d_raw) return set_error(PLO_ERR_INVALID_ARG, "points or raw output is NULL");
    if (n > (int64_t)1 << 30) return set_error(PLO_ERR_INVALID_ARG, "n too large");
    cudaStream_t s = (cudaStream_t)stream;
    plo_status st = ensure_workspace(m, n, m->cap_rays);
    if (st != PLO_OK) return st;
    k_pe_points<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_points, n, m->H[0]);
    st = forward_layers(m, n, s);
    if (st != PLO_OK) return st;
    cudaError_t e = cudaMemcpy2DAsync(d_raw, (size_t)m->n_out * 4, m->raw, OUT_PAD * 4, (size_t)m->n_out * 4, (size_t)n,
                                      cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "raw output copy");
}

extern "C" plo_status plo_mlp_train_step(plo_mlp* m, const float* d_rays, const float* d_rgb_gt,
                                         const float* d_alpha_gt, int32_t n_rays, int32_t n_samples,
                                         const float* d_jitter, float* d_loss_out, void* stream) {
    if (!m) return set_error(PLO_ERR_INVALID_ARG, "mlp is NULL");
    if (!d_rays || !d_rgb_gt || !d_alpha_gt || !d_loss_out)
        return set_error(PLO_ERR_INVALID_ARG, "rays, targets or loss output is NULL");
    if (n_rays <= 0 || n_samples <= 0) return set_error(PLO_ERR_INVALID_ARG, "n_rays and n_samples must be > 0");
    if (n_samples != 32 && n_samples != 64 && n_samples != 128 && n_samples != 256)
        return set_error(PLO_ERR_UNSUPPORTED, "n_samples must be 32, 64, 128 or 256");
    const int64_t M = (int64_t)n_rays * n_samples;
    if (M % 128 != 0) return set_error(PLO_ERR_INVALID_ARG, "n_rays * n_samples must be a multiple of 128");
    if (M > ((int64_t)1 << 28)) return set_error(PLO_ERR_INVALID_ARG, "batch too large");
    cudaStream_t s = (cudaStream_t)stream;
    plo_status st = ensure_workspace(m, M, n_rays);
    if (st != PLO_OK) return st;
    const plo_mlp_desc& D = m->desc;
    ++m->step;
    cudaError_t e = cudaMemsetAsync(m->grad, 0, (size_t)m->n_params_pad * 4, s);
    if (e != cudaSuccess) return cuda_error(e, "gradient clear");
    k_pe<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(d_rays, n_rays, n_samples, d_jitter, D.seed, (uint64_t)m->step,
                                                     m->H[0], m->delta, nullptr);
    st = forward_layers(m, M, s, true);
    if (st != PLO_OK) return st;
    e = launch_quad(m, n_samples, d_rays, d_rgb_gt, d_alpha_gt, n_rays, D.loss, nullptr, s);
    if (e != cudaSuccess) return cuda_error(e, "quadrature kernel launch");
    st = backward_update(m, M, s);
    if (st != PLO_OK) return st;
    k_mean<<<1, 256, 0, s>>>(m->ray_loss, n_rays, d_loss_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "MLP update launch");
}

namespace {
bool hier_counts_ok(int Nc, int Nf) {
    const int N = Nc + Nf;
    return Nc % 32 == 0 && Nf % 32 == 0 && Nc >= 32 && Nf >= 32 && Nc <= HIER_MAX_NC &&
           (N == 64 || N == 96 || N == 128 || N == 192 || N == 256);
}
}  // namespace

extern "C" plo_status plo_mlp_train_step_hier(plo_mlp* coarse, plo_mlp* fine, const float* d_rays,
                                              const float* d_rgb_gt, const float* d_alpha_gt, int32_t n_rays,
                                              int32_t n_coarse, int32_t n_fine, const float* d_jitter,
                                              const float* d_xi, float* d_loss_out, void* stream) {
    if (!coarse || !fine || coarse == fine) return set_error(PLO_ERR_INVALID_ARG, "need two distinct networks");
    if (!d_rays || !d_rgb_gt || !d_alpha_gt || !d_loss_out)
        return set_error(PLO_ERR_INVALID_ARG, "rays, targets or loss output is NULL");
    if (n_rays <= 0) return set_error(PLO_ERR_INVALID_ARG, "n_rays must be > 0");
    if (!hier_counts_ok(n_coarse, n_fine))
        return set_error(PLO_ERR_UNSUPPORTED, "n_coarse, n_fine: multiples of 32, n_coarse <= 128, and "
                                              "n_coarse + n_fine in {64, 96, 128, 192, 256}");
    if (coarse->desc.l_max != fine->desc.l_max || coarse->desc.transmittance != fine->desc.transmittance ||
        coarse->desc.loss != fine->desc.loss)
        return set_error(PLO_ERR_INVALID_ARG, "coarse and fine networks need the same l_max, transmittance and loss");
    const int N = n_coarse + n_fine;
    const int64_t Mc = (int64_t)n_rays * n_coarse, Mf = (int64_t)n_rays * N;
    if (Mc % 128 != 0) return set_error(PLO_ERR_INVALID_ARG, "n_rays * n_coarse must be a multiple of 128");
    if (Mf > ((int64_t)1 << 28)) return set_error(PLO_ERR_INVALID_ARG, "batch too large");
    cudaStream_t s = (cudaStream_t)stream;
    plo_status st = ensure_workspace(coarse, Mc, n_rays);
    if (st == PLO_OK) st = ensure_workspace(fine, Mf, n_rays);
    if (st != PLO_OK) return st;
    ++coarse->step;
    ++fine->step;
    const plo_mlp_desc& D = fine->desc;
    // coarse pass: colour loss only (alpha is supervised on the fine pass)
    cudaError_t e = cudaMemsetAsync(coarse->grad, 0, (size_t)coarse->n_params_pad * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(fine->grad, 0, (size_t)fine->n_params_pad * 4, s);
    if (e != cudaSuccess) return cuda_error(e, "gradient clear");
    k_pe<<<(unsigned)((Mc + 255) / 256), 256, 0, s>>>(d_rays, n_rays, n_coarse, d_jitter, coarse->desc.seed,
                                                      (uint64_t)coarse->step, coarse->H[0], coarse->delta,
                                                      coarse->tsamp);
    st = forward_layers(coarse, Mc, s, true);
    if (st != PLO_OK) return st;
    const int coarse_loss = D.loss == PLO_LOSS_PAPER ? PLO_LOSS_REG : D.loss;
    e = launch_quad(coarse, n_coarse, d_rays, d_rgb_gt, d_alpha_gt, n_rays, coarse_loss, coarse->wts, s);
    if (e != cudaSuccess) return cuda_error(e, "quadrature kernel launch");
    // fine samples placed by the coarse weights (no gradient through them)
    k_fine<<<(unsigned)((n_rays + HIER_WARPS - 1) / HIER_WARPS), 32 * HIER_WARPS, 0, s>>>(
        d_rays, n_rays, n_coarse, n_fine, coarse->tsamp, coarse->delta, coarse->wts, d_xi, D.seed,
        (uint64_t)fine->step, fine->H[0], fine->delta, nullptr);
    st = backward_update(coarse, Mc, s);
    if (st != PLO_OK) return st;
    st = forward_layers(fine, Mf, s, true);
    if (st != PLO_OK) return st;
    e = launch_quad(fine, N, d_rays, d_rgb_gt, d_alpha_gt, n_rays, D.loss, nullptr, s);
    if (e != cudaSuccess) return cuda_error(e, "quadrature kernel launch");
    st = backward_update(fine, Mf, s);
    if (st != PLO_OK) return st;
    k_mean<<<1, 256, 0, s>>>(coarse->ray_loss, n_rays, d_loss_out, fine->ray_loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "loss reduction launch");
}

extern "C" plo_status plo_hier_samples(const float* d_rays, int32_t n_rays, int32_t n_coarse, int32_t n_fine,
                                       const float* d_t, const float* d_delta, const float* d_w, const float* d_xi,
                                       float* d_t_out, float* d_delta_out, void* stream) {
    if (!d_rays || !d_t || !d_delta || !d_w || !d_xi || !d_t_out || !d_delta_out)
        return set_error(PLO_ERR_INVALID_ARG, "a buffer is NULL");
    if (n_rays < 0) return set_error(PLO_ERR_INVALID_ARG, "n_rays must be >= 0");
    if (!hier_counts_ok(n_coarse, n_fine))
        return set_error(PLO_ERR_UNSUPPORTED, "n_coarse, n_fine: multiples of 32, n_coarse <= 128, and "
                                              "n_coarse + n_fine in {64, 96, 128, 192, 256}");
    if (n_rays == 0) return PLO_OK;
    k_fine<<<(unsigned)((n_rays + HIER_WARPS - 1) / HIER_WARPS), 32 * HIER_WARPS, 0, (cudaStream_t)stream>>>(
        d_rays, n_rays, n_coarse, n_fine, d_t, d_delta, d_w, d_xi, 0, 0, nullptr, d_delta_out, d_t_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "fine-sample kernel launch");
}

extern "C" plo_status plo_mlp_check(const plo_mlp* m, void* stream) {
    if (!m) return set_error(PLO_ERR_INVALID_ARG, "mlp is NULL");
    unsigned int flags = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&flags, m->d_err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "plo_mlp_check");
    if (flags) {
        cudaMemsetAsync(m->d_err, 0, 4, s);
        cudaStreamSynchronize(s);
        return set_error(PLO_ERR_TIMEOUT, "a tensor-core kernel gave up waiting on a pipeline barrier");
    }
    return PLO_OK;
}

extern "C" int64_t plo_mlp_step(const plo_mlp* m) { return m ? m->step : -1; }

// ---------------------------------------------------------------- test hooks of the training step
namespace plo {
namespace {
// d loss / d raw as fp32 [M][n_out] from the kernel's bf16 [M][64] (column 0
// from the paper architecture's sigma column when dsig is given)
__global__ void k_widen_grad(const __nv_bfloat16* dO, const __nv_bfloat16* dsig, int dsig_ld, int64_t M, int n_out,
                             float* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * n_out) return;
    const int64_t row = i / n_out;
    const int c = (int)(i - row * n_out);
    out[i] = __bfloat162float(c == 0 && dsig ? dsig[row * dsig_ld] : dO[row * OUT_PAD + c]);
}
}  // namespace
}  // namespace plo

extern "C" plo_status plo_mlp_get_activation(const plo_mlp* m, int32_t layer, void* d_out, int64_t n_rows,
                                             void* stream) {
    if (!m || !d_out) return set_error(PLO_ERR_INVALID_ARG, "mlp or output is NULL");
    const bool grad = layer >= PLO_MLP_DZ_BASE && layer < PLO_MLP_DZ_BASE + DEPTH;
    if (!grad && (layer < 0 || layer >= m->n_layers)) return set_error(PLO_ERR_INVALID_ARG, "layer out of range");
    if (n_rows < 0 || n_rows > m->cap) return set_error(PLO_ERR_INVALID_ARG, "n_rows exceeds the stored batch");
    if (n_rows == 0) return PLO_OK;
    const size_t bytes = (size_t)n_rows * (grad ? WIDTH : m->geom.in_pad[layer]) * 2;
    const void* src = grad ? (const void*)m->dZ[layer - PLO_MLP_DZ_BASE] : (const void*)m->H[layer];
    if (!src) return set_error(PLO_ERR_INVALID_ARG, "no stored batch");
    cudaError_t e = cudaMemcpyAsync(d_out, src, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "activation copy");
}

extern "C" plo_status plo_mlp_quad(plo_mlp* m, const float* d_rays, const float* d_raw, const float* d_delta,
                                   const float* d_rgb_gt, const float* d_alpha_gt, int32_t n_rays, int32_t n_samples,
                                   float* d_ray_out, float* d_draw, void* stream) {
    if (!m) return set_error(PLO_ERR_INVALID_ARG, "mlp is NULL");
    if (!d_rays || !d_raw || !d_delta || !d_rgb_gt || !d_alpha_gt || !d_ray_out)
        return set_error(PLO_ERR_INVALID_ARG, "a buffer is NULL");
    if (n_rays <= 0) return set_error(PLO_ERR_INVALID_ARG, "n_rays must be > 0");
    if (n_samples != 32 && n_samples != 64 && n_samples != 96 && n_samples != 128 && n_samples != 192 &&
        n_samples != 256)
        return set_error(PLO_ERR_UNSUPPORTED, "n_samples must be 32, 64, 96, 128, 192 or 256");
    const int64_t M = (int64_t)n_rays * n_samples;
    if (M > ((int64_t)1 << 28)) return set_error(PLO_ERR_INVALID_ARG, "batch too large");
    cudaStream_t s = (cudaStream_t)stream;
    plo_status st = ensure_workspace(m, M, n_rays);
    if (st != PLO_OK) return st;
    cudaError_t e = cudaMemcpy2DAsync(m->raw, OUT_PAD * 4, d_raw, (size_t)m->n_out * 4, (size_t)m->n_out * 4,
                                      (size_t)M, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->delta, d_delta, (size_t)M * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "quadrature input copy");
    e = launch_quad(m, n_samples, d_rays, d_rgb_gt, d_alpha_gt, n_rays, m->desc.loss, nullptr, s, d_ray_out);
    if (e != cudaSuccess) return cuda_error(e, "quadrature kernel launch");
    if (d_draw) {
        const __nv_bfloat16* dsig = m->arch == PLO_ARCH_PAPER ? m->dZc + FEAT : nullptr;
        const int64_t total = M * m->n_out;
        k_widen_grad<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m->dO, dsig, COMB_PAD, M, m->n_out, d_draw);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "gradient copy");
    }
    return PLO_OK;
}

// ---------------------------------------------------------------- raw GEMM entry points
extern "C" plo_status plo_gemm_bf16(const void* d_A, const void* d_B, int32_t M, int32_t N, int32_t K,
                                    int32_t epilogue, const float* d_bias, const void* d_mask, uint32_t* d_bits,
                                    void* d_out, unsigned int* d_err, void* stream) {
    if (!d_A || !d_B || !d_out || !d_err) return set_error(PLO_ERR_INVALID_ARG, "A, B, out or err is NULL");
    if (M <= 0) return set_error(PLO_ERR_INVALID_ARG, "M must be > 0");
    const bool shape_ok = (N == 256 && (K == 64 || K == 256)) || (N == 64 && K == 256);
    if (!shape_ok) return set_error(PLO_ERR_UNSUPPORTED, "(N, K) must be (256, 64), (256, 256) or (64, 256)");
    if (epilogue < 0 || epilogue > 3) return set_error(PLO_ERR_INVALID_ARG, "unknown epilogue");
    if ((epilogue <= 1 && !d_bias) || (epilogue == 2 && !d_mask) || (epilogue == 3 && !d_bits))
        return set_error(PLO_ERR_INVALID_ARG, "bias (epilogues 0, 1), mask (2) or bits (3) is NULL");
    if (d_bias && reinterpret_cast<uintptr_t>(d_bias) % 16 != 0)
        return set_error(PLO_ERR_INVALID_ARG, "bias must be 16-byte aligned (the epilogue reads it as float4)");
    const int epi = epilogue == 3 ? (int)gemm::EPI_MASKBITS_BF16 : epilogue;
    CUtensorMap mA, mB, mO;
    plo_status st = make_map(&mA, d_A, (uint64_t)M, (uint64_t)K, 128);
    if (st == PLO_OK) st = make_map(&mB, d_B, (uint64_t)N, (uint64_t)K, (uint32_t)N);
    if (st == PLO_OK && epilogue != gemm::EPI_BIAS_F32) st = make_store_map(&mO, d_out, (uint64_t)M, (uint64_t)N);
    if (st != PLO_OK) return st;
    gemm::EpiArgs ep{};
    ep.bias = d_bias;
    ep.out_bf16 = static_cast<__nv_bfloat16*>(d_out);
    ep.out_f32 = static_cast<float*>(d_out);
    ep.ldo = N;
    ep.mask = static_cast<const __nv_bfloat16*>(d_mask);
    ep.ldm = N;
    ep.bits_out = epilogue == 0 ? d_bits : nullptr;
    ep.bits = d_bits;
    ep.ldb = N / 32;
    ep.err = d_err;
    const int sms = sm_count_of_current();
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    const CUtensorMap* O = epilogue == gemm::EPI_BIAS_F32 ? nullptr : &mO;
    if (N == 256 && K == 64) e = launch_gemm<256, 64>(mA, mB, O, ep, epi, M, sms, s);
    else if (N == 256) e = launch_gemm<256, 256>(mA, mB, O, ep, epi, M, sms, s);
    else e = launch_gemm<64, 256>(mA, mB, O, ep, epi, M, sms, s);
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "GEMM launch");
}

// Test hook for failure detection: a GEMM whose producer issues no loads, so
// that every pipeline wait runs out after `wait_limit` polls; the kernel sets
// bit 1 of *d_err, frees its TMEM and returns (no trap, the context stays
// usable).  Same buffers as plo_gemm_bf16 with N = 256, K = 64.
extern "C" plo_status plo_debug_gemm_stall(const void* d_A, const void* d_B, int32_t M, void* d_out,
                                          unsigned int* d_err, uint32_t wait_limit, void* stream) {
    if (!d_A || !d_B || !d_out || !d_err || M <= 0) return set_error(PLO_ERR_INVALID_ARG, "bad argument");
    CUtensorMap mA, mB;
    plo_status st = make_map(&mA, d_A, (uint64_t)M, 64, 128);
    if (st == PLO_OK) st = make_map(&mB, d_B, 256, 64, 256);
    if (st != PLO_OK) return st;
    gemm::EpiArgs ep{};
    ep.out_bf16 = static_cast<__nv_bfloat16*>(d_out);
    ep.ldo = 256;
    ep.err = d_err;
    ep.wait_limit = wait_limit > 0 ? wait_limit : 1;
    ep.debug_skip_loads = 1;
    ep.mask = static_cast<const __nv_bfloat16*>(d_out);
    ep.ldm = 256;
    cudaError_t e =
        launch_gemm<256, 64>(mA, mB, nullptr, ep, gemm::EPI_MASK_BF16, M, sm_count_of_current(), (cudaStream_t)stream);
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "GEMM launch");
}

extern "C" plo_status plo_wgrad_bf16(const void* d_dZ, int32_t n_out, const void* d_H, int32_t n_in, int32_t M,
                                     float* d_dW, float* d_db, unsigned int* d_err, void* stream) {
    if (!d_dZ || !d_H || !d_dW || !d_err) return set_error(PLO_ERR_INVALID_ARG, "dZ, H, dW or err is NULL");
    if (M <= 0 || M % 64) return set_error(PLO_ERR_INVALID_ARG, "M must be a positive multiple of 64");
    if (!((n_out == 64 || n_out == 256) && (n_in == 64 || n_in == 256)))
        return set_error(PLO_ERR_UNSUPPORTED, "n_out and n_in must be 64 or 256");
    CUtensorMap mZ, mH;
    plo_status st = make_map(&mZ, d_dZ, (uint64_t)M, (uint64_t)n_out, 64);
    if (st == PLO_OK) st = make_map(&mH, d_H, (uint64_t)M, (uint64_t)n_in, 64);
    if (st != PLO_OK) return st;
    const int sms = sm_count_of_current();
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = n_in == 256 ? launch_wgrad<256>(mZ, mH, d_dW, n_out, M, sms, d_err, s, d_db)
                                : launch_wgrad<64>(mZ, mH, d_dW, n_out, M, sms, d_err, s, d_db);
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "weight-gradient GEMM launch");
}

// ---------------------------------------------------------------- distillation
// plo_distill (Sec. 5, "Creating the plenoctree"): the network's sigma at the
// centre of every voxel at `depth` decides which voxels are kept (sigma >=
// sigma_thresh); each kept voxel gets the mean of ReLU(sigma_raw) and of the
// raw SH coefficients over `samples` jittered positions inside it.  Voxels
// are visited in Morton order, so the kept list is sorted, and the octree is
// packed on the device from it (pack.cu): no host copy of the leaves.
namespace {
plo_status distill(plo_mlp* m, int32_t depth, int32_t samples, float sigma_thresh, int32_t precision, plo_tree** out,
                   void* stream) {
    if (!m || !out) return set_error(PLO_ERR_INVALID_ARG, "mlp or out is NULL");
    *out = nullptr;
    if (depth < 1 || depth > 10) return set_error(PLO_ERR_INVALID_ARG, "depth must be in [1, 10]");
    if (samples < 1 || samples > 256) return set_error(PLO_ERR_INVALID_ARG, "samples must be in [1, 256]");
    if (!(sigma_thresh >= 0.0f)) return set_error(PLO_ERR_INVALID_ARG, "sigma_thresh must be >= 0");
    if (precision < PLO_PREC_FP32 || precision > PLO_PREC_BF16)
        return set_error(PLO_ERR_INVALID_ARG, "precision must be PLO_PREC_FP32, _FP16 or _BF16");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t total = (int64_t)1 << (3 * depth);
    const int64_t C = total < ((int64_t)1 << 19) ? total : ((int64_t)1 << 19);
    plo_status st = ensure_workspace(m, C < 128 ? 128 : C, m->cap_rays);
    if (st != PLO_OK) return st;
    const int K = m->K;
    const int stride = sh_stride_bytes(K, precision);
    // pass 1: sigma at every voxel centre, in chunks of C voxels (Morton
    // order); the kept voxels' codes are appended on the device in that
    // order (a Morton code at depth <= 10 fits 30 bits)
    uint32_t *d_flag = nullptr, *d_pos = nullptr, *d_count = nullptr, *d_codes = nullptr;
    cudaError_t e = (cudaError_t)dev_malloc((void**)&d_flag, (size_t)C * 4);
    if (e == cudaSuccess) e = (cudaError_t)dev_malloc((void**)&d_pos, (size_t)C * 4);
    if (e == cudaSuccess) e = (cudaError_t)dev_malloc((void**)&d_count, 256);
    if (e == cudaSuccess) e = (cudaError_t)dev_malloc((void**)&d_codes, (size_t)total * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_count, 0, 4, s);
    auto free_pass1 = [&]() {
        cudaStreamSynchronize(s);
        cudaFree(d_flag);
        cudaFree(d_pos);
        cudaFree(d_count);
    };
    for (int64_t base = 0; e == cudaSuccess && st == PLO_OK && base < total; base += C) {
        const int64_t n = total - base < C ? total - base : C;
        k_pe_centres<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((uint64_t)base, n, depth, m->H[0]);
        st = forward_layers(m, n, s, false, false);  // only H[8] is read (by the head)
        if (st != PLO_OK) break;
        k_keep<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m->raw, n, sigma_thresh, d_flag);
        e = device_exclusive_scan(d_flag, d_pos, n, s);
        if (e != cudaSuccess) break;
        k_compact_kept<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((uint64_t)base, n, d_flag, d_pos, d_count, d_codes);
        k_advance_count<<<1, 1, 0, s>>>(d_flag, d_pos, n, d_count);
        e = cudaGetLastError();
    }
    uint32_t nl32 = 0;
    if (e == cudaSuccess && st == PLO_OK) e = cudaMemcpyAsync(&nl32, d_count, 4, cudaMemcpyDeviceToHost, s);
    free_pass1();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (st != PLO_OK || e != cudaSuccess) {
        cudaFree(d_codes);
        return st != PLO_OK ? st : cuda_error(e, "plo_distill");
    }
    const int64_t nl = nl32;
    // pass 2: the mean of `samples` jittered evaluations per kept voxel,
    // packed straight into the leaf's record and entry word
    uint32_t* d_yword = nullptr;
    uint8_t *d_emits = nullptr, *d_rec = nullptr;
    e = (cudaError_t)dev_malloc((void**)&d_yword, (size_t)std::max<int64_t>(nl, 1) * 4);
    if (e == cudaSuccess) e = (cudaError_t)dev_malloc((void**)&d_emits, (size_t)std::max<int64_t>(nl, 1));
    if (e == cudaSuccess) e = (cudaError_t)dev_malloc((void**)&d_rec, (size_t)std::max<int64_t>(nl, 1) * stride);
    const int64_t vmax = C / samples > 0 ? C / samples : 1;
    for (int64_t off = 0; off < nl && e == cudaSuccess && st == PLO_OK; off += vmax) {
        const int64_t nv = nl - off < vmax ? nl - off : vmax;
        k_pe_jitter<<<(unsigned)((nv * samples + 255) / 256), 256, 0, s>>>(d_codes + off, nv, samples, depth,
                                                                          m->desc.seed, m->H[0]);
        st = forward_layers(m, nv * samples, s, false, false);
        if (st != PLO_OK) break;
        const unsigned g = (unsigned)((nv + 127) / 128);
        uint8_t* rec = d_rec + (size_t)off * stride;
        if (precision == PLO_PREC_FP32)
            k_pack_leaves<PLO_PREC_FP32><<<g, 128, 0, s>>>(m->raw, nv, samples, K, stride, d_yword + off, d_emits + off, rec);
        else if (precision == PLO_PREC_FP16)
            k_pack_leaves<PLO_PREC_FP16><<<g, 128, 0, s>>>(m->raw, nv, samples, K, stride, d_yword + off, d_emits + off, rec);
        else
            k_pack_leaves<PLO_PREC_BF16><<<g, 128, 0, s>>>(m->raw, nv, samples, K, stride, d_yword + off, d_emits + off, rec);
        e = cudaGetLastError();
    }
    if (st == PLO_OK && e == cudaSuccess) st = plo_mlp_check(m, stream);
    // the octree over the kept voxels, leaves at level `depth`, packed on
    // the device from the sorted codes
    if (st == PLO_OK && e == cudaSuccess)
        st = pack_voxel_tree(depth, m->desc.sh_degree, precision, d_codes, nl, d_yword, d_emits, d_rec, s, out);
    cudaStreamSynchronize(s);
    cudaFree(d_codes);
    cudaFree(d_yword);
    cudaFree(d_emits);
    if (st != PLO_OK || e != cudaSuccess) {
        cudaFree(d_rec);
        return st != PLO_OK ? st : cuda_error(e, "plo_distill");
    }
    return PLO_OK;
}
}  // namespace

// Everything stays on the device (per kept voxel: a 4-byte code, an entry
// word and its SH record); an allocation failure is returned as
// PLO_ERR_OOM, never thrown through the C ABI.
extern "C" plo_status plo_distill(plo_mlp* m, int32_t depth, int32_t samples, float sigma_thresh,
                                  int32_t precision, plo_tree** out, void* stream) {
    try {
        return distill(m, depth, samples, sigma_thresh, precision, out, stream);
    } catch (const std::bad_alloc&) {
        if (out) *out = nullptr;
        return set_error(PLO_ERR_OOM, "host allocation during distillation failed");
    }
}

// ---------------------------------------------------------------- checkpoints
// File layout (little-endian):
//   bytes 0..7    magic "PLOMLP01"
//   bytes 8..15   uint64 length H of the header
//   bytes 16..    the header: flat JSON object, ASCII, H bytes, with the
//                 network description (arch, sh_degree, transmittance, loss,
//                 total_steps, l_max, eps, lr0, lr1, init_radiance: floats
//                 printed with 9 significant digits, which round-trips FP32;
//                 seed as a decimal string), the step count and the blob table
//   then the blobs, each starting at a multiple of 64 bytes from the file
//   start: "master", "adam_m", "adam_v" (f32, n_params each, the canonical
//   parameter order of plo_mlp_get_params) and "weights_bf16" (bf16, the
//   trained weights W of every canonical block, no biases, the copies the
//   forward pass multiplies with).
// The jitter of the stratified samples is keyed by (seed, step), so the two
// restore the sample stream of an interrupted run.
namespace {

constexpr char kCkptMagic[9] = "PLOMLP01";
constexpr const char* kBlobNames[4] = {"master", "adam_m", "adam_v", "weights_bf16"};

int64_t weight_count(int arch, int n_out) {
    Block bl[MAX_LAYERS + 2];
    const int nb = canonical_blocks(arch, n_out, bl);
    int64_t c = 0;
    for (int k = 0; k < nb; ++k) c += (int64_t)bl[k].rows * bl[k].cols;
    return c;
}

std::string fmt_float(float v) {
    char buf[48];
    std::snprintf(buf, sizeof(buf), "%.9g", (double)v);
    return buf;
}

// Value of "key" in the flat JSON header (number or string, without quotes).
bool json_value(const std::string& h, const char* key, std::string& out) {
    const std::string pat = std::string("\"") + key + "\":";
    size_t p = h.find(pat);
    if (p == std::string::npos) return false;
    p += pat.size();
    while (p < h.size() && h[p] == ' ') ++p;
    if (p >= h.size()) return false;
    if (h[p] == '"') {
        size_t q = h.find('"', p + 1);
        if (q == std::string::npos) return false;
        out = h.substr(p + 1, q - p - 1);
        return true;
    }
    size_t q = p;
    while (q < h.size() && h[q] != ',' && h[q] != '}' && h[q] != ' ') ++q;
    out = h.substr(p, q - p);
    return !out.empty();
}

bool json_int(const std::string& h, const char* key, int64_t& v) {
    std::string s;
    if (!json_value(h, key, s)) return false;
    char* end = nullptr;
    const long long x = std::strtoll(s.c_str(), &end, 10);
    if (!end || *end) return false;
    v = x;
    return true;
}

bool json_float(const std::string& h, const char* key, float& v) {
    std::string s;
    if (!json_value(h, key, s)) return false;
    char* end = nullptr;
    const float x = std::strtof(s.c_str(), &end);
    if (!end || *end) return false;
    v = x;
    return true;
}

struct CkptHeader {
    plo_mlp_desc desc;
    int64_t step, n_params, n_weights;
    int64_t off[4];  // blob offsets from the file start
    int64_t data_end;
};

// Reads and checks the header (magic, keys, counts against the arch, blob
// offsets and the file size); host only.
plo_status read_ckpt_header(std::FILE* f, CkptHeader* out) {
    char magic[8];
    uint64_t hl = 0;
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kCkptMagic, 8) != 0)
        return set_error(PLO_ERR_INVALID_ARG, "not a plo network checkpoint (bad magic)");
    if (std::fread(&hl, 8, 1, f) != 1 || hl == 0 || hl > (1u << 20))
        return set_error(PLO_ERR_INVALID_ARG, "checkpoint header length is missing or out of range");
    std::string h(hl, '\0');
    if (std::fread(&h[0], 1, hl, f) != hl) return set_error(PLO_ERR_INVALID_ARG, "checkpoint header is truncated");
    std::string fmt;
    int64_t version = 0;
    if (!json_value(h, "format", fmt) || fmt != "plo-mlp" || !json_int(h, "version", version) || version != 1)
        return set_error(PLO_ERR_UNSUPPORTED, "unknown checkpoint format or version");
    plo_mlp_desc d{};
    int64_t arch, deg, trans, loss, total, step, np;
    std::string seed;
    if (!json_int(h, "arch", arch) || !json_int(h, "sh_degree", deg) || !json_int(h, "transmittance", trans) ||
        !json_int(h, "loss", loss) || !json_int(h, "total_steps", total) || !json_float(h, "l_max", d.l_max) ||
        !json_float(h, "eps", d.eps) || !json_float(h, "lr0", d.lr0) || !json_float(h, "lr1", d.lr1) ||
        !json_float(h, "init_radiance", d.init_radiance) || !json_value(h, "seed", seed) ||
        !json_int(h, "step", step) || !json_int(h, "n_params", np))
        return set_error(PLO_ERR_INVALID_ARG, "checkpoint header lacks a required key");
    d.arch = (int32_t)arch;
    d.sh_degree = (int32_t)deg;
    d.transmittance = (int32_t)trans;
    d.loss = (int32_t)loss;
    d.total_steps = (int32_t)total;
    char* end = nullptr;
    d.seed = std::strtoull(seed.c_str(), &end, 10);
    if (seed.empty() || !end || *end) return set_error(PLO_ERR_INVALID_ARG, "checkpoint seed is not a decimal integer");
    plo_status st = check_mlp_desc(&d);
    if (st != PLO_OK) return st;
    if (step < 0) return set_error(PLO_ERR_INVALID_ARG, "checkpoint step is negative");
    const int n_out = 1 + 3 * (d.sh_degree + 1) * (d.sh_degree + 1);
    if (np != canonical_count(d.arch, n_out))
        return set_error(PLO_ERR_INVALID_ARG, "checkpoint n_params does not match its architecture");
    const int64_t nw = weight_count(d.arch, n_out);
    int64_t pos = 16 + (int64_t)hl;
    for (int b = 0; b < 4; ++b) {
        const std::string key = std::string(kBlobNames[b]) + "_offset";
        int64_t o = 0;
        if (!json_int(h, key.c_str(), o)) return set_error(PLO_ERR_INVALID_ARG, "checkpoint lacks a blob offset");
        if (o < pos || o % 64 != 0) return set_error(PLO_ERR_INVALID_ARG, "checkpoint blob offsets are out of order");
        out->off[b] = o;
        pos = o + (b < 3 ? np * 4 : nw * 2);
    }
    if (std::fseek(f, 0, SEEK_END) != 0) return set_error(PLO_ERR_INVALID_ARG, "checkpoint is not seekable");
    const long size = std::ftell(f);
    if (size < 0 || (int64_t)size < pos) return set_error(PLO_ERR_INVALID_ARG, "checkpoint file is truncated");
    out->desc = d;
    out->step = step;
    out->n_params = np;
    out->n_weights = nw;
    out->data_end = pos;
    return PLO_OK;
}

// bf16 weights of the canonical blocks, gathered from the device copies
plo_status download_bf16_weights(const plo_mlp* m, std::vector<uint16_t>& out) {
    Block bl[MAX_LAYERS + 2];
    const int nb = canonical_blocks(m->arch, m->n_out, bl);
    const LayerGeom& g = m->geom;
    out.clear();
    for (int k = 0; k < nb; ++k) {
        const Block& B = bl[k];
        std::vector<uint16_t> pad((size_t)g.out_pad[B.layer] * g.in_pad[B.layer]);
        cudaError_t e = cudaMemcpy(pad.data(), m->W[B.layer], pad.size() * 2, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_error(e, "bf16 weight download");
        for (int o = 0; o < B.rows; ++o)
            for (int i = 0; i < B.cols; ++i) out.push_back(pad[(size_t)(B.row0 + o) * g.in_pad[B.layer] + i]);
    }
    return PLO_OK;
}

plo_status save_mlp(const plo_mlp* m, const char* path) {
    const int64_t np = canonical_count(m->arch, m->n_out);
    std::vector<float> blobs[3];
    const float* src[3] = {m->master, m->adam_m, m->adam_v};
    for (int b = 0; b < 3; ++b) {
        blobs[b].resize(np);
        plo_status st = download_canonical(m, src[b], blobs[b].data(), np);
        if (st != PLO_OK) return st;
    }
    std::vector<uint16_t> wb;
    plo_status st = download_bf16_weights(m, wb);
    if (st != PLO_OK) return st;
    const plo_mlp_desc& d = m->desc;
    // the header's length depends on the offsets it lists: fix the offsets
    // for a header of at most 1 KiB of padding, then pad to that length
    std::string h;
    int64_t off[4];
    for (int pass = 0; pass < 2; ++pass) {
        int64_t pos = pass == 0 ? 0 : (int64_t)(16 + h.size() + 63) / 64 * 64;
        for (int b = 0; b < 4; ++b) {
            off[b] = pos;
            pos = (pos + (b < 3 ? np * 4 : (int64_t)wb.size() * 2) + 63) / 64 * 64;
        }
        h = "{\"format\": \"plo-mlp\", \"version\": 1, \"arch\": " + std::to_string(d.arch) +
            ", \"sh_degree\": " + std::to_string(d.sh_degree) + ", \"transmittance\": " +
            std::to_string(d.transmittance) + ", \"loss\": " + std::to_string(d.loss) + ", \"total_steps\": " +
            std::to_string(d.total_steps) + ", \"l_max\": " + fmt_float(d.l_max) + ", \"eps\": " + fmt_float(d.eps) +
            ", \"lr0\": " + fmt_float(d.lr0) + ", \"lr1\": " + fmt_float(d.lr1) + ", \"init_radiance\": " +
            fmt_float(d.init_radiance) + ", \"seed\": \"" + std::to_string((unsigned long long)d.seed) +
            "\", \"step\": " + std::to_string(m->step) + ", \"n_params\": " + std::to_string(np);
        for (int b = 0; b < 4; ++b)
            h += std::string(", \"") + kBlobNames[b] + "_offset\": " + std::to_string(off[b] + (pass ? 0 : 100000000000LL));
        h += "}";
    }
    // pass 0 used wide placeholder offsets, so the real header is no longer
    const int64_t data0 = (int64_t)(16 + h.size() + 63) / 64 * 64;
    if (off[0] < data0) return set_error(PLO_ERR_CUDA, "checkpoint header layout");  // cannot happen
    std::FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(PLO_ERR_INVALID_ARG, std::string("cannot open checkpoint for writing: ") + path);
    const uint64_t hl = h.size();
    bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(&hl, 8, 1, f) == 1 &&
              std::fwrite(h.data(), 1, h.size(), f) == h.size();
    int64_t pos = 16 + (int64_t)h.size();
    static const char zeros[64] = {};
    for (int b = 0; b < 4 && ok; ++b) {
        for (int64_t gap = off[b] - pos; gap > 0 && ok; gap -= 64) {
            const size_t z = (size_t)(gap < 64 ? gap : 64);
            ok = std::fwrite(zeros, 1, z, f) == z;
        }
        const size_t n = b < 3 ? (size_t)np : wb.size();
        const size_t es = b < 3 ? 4 : 2;
        const void* p = b < 3 ? (const void*)blobs[b].data() : (const void*)wb.data();
        ok = ok && std::fwrite(p, es, n, f) == n;
        pos = off[b] + (int64_t)(n * es);
    }
    ok = std::fclose(f) == 0 && ok;
    return ok ? PLO_OK : set_error(PLO_ERR_INVALID_ARG, std::string("writing the checkpoint failed: ") + path);
}

}  // namespace

extern "C" plo_status plo_mlp_save(const plo_mlp* m, const char* path) {
    if (!m || !path) return set_error(PLO_ERR_INVALID_ARG, "mlp or path is NULL");
    try {
        return save_mlp(m, path);
    } catch (const std::bad_alloc&) {
        return set_error(PLO_ERR_OOM, "host allocation while saving the network failed");
    }
}

extern "C" plo_status plo_mlp_checkpoint_info(const char* path, plo_mlp_desc* desc, int64_t* step) {
    if (!path) return set_error(PLO_ERR_INVALID_ARG, "path is NULL");
    std::FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(PLO_ERR_INVALID_ARG, std::string("cannot open checkpoint: ") + path);
    CkptHeader hd{};
    plo_status st;
    try {
        st = read_ckpt_header(f, &hd);
    } catch (const std::bad_alloc&) {
        st = set_error(PLO_ERR_OOM, "host allocation while reading the checkpoint failed");
    }
    std::fclose(f);
    if (st != PLO_OK) return st;
    if (desc) *desc = hd.desc;
    if (step) *step = hd.step;
    return PLO_OK;
}

namespace {
plo_status load_mlp(const char* path, plo_mlp** out) {
    std::FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(PLO_ERR_INVALID_ARG, std::string("cannot open checkpoint: ") + path);
    CkptHeader hd{};
    plo_status st = read_ckpt_header(f, &hd);
    std::vector<float> blobs[3];
    std::vector<uint16_t> wb;
    for (int b = 0; b < 4 && st == PLO_OK; ++b) {
        const size_t n = b < 3 ? (size_t)hd.n_params : (size_t)hd.n_weights;
        void* p;
        size_t es;
        if (b < 3) {
            blobs[b].resize(n);
            p = blobs[b].data();
            es = 4;
        } else {
            wb.resize(n);
            p = wb.data();
            es = 2;
        }
        if (std::fseek(f, (long)hd.off[b], SEEK_SET) != 0 || std::fread(p, es, n, f) != n)
            st = set_error(PLO_ERR_INVALID_ARG, "checkpoint blob is truncated");
    }
    std::fclose(f);
    if (st != PLO_OK) return st;
    plo_mlp* m = nullptr;
    st = plo_mlp_create(&hd.desc, 0, &m);
    if (st != PLO_OK) return st;
    std::vector<float> pad;
    float* dst[3] = {m->master, m->adam_m, m->adam_v};
    for (int b = 0; b < 3 && st == PLO_OK; ++b) {
        canonical_to_padded(m, blobs[b].data(), pad);
        cudaError_t e = cudaMemcpy(dst[b], pad.data(), pad.size() * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_error(e, "checkpoint upload");
    }
    if (st == PLO_OK) st = refresh_bf16(m, nullptr);
    if (st == PLO_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_error(e, "checkpoint upload");
    }
    // the bf16 copies are the rounding of the masters: a mismatch means the
    // file's blobs do not belong together
    std::vector<uint16_t> now;
    if (st == PLO_OK) st = download_bf16_weights(m, now);
    if (st == PLO_OK && now != wb)
        st = set_error(PLO_ERR_INVALID_ARG, "checkpoint's bf16 weights are not the rounding of its FP32 masters");
    if (st != PLO_OK) {
        plo_mlp_free(m);
        return st;
    }
    m->step = hd.step;
    *out = m;
    return PLO_OK;
}
}  // namespace

extern "C" plo_status plo_mlp_load(const char* path, plo_mlp** out) {
    if (!out) return set_error(PLO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!path) return set_error(PLO_ERR_INVALID_ARG, "path is NULL");
    try {
        return load_mlp(path, out);
    } catch (const std::bad_alloc&) {
        return set_error(PLO_ERR_OOM, "host allocation while loading the network failed");
    }
}
