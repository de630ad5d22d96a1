// Direct optimisation of the octree's leaves (Sec. 7, "Limitations --
// Precomputation cost": the SH octree fitted by itself, with a
// total-variation regulariser, instead of a network projected onto it).
//
// One step on a batch of rays:
//   1. plo_trace_rays of the structure tree (the octree with zero leaves, so
//      no ray saturates): per ray its cells in order with their canonical
//      leaf ids and [t_in, t_out] -- the same walk as plo_render_rays;
//   2. k_grad: per ray (one thread), the forward composite over the leaves
//      with sigma = max(0, s) > 0 (Eq. 3-5), compacting them at the front of
//      the ray's trace row as (leaf, delta) and (w, T_out); the loss (Sec.
//      4.3, Eq. 7-9); then, back to front, d loss / d a_j and the SH
//      gradients, added to the leaves with atomics;
//   3. k_tv_terms, k_tv_grad: the TV terms and their gradients over the
//      face-neighbour table and its reverse (two gathers, no atomics);
//   4. k_adam: Adam over the raw densities and the coefficients.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "plo_internal.h"
#include "sh.cuh"

struct plo_octopt {
    int32_t depth = 0, sh_degree = 0, K = 0;
    int64_t n_leaves = 0, n_nodes = 0;
    int32_t device = 0;
    int32_t max_cells = 0;
    plo_octopt_config cfg{};
    float bbox_min[3]{}, bbox_max[3]{};
    std::vector<int32_t> child;  // canonical child table of the structure
    plo_tree* walk = nullptr;    // the structure with zero leaves (trace only)
    int64_t step = 0;            // Adam updates done
    float* d_s = nullptr;        // raw densities [n_leaves]
    float* d_k = nullptr;        // coefficients [n_leaves][3K]
    float* d_gs = nullptr;       // gradients of the last grad / step
    float* d_gk = nullptr;
    float* d_ms = nullptr;       // Adam moments
    float* d_vs = nullptr;
    float* d_mk = nullptr;
    float* d_vk = nullptr;
    int32_t* d_nb = nullptr;     // face neighbours [n_leaves][3], -1 none
    int32_t* d_rev_off = nullptr;  // reverse neighbours: leaf i's are d_rev[d_rev_off[i] .. d_rev_off[i+1])
    int32_t* d_rev = nullptr;      // the leaves j with n_a(j) = i for some axis a
    float* d_tv_s = nullptr;       // per (leaf, channel): sqrt(eps + sum_a d_a^2) of the last TV pass
    float* d_tv_own = nullptr;     // per (leaf, channel): -sum_a d_a / s
    int64_t* d_tr_leaf = nullptr;  // trace scratch [max_rays][max_cells]
    float* d_tr_t = nullptr;       // [max_rays][max_cells][2]
    int32_t* d_tr_count = nullptr; // [max_rays]
    float* d_acc = nullptr;        // mean loss, TV(s), TV(k)
    unsigned int* d_flags = nullptr;  // bit 0: a ray crossed more than max_cells cells
};

namespace plo {
namespace {

constexpr int THREADS = 128;
constexpr float TV_EPS = 1e-8f;

struct GradArgs {
    const float* rays;
    const float* rgb_gt;
    const float* alpha_gt;
    int64_t n;
    int64_t* tr_leaf;  // rewritten in place: (int32 leaf, float delta) pairs
    float* tr_t;       // rewritten in place: (w, T_out) pairs
    const int32_t* tr_count;
    int32_t max_cells;
    const float* s;
    const float* k;
    float* gs;
    float* gk;
    float* ray_out;
    float* acc;
    unsigned int* flags;
    int32_t transmittance, loss_kind;
    float l_max, eps, inv_n;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Emission of one leaf in the ray's direction: sigmoid(sum_k k_{ch,k} Y_k)
// per channel (times l_max by the caller).
template <int K>
__device__ __forceinline__ void leaf_sigmoid(const float* kk, const float* Y, float* sg) {
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float z = 0.0f;
#pragma unroll
        for (int j = 0; j < K; ++j) z = __fmaf_rn(__ldg(kk + ch * K + j), Y[j], z);
        sg[ch] = 1.0f / (1.0f + expf(-z));
    }
}

// One thread per ray.  Pass 1 composites the ray front to back over its
// leaves (Eq. 3-5; the optical depth as a compensated sum, exponential
// weights T_in (1 - e^{-a}), linear ones min(T_in, a)) and keeps, at the
// front of the ray's trace row, each leaf with sigma > 0 as (leaf, delta)
// and (w, T_out).  Pass 2 runs back to front over those entries with
// g_j = sum_ch c_{j,ch} dL/dC_ch + dL/dalpha (dL/dw_j):
//   exponential: dL/da_j = T_out,j g_j - sum_{k>j} w_k g_k;
//   linear:      dL/da_j = g_j before the leaf s where T reaches 0, minus
//                g_s for j < s; 0 from s on;
// d L / d s_j = dL/da_j delta_j (sigma_j > 0 here), and per channel
// d L / d k_{j,ch,k} = w_j dL/dC_ch l_max sig (1 - sig) Y_k.
template <int K>
__global__ void __launch_bounds__(THREADS) k_grad(GradArgs p) {
    const int64_t r = (int64_t)blockIdx.x * THREADS + threadIdx.x;
    float loss = 0.0f;
    if (r < p.n) {
        int32_t cnt = p.tr_count[r];
        const bool over = cnt > p.max_cells;
        if (over) {
            atomicOr(p.flags, 1u);
            cnt = 0;
        }
        float dw[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) dw[a] = __ldg(p.rays + 6 * r + 3 + a);
        const float inv = rsqrtf(__fadd_rn(__fadd_rn(__fmul_rn(dw[0], dw[0]), __fmul_rn(dw[1], dw[1])),
                                           __fmul_rn(dw[2], dw[2])));
        float Y[K];
        sh_basis<K>(__fmul_rn(dw[0], inv), __fmul_rn(dw[1], inv), __fmul_rn(dw[2], inv), Y);
        int64_t* row_leaf = p.tr_leaf + r * p.max_cells;
        int2* packed = reinterpret_cast<int2*>(row_leaf);
        float2* wt = reinterpret_cast<float2*>(p.tr_t + 2 * r * p.max_cells);
        const bool lin = p.transmittance == PLO_TRANS_LINEAR;

        // pass 1
        float T = 1.0f, od_hi = 0.0f, od_lo = 0.0f, alpha = 0.0f;
        float C[3] = {0.0f, 0.0f, 0.0f}, csat[3] = {0.0f, 0.0f, 0.0f};
        int m = 0, sat = -1;
        for (int j = 0; j < cnt; ++j) {
            const int64_t leaf = row_leaf[j];
            const float2 tt = wt[j];
            if (leaf < 0) continue;
            const float sv = __ldg(p.s + leaf);
            if (!(sv > 0.0f)) continue;
            const float delta = __fsub_rn(tt.y, tt.x);
            const float a = sv * delta;
            // compensated optical depth (two-sum)
            const float sh = od_hi + a;
            const float bb = sh - od_hi;
            const float err = (od_hi - (sh - bb)) + (a - bb);
            const float lo = od_lo + err;
            od_hi = sh + lo;
            od_lo = lo - (od_hi - sh);
            float w, Tn;
            if (!lin) {
                w = T * (-expm1f(-a));
                Tn = expf(-(od_hi + od_lo));
            } else {
                Tn = fmaxf(0.0f, __fsub_rn(__fsub_rn(1.0f, od_hi), od_lo));
                w = fminf(T, a);
            }
            float sg[3];
            leaf_sigmoid<K>(p.k + leaf * 3 * K, Y, sg);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) C[ch] = __fmaf_rn(w, p.l_max * sg[ch], C[ch]);
            alpha += w;
            packed[m] = make_int2((int)leaf, __float_as_int(delta));
            wt[m] = make_float2(w, Tn);
            ++m;
            T = Tn;
            if (T <= 0.0f) {  // nothing behind contributes
                if (lin) {
                    sat = m - 1;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) csat[ch] = p.l_max * sg[ch];
                }
                break;
            }
        }

        // the loss on values divided by l_max (denominator held constant)
        float dC[3];
        const float inv_l = 1.0f / p.l_max;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float cn = C[ch] * inv_l, gn = __ldg(p.rgb_gt + 3 * r + ch) * inv_l;
            const float den = p.loss_kind == PLO_LOSS_MSE ? 1.0f : cn + p.eps;
            const float res = (cn - gn) / den;
            loss += res * res;
            dC[ch] = 2.0f * res / den * inv_l * p.inv_n;
        }
        float dA = 0.0f;
        if (p.loss_kind == PLO_LOSS_PAPER) {
            const float da = alpha - __ldg(p.alpha_gt + r);
            loss += da * da;
            dA = 2.0f * da * p.inv_n;
        }
        if (over) loss = 0.0f;
        if (p.ray_out) {
            float* o = p.ray_out + 5 * r;
            const float nan = __int_as_float(0x7fc00000);
            o[0] = over ? nan : C[0];
            o[1] = over ? nan : C[1];
            o[2] = over ? nan : C[2];
            o[3] = over ? nan : alpha;
            o[4] = over ? nan : loss;
        }

        // pass 2, back to front
        const float gsat = sat >= 0 ? __fmaf_rn(csat[0], dC[0], __fmaf_rn(csat[1], dC[1], __fmaf_rn(csat[2], dC[2], dA)))
                                    : 0.0f;
        float after = 0.0f;  // sum over the later leaves of w g
        for (int j = m - 1; j >= 0; --j) {
            const int2 e = packed[j];
            const float2 q = wt[j];
            const int64_t leaf = e.x;
            const float delta = __int_as_float(e.y), w = q.x, Tn = q.y;
            float sg[3];
            leaf_sigmoid<K>(p.k + leaf * 3 * K, Y, sg);
            float g = dA;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) g = __fmaf_rn(p.l_max * sg[ch], dC[ch], g);
            float da;
            if (!lin) {
                da = __fmaf_rn(Tn, g, -after);
                after = __fmaf_rn(w, g, after);
            } else {
                da = sat < 0 ? g : (j < sat ? g - gsat : 0.0f);
            }
            atomicAdd(p.gs + leaf, da * delta);
            float* gk = p.gk + leaf * 3 * K;
            float dz[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) dz[ch] = w * dC[ch] * p.l_max * sg[ch] * (1.0f - sg[ch]);
            if constexpr ((3 * K) % 4 == 0) {
                // a leaf's 3K coefficients are whole 16-byte groups (rows of
                // 3K floats from a 256-byte aligned base): one vector
                // reduction per four coefficients instead of four
#pragma unroll
                for (int q = 0; q < 3 * K / 4; ++q) {
                    float4 v;
                    v.x = dz[(4 * q + 0) / K] * Y[(4 * q + 0) % K];
                    v.y = dz[(4 * q + 1) / K] * Y[(4 * q + 1) % K];
                    v.z = dz[(4 * q + 2) / K] * Y[(4 * q + 2) % K];
                    v.w = dz[(4 * q + 3) / K] * Y[(4 * q + 3) % K];
                    atomicAdd(reinterpret_cast<float4*>(gk) + q, v);
                }
            } else {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) atomicAdd(gk + ch * K + kk, dz[ch] * Y[kk]);
            }
        }
    }
    loss = warp_sum(loss);
    if ((threadIdx.x & 31) == 0 && loss != 0.0f) atomicAdd(p.acc, loss * p.inv_n);
}

// TV of C channels x [n][C], pass 1, over every (leaf i, channel c) in a
// grid-stride loop: d_a = x[n_a(i)] - x[i] (0 without a neighbour), s =
// sqrt(eps + sum_a d_a^2); stores s and own = -sum_a d_a / s, and adds the
// sum of s / n to *val once per block (one address: a per-warp atomic cost
// ~1 ms on 24M elements).
__global__ void __launch_bounds__(THREADS) k_tv_terms(const float* x, int C, const int32_t* nb, int64_t n,
                                                       float* s_out, float* own_out, float* val) {
    __shared__ float s_part[THREADS / 32];
    float v = 0.0f;
    for (int64_t idx = (int64_t)blockIdx.x * THREADS + threadIdx.x; idx < n * C;
         idx += (int64_t)gridDim.x * THREADS) {
        const int64_t i = idx / C;
        const int c = (int)(idx - i * C);
        const float xi = x[idx];
        float d[3], q = TV_EPS;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int32_t j = nb[3 * i + a];
            d[a] = j >= 0 ? x[(int64_t)j * C + c] - xi : 0.0f;
            q = __fmaf_rn(d[a], d[a], q);
        }
        const float sv = sqrtf(q);
        s_out[idx] = sv;
        own_out[idx] = -(d[0] + d[1] + d[2]) / sv;
        v += sv;
    }
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < THREADS / 32; ++w) t += s_part[w];
        if (t != 0.0f) atomicAdd(val, t / (float)n);
    }
}

// Pass 2: d TV / d x[i][c] = (own + sum over the leaves j that have i as a
// neighbour of (x[i] - x[j]) / s[j]) / n, times lambda: added to g (one
// writer per element).
__global__ void __launch_bounds__(THREADS) k_tv_grad(const float* x, int C, const int32_t* rev_off,
                                                      const int32_t* rev, int64_t n, const float* s_in,
                                                      const float* own_in, float scale, float* g) {
    const int64_t idx = (int64_t)blockIdx.x * THREADS + threadIdx.x;
    if (idx >= n * C) return;
    const int64_t i = idx / C;
    const int c = (int)(idx - i * C);
    const float xi = x[idx];
    float acc = own_in[idx];
    for (int32_t r = rev_off[i]; r < rev_off[i + 1]; ++r) {
        const int64_t jc = (int64_t)rev[r] * C + c;
        acc += (xi - x[jc]) / s_in[jc];
    }
    g[idx] += scale * acc;
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8); bc1, bc2 = 1 - beta^t.
__global__ void __launch_bounds__(256) k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                                              float bc1, float bc2) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const float gi = g[i];
        const float mi = __fmaf_rn(0.9f, m[i], 0.1f * gi);
        const float vi = __fmaf_rn(0.999f, v[i], 0.001f * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    }
}

// int64 lookup results -> int32 neighbour ids (-1: none).
__global__ void k_nb_from_lookup(const int64_t* leaf, int64_t n, int32_t* nb) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i < n) nb[i] = leaf[i] >= 0 ? (int32_t)leaf[i] : -1;
}

unsigned grid_of(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <int K>
cudaError_t launch_grad(const GradArgs& a, cudaStream_t s) {
    k_grad<K><<<grid_of(a.n, THREADS), THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t dispatch_grad(int K, const GradArgs& a, cudaStream_t s) {
    switch (K) {
        case 1: return launch_grad<1>(a, s);
        case 4: return launch_grad<4>(a, s);
        case 9: return launch_grad<9>(a, s);
        case 16: return launch_grad<16>(a, s);
        case 25: return launch_grad<25>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

plo_status check_config(const plo_octopt_config* c) {
    if (!c) return set_error(PLO_ERR_INVALID_ARG, "config is NULL");
    if (c->transmittance != PLO_TRANS_EXP && c->transmittance != PLO_TRANS_LINEAR)
        return set_error(PLO_ERR_INVALID_ARG, "transmittance must be PLO_TRANS_EXP or PLO_TRANS_LINEAR");
    if (c->loss < PLO_LOSS_PAPER || c->loss > PLO_LOSS_MSE) return set_error(PLO_ERR_INVALID_ARG, "unknown loss");
    if (!(c->l_max > 0.0f) || !std::isfinite(c->l_max)) return set_error(PLO_ERR_INVALID_ARG, "l_max must be finite and > 0");
    if (!(c->eps >= 0.0f) || !std::isfinite(c->eps)) return set_error(PLO_ERR_INVALID_ARG, "eps must be finite and >= 0");
    if (!(c->lr_sigma >= 0.0f) || !(c->lr_sh >= 0.0f) || !std::isfinite(c->lr_sigma) || !std::isfinite(c->lr_sh))
        return set_error(PLO_ERR_INVALID_ARG, "step sizes must be finite and >= 0");
    if (!(c->lr_decay > 0.0f && c->lr_decay <= 1.0f)) return set_error(PLO_ERR_INVALID_ARG, "lr_decay must be in (0, 1]");
    if (c->total_steps < 1) return set_error(PLO_ERR_INVALID_ARG, "total_steps must be >= 1");
    if (!(c->tv_sigma >= 0.0f) || !(c->tv_sh >= 0.0f) || !std::isfinite(c->tv_sigma) || !std::isfinite(c->tv_sh))
        return set_error(PLO_ERR_INVALID_ARG, "TV weights must be finite and >= 0");
    if (c->max_rays < 1) return set_error(PLO_ERR_INVALID_ARG, "max_rays must be >= 1");
    if (c->max_cells < 0) return set_error(PLO_ERR_INVALID_ARG, "max_cells must be >= 0");
    return PLO_OK;
}

void release(plo_octopt* o) {
    if (!o) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(o->device);
    cudaDeviceSynchronize();
    void* bufs[] = {o->d_s, o->d_k, o->d_gs, o->d_gk, o->d_ms, o->d_vs, o->d_mk, o->d_vk, o->d_nb,
                    o->d_rev_off, o->d_rev, o->d_tv_s, o->d_tv_own,
                    o->d_tr_leaf, o->d_tr_t, o->d_tr_count, o->d_acc, o->d_flags};
    for (void* b : bufs)
        if (b) cudaFree(b);
    plo_tree_free(o->walk);
    cudaSetDevice(cur);
    delete o;
}

}  // namespace
}  // namespace plo

using namespace plo;

extern "C" plo_status plo_octopt_create(const plo_tree_desc* init, const plo_octopt_config* config,
                                        plo_octopt** out) {
    if (!out) return set_error(PLO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    plo_status st = check_config(config);
    if (st != PLO_OK) return st;
    st = plo_validate_tree(init);
    if (st != PLO_OK) return st;
    if (init->n_leaves < 1) return set_error(PLO_ERR_INVALID_ARG, "the tree has no leaves");
    if (init->depth > 10) return set_error(PLO_ERR_UNSUPPORTED, "direct optimisation supports depth <= 10");
    if (init->n_leaves >= ((int64_t)1 << 31)) return set_error(PLO_ERR_UNSUPPORTED, "2^31 leaves or more");
    plo_octopt* o = nullptr;
    try {
        o = new plo_octopt;
        o->cfg = *config;
        o->depth = init->depth;
        o->sh_degree = init->sh_degree;
        o->K = sh_K(init->sh_degree);
        o->n_leaves = init->n_leaves;
        o->n_nodes = init->n_nodes;
        for (int a = 0; a < 3; ++a) {
            o->bbox_min[a] = init->bbox_min[a];
            o->bbox_max[a] = init->bbox_max[a];
        }
        const int walk_depth = init->depth > 0 ? init->depth : 1;
        o->max_cells = config->max_cells > 0 ? config->max_cells : 3 * (1 << walk_depth) + 2;
        o->child.assign(init->child, init->child + init->n_nodes * 8);
        cudaGetDevice(&o->device);

        // the structure with zero leaves: its trace crosses every cell
        {
            std::vector<float> zs((size_t)o->n_leaves, 0.0f), zk((size_t)o->n_leaves * 3, 0.0f);
            plo_tree_desc sd = *init;
            sd.sh_degree = 0;
            sd.sigma = zs.data();
            sd.sh = zk.data();
            st = plo_build_tree(&sd, PLO_PREC_FP32, &o->walk);
            if (st != PLO_OK) {
                release(o);
                return st;
            }
        }

        const int64_t nl = o->n_leaves, nk = nl * 3 * o->K;
        const int64_t cells = config->max_rays * (int64_t)o->max_cells;
        struct Buf {
            void** p;
            size_t bytes;
        } bufs[] = {{(void**)&o->d_s, (size_t)nl * 4},
                    {(void**)&o->d_k, (size_t)nk * 4},
                    {(void**)&o->d_gs, (size_t)nl * 4},
                    {(void**)&o->d_gk, (size_t)nk * 4},
                    {(void**)&o->d_ms, (size_t)nl * 4},
                    {(void**)&o->d_vs, (size_t)nl * 4},
                    {(void**)&o->d_mk, (size_t)nk * 4},
                    {(void**)&o->d_vk, (size_t)nk * 4},
                    {(void**)&o->d_nb, (size_t)nl * 12},
                    {(void**)&o->d_rev_off, (size_t)(nl + 1) * 4},
                    {(void**)&o->d_rev, (size_t)nl * 12},
                    {(void**)&o->d_tv_s, (size_t)nk * 4},
                    {(void**)&o->d_tv_own, (size_t)nk * 4},
                    {(void**)&o->d_tr_leaf, (size_t)cells * 8},
                    {(void**)&o->d_tr_t, (size_t)cells * 8},
                    {(void**)&o->d_tr_count, (size_t)config->max_rays * 4},
                    {(void**)&o->d_acc, (size_t)16},
                    {(void**)&o->d_flags, (size_t)4}};
        for (auto& b : bufs) {
            int e = dev_malloc(b.p, b.bytes);
            if (e != 0) {
                *b.p = nullptr;
                release(o);
                return cuda_error(e, "optimiser buffers");
            }
        }
        cudaError_t e = cudaMemcpy(o->d_s, init->sigma, nl * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(o->d_k, init->sh, (size_t)nk * 4, cudaMemcpyHostToDevice);
        for (float* z : {o->d_gs, o->d_ms, o->d_vs})
            if (e == cudaSuccess) e = cudaMemset(z, 0, nl * 4);
        for (float* z : {o->d_gk, o->d_mk, o->d_vk})
            if (e == cudaSuccess) e = cudaMemset(z, 0, (size_t)nk * 4);
        if (e == cudaSuccess) e = cudaMemset(o->d_acc, 0, 16);
        if (e == cudaSuccess) e = cudaMemset(o->d_flags, 0, 4);
        if (e != cudaSuccess) {
            release(o);
            return cuda_error(e, "optimiser set-up");
        }

        // face neighbours: per leaf and axis the point just across the upper
        // face at its centre, in units of 2^-(depth+1) (exact in float)
        std::vector<float> pts((size_t)nl * 9);
        const float unit = std::ldexp(1.0f, -(init->depth + 1));
        auto put = [&](int64_t leaf, const uint32_t lo[3], uint32_t size2) {
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const uint32_t v = b == a ? 2 * lo[b] + size2 + 1 : 2 * lo[b] + size2 / 2;
                    pts[(size_t)leaf * 9 + a * 3 + b] = (float)v * unit;
                }
        };
        if (init->n_nodes == 0) {
            const uint32_t z[3] = {0, 0, 0};
            put(0, z, 2u << init->depth);
        } else {
            struct Item {
                int32_t node;
                uint32_t lo[3];
                int level;
            };
            std::vector<Item> stack{{0, {0, 0, 0}, 0}};
            while (!stack.empty()) {
                Item it = stack.back();
                stack.pop_back();
                if (it.level >= init->depth) continue;  // not in a validated tree
                const uint32_t half = 1u << (init->depth - it.level - 1);  // child size in depth-grid cells
                for (int slot = 0; slot < 8; ++slot) {
                    uint32_t lo[3] = {it.lo[0] + half * (slot & 1), it.lo[1] + half * ((slot >> 1) & 1),
                                      it.lo[2] + half * ((slot >> 2) & 1)};
                    const int32_t c = init->child[(int64_t)it.node * 8 + slot];
                    if (c >= 0) stack.push_back({c, {lo[0], lo[1], lo[2]}, it.level + 1});
                    else if (c <= -2) put(-(int64_t)c - 2, lo, 2 * half);
                }
            }
        }
        float* d_pts = nullptr;
        int64_t* d_leaf = nullptr;
        int e1 = dev_malloc((void**)&d_pts, pts.size() * 4);
        int e2 = e1 == 0 ? dev_malloc((void**)&d_leaf, (size_t)nl * 3 * 8) : 0;
        st = PLO_OK;
        if (e1 != 0 || e2 != 0) {
            st = cuda_error(e1 ? e1 : e2, "neighbour lookup buffers");
        } else {
            e = cudaMemcpy(d_pts, pts.data(), pts.size() * 4, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_error(e, "neighbour points upload");
            if (st == PLO_OK) st = plo_lookup_points(o->walk, d_pts, nullptr, nl * 3, d_leaf, nullptr, nullptr);
            if (st == PLO_OK) {
                k_nb_from_lookup<<<grid_of(nl * 3, 256), 256>>>(d_leaf, nl * 3, o->d_nb);
                e = cudaDeviceSynchronize();
                if (e == cudaSuccess) e = cudaGetLastError();
                // the reverse table (counting sort of the (j, a) pairs by their neighbour)
                std::vector<int32_t> nbh((size_t)nl * 3), off((size_t)nl + 1, 0), rev;
                if (e == cudaSuccess) e = cudaMemcpy(nbh.data(), o->d_nb, (size_t)nl * 12, cudaMemcpyDeviceToHost);
                if (e == cudaSuccess) {
                    for (int32_t v : nbh)
                        if (v >= 0) ++off[(size_t)v + 1];
                    for (int64_t i = 0; i < nl; ++i) off[i + 1] += off[i];
                    rev.assign((size_t)off[nl] > 0 ? (size_t)off[nl] : 1, 0);
                    std::vector<int32_t> fill(off.begin(), off.end() - 1);
                    for (int64_t j = 0; j < nl; ++j)
                        for (int a2 = 0; a2 < 3; ++a2) {
                            const int32_t v = nbh[(size_t)j * 3 + a2];
                            if (v >= 0) rev[(size_t)fill[v]++] = (int32_t)j;
                        }
                    e = cudaMemcpy(o->d_rev_off, off.data(), ((size_t)nl + 1) * 4, cudaMemcpyHostToDevice);
                    if (e == cudaSuccess) e = cudaMemcpy(o->d_rev, rev.data(), (size_t)off[nl] * 4, cudaMemcpyHostToDevice);
                }
                if (e != cudaSuccess) st = cuda_error(e, "neighbour table");
            }
        }
        if (d_pts) cudaFree(d_pts);
        if (d_leaf) cudaFree(d_leaf);
        if (st != PLO_OK) {
            release(o);
            return st;
        }
    } catch (const std::bad_alloc&) {
        release(o);
        return set_error(PLO_ERR_OOM, "host allocation of the optimiser failed");
    }
    *out = o;
    return PLO_OK;
}

extern "C" void plo_octopt_free(plo_octopt* opt) { release(opt); }

namespace {

plo_status run_grad(plo_octopt* o, const float* d_rays, const float* d_rgb_gt, const float* d_alpha_gt, int64_t n,
                    float* d_ray_out, float* d_loss_out, void* stream) {
    if (!o) return set_error(PLO_ERR_INVALID_ARG, "optimiser is NULL");
    if (n < 0 || n > o->cfg.max_rays) return set_error(PLO_ERR_INVALID_ARG, "n must be in [0, max_rays]");
    if (n > 0 && (!d_rays || !d_rgb_gt || !d_alpha_gt))
        return set_error(PLO_ERR_INVALID_ARG, "rays, rgb_gt or alpha_gt is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nl = o->n_leaves, nk = nl * 3 * o->K;
    cudaError_t e = cudaMemsetAsync(o->d_gs, 0, (size_t)nl * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o->d_gk, 0, (size_t)nk * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o->d_acc, 0, 16, s);
    if (e != cudaSuccess) return cuda_error(e, "gradient reset");
    if (n > 0) {
        plo_render_params prm{};  // exponential, no early stop: the zero leaves never saturate
        plo_status st = plo_trace_rays(o->walk, d_rays, n, &prm, o->max_cells, o->d_tr_leaf, o->d_tr_t,
                                       o->d_tr_count, stream);
        if (st != PLO_OK) return st;
        GradArgs a{};
        a.rays = d_rays;
        a.rgb_gt = d_rgb_gt;
        a.alpha_gt = d_alpha_gt;
        a.n = n;
        a.tr_leaf = o->d_tr_leaf;
        a.tr_t = o->d_tr_t;
        a.tr_count = o->d_tr_count;
        a.max_cells = o->max_cells;
        a.s = o->d_s;
        a.k = o->d_k;
        a.gs = o->d_gs;
        a.gk = o->d_gk;
        a.ray_out = d_ray_out;
        a.acc = o->d_acc;
        a.flags = o->d_flags;
        a.transmittance = o->cfg.transmittance;
        a.loss_kind = o->cfg.loss;
        a.l_max = o->cfg.l_max;
        a.eps = o->cfg.eps;
        a.inv_n = 1.0f / (float)n;
        e = dispatch_grad(o->K, a, s);
        if (e != cudaSuccess) return cuda_error(e, "gradient kernel launch");
    }
    // the TV terms: densities (1 channel), then coefficients (3K channels);
    // the two passes share the (s, own) scratch
    const int chans[2] = {1, 3 * o->K};
    const float lam[2] = {o->cfg.tv_sigma, o->cfg.tv_sh};
    const float* xs[2] = {o->d_s, o->d_k};
    float* gs[2] = {o->d_gs, o->d_gk};
    for (int q = 0; q < 2; ++q) {
        if (!(lam[q] > 0.0f)) continue;
        const unsigned blocks = grid_of(nl * chans[q], THREADS);
        const unsigned terms_blocks = std::min<unsigned>(blocks, 8u * 152u);
        k_tv_terms<<<terms_blocks, THREADS, 0, s>>>(xs[q], chans[q], o->d_nb, nl, o->d_tv_s, o->d_tv_own,
                                                    o->d_acc + 1 + q);
        k_tv_grad<<<blocks, THREADS, 0, s>>>(xs[q], chans[q], o->d_rev_off, o->d_rev, nl, o->d_tv_s, o->d_tv_own,
                                             lam[q] / (float)nl, gs[q]);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "TV kernel launch");
    if (d_loss_out) {
        e = cudaMemcpyAsync(d_loss_out, o->d_acc, 3 * sizeof(float), cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_error(e, "loss copy");
    }
    return PLO_OK;
}

// Elements and element size of a PLO_OCTOPT_* array; NULL pointer if unknown.
void* octopt_array(const plo_octopt* o, int32_t what, size_t* bytes) {
    const size_t nl = (size_t)o->n_leaves, nk = nl * 3 * (size_t)o->K;
    switch (what) {
        case PLO_OCTOPT_SIGMA: *bytes = nl * 4; return o->d_s;
        case PLO_OCTOPT_SH: *bytes = nk * 4; return o->d_k;
        case PLO_OCTOPT_GRAD_SIGMA: *bytes = nl * 4; return o->d_gs;
        case PLO_OCTOPT_GRAD_SH: *bytes = nk * 4; return o->d_gk;
        case PLO_OCTOPT_NEIGHBOURS: *bytes = nl * 12; return o->d_nb;
        default: *bytes = 0; return nullptr;
    }
}

}  // namespace

extern "C" plo_status plo_octopt_grad(plo_octopt* opt, const float* d_rays, const float* d_rgb_gt,
                                      const float* d_alpha_gt, int64_t n, float* d_ray_out, float* d_loss_out,
                                      void* stream) {
    return run_grad(opt, d_rays, d_rgb_gt, d_alpha_gt, n, d_ray_out, d_loss_out, stream);
}

extern "C" plo_status plo_octopt_step(plo_octopt* opt, const float* d_rays, const float* d_rgb_gt,
                                      const float* d_alpha_gt, int64_t n, float* d_ray_out, float* d_loss_out,
                                      void* stream) {
    if (opt && n == 0) return PLO_OK;
    plo_status st = run_grad(opt, d_rays, d_rgb_gt, d_alpha_gt, n, d_ray_out, d_loss_out, stream);
    if (st != PLO_OK) return st;
    const int64_t t = ++opt->step;
    const double f = std::pow((double)opt->cfg.lr_decay,
                              (double)std::min<int64_t>(t - 1, opt->cfg.total_steps) / opt->cfg.total_steps);
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)t)), bc2 = (float)(1.0 - std::pow(0.999, (double)t));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nl = opt->n_leaves, nk = nl * 3 * opt->K;
    const unsigned gs = std::min<unsigned>(grid_of(nl, 256), 4096u), gk = std::min<unsigned>(grid_of(nk, 256), 4096u);
    k_adam<<<gs, 256, 0, s>>>(opt->d_s, opt->d_gs, opt->d_ms, opt->d_vs, nl, (float)(opt->cfg.lr_sigma * f), bc1, bc2);
    k_adam<<<gk, 256, 0, s>>>(opt->d_k, opt->d_gk, opt->d_mk, opt->d_vk, nk, (float)(opt->cfg.lr_sh * f), bc1, bc2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "Adam kernel launch");
    return PLO_OK;
}

extern "C" plo_status plo_octopt_read(const plo_octopt* opt, int32_t what, void* dst, void* stream) {
    if (!opt || !dst) return set_error(PLO_ERR_INVALID_ARG, "optimiser or dst is NULL");
    size_t bytes = 0;
    void* src = octopt_array(opt, what, &bytes);
    if (!src) return set_error(PLO_ERR_INVALID_ARG, "unknown array");
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, (cudaStream_t)stream);
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "optimiser read");
}

extern "C" plo_status plo_octopt_write(plo_octopt* opt, int32_t what, const void* src, void* stream) {
    if (!opt || !src) return set_error(PLO_ERR_INVALID_ARG, "optimiser or src is NULL");
    if (what != PLO_OCTOPT_SIGMA && what != PLO_OCTOPT_SH)
        return set_error(PLO_ERR_INVALID_ARG, "only PLO_OCTOPT_SIGMA and PLO_OCTOPT_SH can be written");
    size_t bytes = 0;
    void* dst = octopt_array(opt, what, &bytes);
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, (cudaStream_t)stream);
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "optimiser write");
}

extern "C" plo_status plo_octopt_check(plo_octopt* opt, void* stream) {
    if (!opt) return set_error(PLO_ERR_INVALID_ARG, "optimiser is NULL");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    unsigned int flags = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flags, opt->d_flags, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flags) e = cudaMemset(opt->d_flags, 0, 4);
    if (e != cudaSuccess) return cuda_error(e, "optimiser check");
    if (flags & 1u)
        return set_error(PLO_ERR_TRAVERSAL_LIMIT, "a ray crossed more than max_cells cells and was left out");
    return PLO_OK;
}

extern "C" plo_status plo_octopt_build_tree(const plo_octopt* opt, const plo_build_options* options, plo_tree** out) {
    if (!opt || !options || !out) return set_error(PLO_ERR_INVALID_ARG, "optimiser, options or out is NULL");
    *out = nullptr;
    try {
        const size_t nl = (size_t)opt->n_leaves, nk = nl * 3 * (size_t)opt->K;
        std::vector<float> sig(nl), sh(nk);
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(sig.data(), opt->d_s, nl * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(sh.data(), opt->d_k, nk * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_error(e, "optimiser download");
        for (float& v : sig) v = v > 0.0f ? v : 0.0f;  // NaN stays NaN and fails validation
        plo_tree_desc d{};
        d.depth = opt->depth;
        d.sh_degree = opt->sh_degree;
        d.n_nodes = opt->n_nodes;
        d.n_leaves = opt->n_leaves;
        d.child = opt->child.data();
        d.sigma = sig.data();
        d.sh = sh.data();
        for (int a = 0; a < 3; ++a) {
            d.bbox_min[a] = opt->bbox_min[a];
            d.bbox_max[a] = opt->bbox_max[a];
        }
        return plo_build_tree_ex(&d, options, out);
    } catch (const std::bad_alloc&) {
        return set_error(PLO_ERR_OOM, "host allocation while packing the optimised tree failed");
    }
}
