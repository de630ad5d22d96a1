// Device-side packing of an octree whose leaves are voxels of one level
// (the distilled plenoctree of Sec. 5, "Creating the plenoctree"), and the
// export of any packed tree back to the canonical host format.
//
// Input: the kept voxels' Morton codes at depth D, sorted (the order the
// distillation visits voxels in), with each leaf's entry word (sigma, and
// the SH scale for 16-bit records) and its packed SH record.  Output: the
// octree layout of plo_internal.h, identical to what plo_build_tree makes of
// the same canonical tree, except that every leaf has a record slot (record
// id = leaf id; leaves whose coefficients are all zero are marked as not
// emitting, as the host packer marks them).
//
// Nodes are the distinct prefixes code >> 3(D - L) of the codes at each
// level L < D (sorted, since the codes are).  Node ids: levels below
// T = min(4, D) in breadth-first order, then the deeper levels in
// depth-first pre-order, i.e. sorted by (first finest cell, level); a node's
// pre-order rank is the number of nodes of every level whose first cell
// comes earlier (a binary search per level), plus its ancestors that start
// at the same cell.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "plo_internal.h"

namespace plo {
namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Exclusive scan of one tile of SCAN_TILE values per block; the block's
// total goes to sums[block].
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile(const uint32_t* in, uint32_t* out, int64_t n,
                                                            uint32_t* sums) {
    __shared__ uint32_t s_warp[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t local = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        local += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SCAN_THREADS / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < SCAN_THREADS / 32) s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t run = incl - local + (warp > 0 ? s_warp[warp - 1] : 0u);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_THREADS - 1) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(uint32_t* out, int64_t n, const uint32_t* offsets) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offsets[i / SCAN_TILE];
}

// flag[i] = 1 where a[i] >> shift starts a new run of equal prefixes
__global__ void k_flag_new_prefix(const uint32_t* a, int64_t n, int shift, uint32_t* flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (i == 0 || (a[i] >> shift) != (a[i - 1] >> shift)) ? 1u : 0u;
}

__global__ void k_scatter_prefix(const uint32_t* a, const uint32_t* flag, const uint32_t* pos, int64_t n, int shift,
                                 uint32_t* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = a[i] >> shift;
}

struct Levels {
    const uint32_t* pref[MAX_DEPTH + 1];  // level L < D: node prefixes; level D: the leaves' codes
    int64_t n[MAX_DEPTH + 1];
    uint32_t* id[MAX_DEPTH];              // packed node id of each node of level L < D
    int D, T;
    int64_t n_top;                        // nodes of the levels below T
};

// first index k in [0, n) with a[k] >= key (a sorted), n if none
__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t* a, int64_t n, uint32_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Node ids of level L: breadth-first below T, pre-order rank above.
__global__ void k_node_ids(Levels lv, int L, int64_t level_offset) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= lv.n[L]) return;
    if (L < lv.T) {
        lv.id[L][j] = (uint32_t)(level_offset + j);
        return;
    }
    const uint32_t p = __ldg(lv.pref[L] + j);
    int64_t pre = 0;
    for (int l = lv.T; l < lv.D; ++l) {
        uint32_t key;
        if (l <= L) {
            const int k = 3 * (L - l);
            key = (uint32_t)(((uint64_t)p + ((1ull << k) - 1)) >> k);  // ceil(p / 8^(L-l))
            if (l < L && (p & ((1u << k) - 1u)) == 0u) ++pre;         // an ancestor starting at the same cell
        } else {
            key = p << (3 * (l - L));
        }
        pre += lower_bound_u32(lv.pref[l], lv.n[l], key);
    }
    lv.id[L][j] = (uint32_t)(lv.n_top + pre);
}

// The eight entries (and canonical leaf ids) of every node of level L.
__global__ void k_node_entries(Levels lv, int L, const uint32_t* yword, const uint8_t* emits, uint2* nodes,
                               int32_t* leaf_ids) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= lv.n[L]) return;
    const uint32_t p = __ldg(lv.pref[L] + j);
    const uint32_t id = lv.id[L][j];
    uint2 e[8];
    int32_t lid[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        e[s] = make_uint2(ENTRY_EMPTY, 0u);
        lid[s] = -1;
    }
    const bool leaves = L + 1 == lv.D;
    const uint32_t* A = lv.pref[L + 1];
    const int64_t nA = lv.n[L + 1];
    for (int64_t k = lower_bound_u32(A, nA, p << 3); k < nA; ++k) {
        const uint32_t c = __ldg(A + k);
        if ((c >> 3) != p) break;
        const int s = (int)(c & 7u);
        if (leaves) {
            e[s] = make_uint2(LEAF_BIT | (emits[k] ? (uint32_t)k : NO_SH_RECORD), yword[k]);
            lid[s] = (int32_t)k;
        } else {
            e[s] = make_uint2(lv.id[L + 1][k], 0u);
        }
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        nodes[(size_t)id * 8 + s] = e[s];
        leaf_ids[(size_t)id * 8 + s] = lid[s];
    }
}

unsigned blocks_of(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t device_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t* sums = nullptr;
    cudaError_t e = (cudaError_t)dev_malloc_async((void**)&sums, (size_t)nb * 4, s);
    if (e != cudaSuccess) return e;
    k_scan_tile<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    e = cudaGetLastError();
    if (e == cudaSuccess && nb > 1) {
        e = device_exclusive_scan(sums, sums, nb, s);
        if (e == cudaSuccess) {
            k_scan_add<<<blocks_of(n), 256, 0, s>>>(out, n, sums);
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(sums, s);
    return e;
}

plo_status pack_voxel_tree(int depth, int sh_degree, int precision, const uint32_t* d_codes, int64_t nl,
                           uint32_t* d_yword, uint8_t* d_emits, void* d_records, cudaStream_t s, plo_tree** out) {
    *out = nullptr;
    const int D = depth, T = std::min(4, depth);
    const int K = sh_K(sh_degree);
    Levels lv{};
    lv.D = D;
    lv.T = T;
    lv.pref[D] = d_codes;
    lv.n[D] = nl;
    std::vector<void*> owned;
    auto alloc = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t e = (cudaError_t)dev_malloc(p, bytes > 0 ? bytes : 4);
        if (e == cudaSuccess) owned.push_back(*p);
        return e;
    };
    auto release = [&]() {
        cudaStreamSynchronize(s);
        for (void* p : owned) cudaFree(p);
        owned.clear();
    };
    cudaError_t e = cudaSuccess;
    uint32_t *flag = nullptr, *pos = nullptr;
    if (nl > 0) {
        e = alloc((void**)&flag, (size_t)nl * 4);
        if (e == cudaSuccess) e = alloc((void**)&pos, (size_t)nl * 4);
    }
    // distinct prefixes, level by level upwards (each from the level below)
    for (int L = D - 1; L >= 0 && e == cudaSuccess; --L) {
        const uint32_t* below = lv.pref[L + 1];
        const int64_t nb = lv.n[L + 1];
        uint32_t* pref = nullptr;
        if (nb == 0) {  // empty tree: the root alone
            lv.n[L] = L == 0 ? 1 : 0;
            e = alloc((void**)&pref, 4);
            if (e == cudaSuccess) e = cudaMemsetAsync(pref, 0, 4, s);
            lv.pref[L] = pref;
            continue;
        }
        k_flag_new_prefix<<<blocks_of(nb), 256, 0, s>>>(below, nb, 3, flag);
        e = device_exclusive_scan(flag, pos, nb, s);
        uint32_t last_pos = 0, last_flag = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&last_pos, pos + nb - 1, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&last_flag, flag + nb - 1, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        lv.n[L] = (int64_t)last_pos + last_flag;
        e = alloc((void**)&pref, (size_t)lv.n[L] * 4);
        if (e != cudaSuccess) break;
        k_scatter_prefix<<<blocks_of(nb), 256, 0, s>>>(below, flag, pos, nb, 3, pref);
        lv.pref[L] = pref;
        e = cudaGetLastError();
    }
    int64_t n_nodes = 0;
    for (int L = 0; L < D; ++L) {
        if (L < T) lv.n_top += lv.n[L];
        n_nodes += lv.n[L];
    }
    if (e == cudaSuccess && n_nodes >= (int64_t)LEAF_BIT - 1) {
        release();
        return set_error(PLO_ERR_UNSUPPORTED, "too many nodes for the packed layout (>= 2^31 - 1)");
    }
    for (int L = 0; L < D && e == cudaSuccess; ++L) e = alloc((void**)&lv.id[L], (size_t)lv.n[L] * 4);
    plo_tree* t = nullptr;
    if (e == cudaSuccess) {
        int64_t off = 0;
        for (int L = 0; L < D && e == cudaSuccess; ++L) {
            if (lv.n[L] > 0) k_node_ids<<<blocks_of(lv.n[L]), 256, 0, s>>>(lv, L, off);
            if (L < T) off += lv.n[L];
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        t = new (std::nothrow) plo_tree();
        if (!t) {
            release();
            return set_error(PLO_ERR_OOM, "host allocation failed");
        }
        e = (cudaError_t)dev_malloc(&t->d_nodes, (size_t)n_nodes * 64);
        if (e == cudaSuccess) e = (cudaError_t)dev_malloc((void**)&t->d_leaf_ids, (size_t)n_nodes * 32);
        if (e == cudaSuccess) e = (cudaError_t)dev_malloc((void**)&t->d_flags, 256);
        if (e == cudaSuccess) e = cudaMemsetAsync(t->d_flags, 0, 256, s);
    }
    for (int L = 0; L < D && e == cudaSuccess; ++L) {
        if (lv.n[L] > 0)
            k_node_entries<<<blocks_of(lv.n[L]), 256, 0, s>>>(lv, L, d_yword, d_emits, static_cast<uint2*>(t->d_nodes),
                                                              t->d_leaf_ids);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release();
    if (e != cudaSuccess) {
        if (t) {
            t->d_sh = nullptr;  // the caller keeps the records on failure
            plo_tree_free(t);
        }
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? set_error(PLO_ERR_OOM, "device allocation while packing failed")
                                              : cuda_error(e, "device packing of the distilled tree");
    }
    t->depth = D;
    t->sh_degree = sh_degree;
    t->K = K;
    t->precision = precision;
    t->top_levels = T;
    t->n_top = (int32_t)lv.n_top;
    t->n_nodes = n_nodes;
    t->n_leaves = nl;
    t->n_sh = nl;
    t->sh_stride = sh_stride_bytes(K, precision);
    for (int a = 0; a < 3; ++a) {
        t->bbox_min[a] = 0.0f;
        t->inv_ext[a] = 1.0f;
        t->inv_ext_lo[a] = 0.0f;
    }
    t->d_sh = d_records;
    t->node_bytes = n_nodes * 64;
    t->sh_bytes = nl * (int64_t)t->sh_stride;
    t->layout = PLO_LAYOUT_OCTREE;
    t->brick_level = D;
    cudaGetDevice(&t->device);
    cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, t->device);
    *out = t;
    return PLO_OK;
}

}  // namespace plo

using namespace plo;

// Canonical export: the packed octree read back and decoded on the host.
extern "C" plo_status plo_tree_export(const plo_tree* t, int32_t* h_child, float* h_sigma, float* h_sh) {
    if (!t) return set_error(PLO_ERR_INVALID_ARG, "tree is NULL");
    if (!h_child || !h_sigma || !h_sh) return set_error(PLO_ERR_INVALID_ARG, "an output is NULL");
    try {
        const int64_t nn = t->n_nodes;
        std::vector<uint32_t> nodes((size_t)nn * 16);
        std::vector<int32_t> ids((size_t)nn * 8);
        const int64_t rec_bytes = std::max<int64_t>(t->sh_bytes, 1);
        std::vector<uint8_t> rec((size_t)rec_bytes);
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(nodes.data(), t->d_nodes, (size_t)nn * 64, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(ids.data(), t->d_leaf_ids, (size_t)nn * 32, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && t->sh_bytes > 0)
            e = cudaMemcpy(rec.data(), t->d_sh, (size_t)t->sh_bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_error(e, "plo_tree_export");
        const int K = t->K;
        for (int64_t i = 0; i < nn; ++i)
            for (int s = 0; s < 8; ++s) {
                const uint32_t x = nodes[(size_t)i * 16 + 2 * s], y = nodes[(size_t)i * 16 + 2 * s + 1];
                int32_t c = -1;
                if (x != ENTRY_EMPTY && !(x & LEAF_BIT)) {
                    c = (int32_t)x;
                } else if (x != ENTRY_EMPTY) {
                    const int32_t leaf = ids[(size_t)i * 8 + s];
                    if (leaf < 0 || leaf >= t->n_leaves) return set_error(PLO_ERR_BAD_TREE, "leaf id out of range");
                    c = -leaf - 2;
                    float sig;
                    if (t->precision == PLO_PREC_FP32) {
                        std::memcpy(&sig, &y, 4);
                    } else {
                        const uint32_t b = (y & 0xFFFFFFu) << 7;
                        std::memcpy(&sig, &b, 4);
                    }
                    h_sigma[leaf] = sig;
                    float* dst = h_sh + (size_t)leaf * 3 * K;
                    const uint32_t r = x & ~LEAF_BIT;
                    for (int k = 0; k < 3 * K; ++k) dst[k] = 0.0f;
                    if (r != NO_SH_RECORD) {
                        const uint8_t* src = rec.data() + (size_t)r * t->sh_stride;
                        if (t->precision == PLO_PREC_FP32) {
                            std::memcpy(dst, src, sizeof(float) * 3 * K);
                        } else {
                            const float scale = std::ldexp(1.0f, (int)(y >> 24) - 127);
                            for (int k = 0; k < 3 * K; ++k) {
                                uint16_t h;
                                std::memcpy(&h, src + 2 * k, 2);
                                float f;
                                if (t->precision == PLO_PREC_FP16) {
                                    __half_raw hr;
                                    hr.x = h;
                                    f = __half2float(__half(hr));
                                } else {
                                    const uint32_t b = (uint32_t)h << 16;
                                    std::memcpy(&f, &b, 4);
                                }
                                dst[k] = f * scale;
                            }
                        }
                    }
                }
                h_child[(size_t)i * 8 + s] = c;
            }
        return PLO_OK;
    } catch (const std::bad_alloc&) {
        return set_error(PLO_ERR_OOM, "host allocation while exporting the tree failed");
    }
}
