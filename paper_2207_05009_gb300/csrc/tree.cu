// plo_validate_tree / plo_build_tree / plo_tree_free / plo_tree_get_info /
// plo_tree_check: validation of the canonical plenoctree (Sec. 5) and its
// packing into the device layout described in plo_internal.h.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "plo_internal.h"

using namespace plo;

namespace {

// f(begin, end) over [0, n) in contiguous ranges on the host's cores; the
// per-leaf passes below (checks, emission flags, record packing) touch each
// leaf's own data only, so the result does not depend on the split.
template <class F>
void parallel_ranges(int64_t n, F f) {
    const int64_t min_per_thread = 1 << 16;
    int threads = (int)std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()), 32);
    threads = (int)std::min<int64_t>(threads, (n + min_per_thread - 1) / min_per_thread);
    if (threads <= 1) {
        f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> pool;
    const int64_t per = (n + threads - 1) / threads;
    for (int t = 0; t < threads; ++t) {
        const int64_t b = t * per, e = std::min(n, b + per);
        if (b < e) pool.emplace_back(f, b, e);
    }
    for (auto& th : pool) th.join();
}

plo_status validate(const plo_tree_desc* t) {
    if (!t) return set_error(PLO_ERR_INVALID_ARG, "tree descriptor is NULL");
    if (t->depth < 0 || t->depth > MAX_DEPTH)
        return set_error(PLO_ERR_INVALID_ARG, "depth must be in [0, 16], got " + std::to_string(t->depth));
    if (t->sh_degree < 0 || t->sh_degree > 4)
        return set_error(PLO_ERR_INVALID_ARG, "sh_degree must be in [0, 4], got " + std::to_string(t->sh_degree));
    if (t->n_nodes < 0 || t->n_leaves < 0) return set_error(PLO_ERR_INVALID_ARG, "negative node or leaf count");
    if (t->n_nodes >= (int64_t)LEAF_BIT - 1) return set_error(PLO_ERR_INVALID_ARG, "too many nodes (>= 2^31 - 1)");
    if (t->n_leaves >= (int64_t)NO_SH_RECORD) return set_error(PLO_ERR_INVALID_ARG, "too many leaves");
    if (t->n_nodes > 0 && !t->child) return set_error(PLO_ERR_INVALID_ARG, "child table is NULL");
    if (t->n_leaves > 0 && (!t->sigma || !t->sh)) return set_error(PLO_ERR_INVALID_ARG, "sigma or sh is NULL");
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(t->bbox_min[a]) || !std::isfinite(t->bbox_max[a]) || !(t->bbox_max[a] > t->bbox_min[a]))
            return set_error(PLO_ERR_INVALID_ARG, "bounding box must be finite with max > min on every axis");
    }
    if (t->n_nodes == 0) {
        if (t->n_leaves > 1)
            return set_error(PLO_ERR_BAD_TREE, "a tree without nodes holds at most one leaf (the root)");
    } else {
        if (t->depth < 1) return set_error(PLO_ERR_BAD_TREE, "a tree with nodes needs depth >= 1");
        std::vector<uint8_t> seen_node(t->n_nodes, 0), seen_leaf(t->n_leaves, 0);
        std::vector<std::pair<int64_t, int>> stack;
        stack.push_back({0, 0});
        seen_node[0] = 1;
        while (!stack.empty()) {
            auto [nid, lev] = stack.back();
            stack.pop_back();
            for (int s = 0; s < 8; ++s) {
                int32_t e = t->child[nid * 8 + s];
                if (e >= 0) {
                    if (e >= t->n_nodes)
                        return set_error(PLO_ERR_BAD_TREE, "node " + std::to_string(nid) + " slot " +
                                                               std::to_string(s) + ": child index out of range");
                    if (lev + 1 >= t->depth)
                        return set_error(PLO_ERR_BAD_TREE, "node " + std::to_string(e) + " sits at level " +
                                                               std::to_string(lev + 1) +
                                                               ", its children would exceed depth " +
                                                               std::to_string(t->depth));
                    if (seen_node[e])
                        return set_error(PLO_ERR_BAD_TREE, "node " + std::to_string(e) +
                                                               " is referenced twice (cycle or shared subtree)");
                    seen_node[e] = 1;
                    stack.push_back({e, lev + 1});
                } else if (e <= -2) {
                    int64_t leaf = -(int64_t)e - 2;
                    if (leaf >= t->n_leaves)
                        return set_error(PLO_ERR_BAD_TREE, "leaf index " + std::to_string(leaf) + " out of range");
                    if (seen_leaf[leaf])
                        return set_error(PLO_ERR_BAD_TREE, "leaf " + std::to_string(leaf) + " is referenced twice");
                    seen_leaf[leaf] = 1;
                }
            }
        }
    }
    const int K = sh_K(t->sh_degree);
    // the first offending leaf of each kind is reported, whatever the split
    std::atomic<int64_t> bad_sigma{INT64_MAX}, bad_sh{INT64_MAX};
    parallel_ranges(t->n_leaves, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i) {
            const float s = t->sigma[i];
            if (!std::isfinite(s) || s < 0.0f) {
                int64_t cur = bad_sigma.load();
                while (i < cur && !bad_sigma.compare_exchange_weak(cur, i)) {
                }
                break;
            }
        }
        for (int64_t i = b * 3 * K; i < e * 3 * K; ++i) {
            if (!std::isfinite(t->sh[i])) {
                const int64_t leaf = i / (3 * K);
                int64_t cur = bad_sh.load();
                while (leaf < cur && !bad_sh.compare_exchange_weak(cur, leaf)) {
                }
                break;
            }
        }
    });
    if (bad_sigma.load() != INT64_MAX)
        return set_error(PLO_ERR_BAD_TREE,
                         "sigma of leaf " + std::to_string(bad_sigma.load()) + " is negative or not finite");
    if (bad_sh.load() != INT64_MAX)
        return set_error(PLO_ERR_BAD_TREE, "SH coefficient of leaf " + std::to_string(bad_sh.load()) +
                                               " is not finite");
    return PLO_OK;
}

uint16_t half_bits(float v) {
    __half h = __float2half_rn(v);
    uint16_t b;
    std::memcpy(&b, &h, 2);
    return b;
}
uint16_t bf16_bits(float v) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    uint16_t b;
    std::memcpy(&b, &h, 2);
    return b;
}
// sigma >= 0 as a 24-bit float: FP32 without its sign bit, mantissa rounded
// to nearest-even at 16 bits (relative error <= 2^-17).
uint32_t sigma24_bits(float v) {
    uint32_t b;
    std::memcpy(&b, &v, 4);
    b &= 0x7FFFFFFFu;
    uint32_t r = (b + 0x3Fu + ((b >> 7) & 1u)) >> 7;
    if (r >= 0xFF0000u) r = 0xFEFFFFu;  // keep it finite (exponent 255 would be inf)
    return r;
}

}  // namespace

// Validation allocates per-node and per-leaf flags sized by the descriptor's
// counts; a descriptor with huge counts gets PLO_ERR_OOM, not an exception.
extern "C" plo_status plo_validate_tree(const plo_tree_desc* desc) {
    try {
        return validate(desc);
    } catch (const std::bad_alloc&) {
        return set_error(PLO_ERR_OOM, "host allocation while validating the tree failed");
    }
}

namespace {
// Bit i of x goes to bit 3 i (x < 8): the Morton interleave of brick-local
// coordinates, x lowest.
inline uint32_t spread3(uint32_t x) { return (x & 1u) | ((x & 2u) << 2) | ((x & 4u) << 4); }

plo_status build_tree(const plo_tree_desc* desc, const plo_build_options* opt, plo_tree** out) {
    if (!out) return set_error(PLO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!opt) return set_error(PLO_ERR_INVALID_ARG, "options are NULL");
    const int32_t precision = opt->precision;
    if (precision < PLO_PREC_FP32 || precision > PLO_PREC_BF16)
        return set_error(PLO_ERR_INVALID_ARG, "precision must be PLO_PREC_FP32, _FP16 or _BF16");
    if (opt->layout != PLO_LAYOUT_OCTREE && opt->layout != PLO_LAYOUT_BRICKS)
        return set_error(PLO_ERR_INVALID_ARG, "layout must be PLO_LAYOUT_OCTREE or PLO_LAYOUT_BRICKS");
    if (opt->brick_log != 0 && (opt->brick_log < 1 || opt->brick_log > 3))
        return set_error(PLO_ERR_INVALID_ARG, "brick_log must be 0 (default), 1, 2 or 3");
    plo_status st = validate(desc);
    if (st != PLO_OK) return st;
    const int K = sh_K(desc->sh_degree);

    // Canonical child table; a tree without nodes is re-rooted one level down
    // (eight slots that all hold the root leaf, or all empty).
    std::vector<int32_t> synth;
    const int32_t* child = desc->child;
    int64_t n_nodes = desc->n_nodes;
    int depth = desc->depth;
    if (n_nodes == 0) {
        synth.assign(8, desc->n_leaves == 1 ? -2 : -1);
        child = synth.data();
        n_nodes = 1;
        depth = 1;
    }

    // Levels by breadth-first search; the first `top` levels keep BFS order.
    std::vector<int32_t> bfs;
    std::vector<int8_t> level(n_nodes, -1);
    bfs.reserve(n_nodes);
    bfs.push_back(0);
    level[0] = 0;
    for (size_t i = 0; i < bfs.size(); ++i) {
        int32_t nid = bfs[i];
        for (int s = 0; s < 8; ++s) {
            int32_t e = child[(int64_t)nid * 8 + s];
            if (e >= 0) {
                level[e] = level[nid] + 1;
                bfs.push_back(e);
            }
        }
    }
    const int top = depth < 4 ? depth : 4;
    std::vector<int32_t> order;  // new id -> canonical id
    order.reserve(bfs.size());
    std::vector<int32_t> new_id(n_nodes, -1);
    for (int32_t nid : bfs)
        if (level[nid] < top) {
            new_id[nid] = (int32_t)order.size();
            order.push_back(nid);
        }
    const int32_t n_top = (int32_t)order.size();
    // depth-first pre-order of the subtrees below the top levels
    std::vector<int32_t> stack;
    for (int32_t nid : bfs) {
        if (level[nid] != top) continue;
        stack.push_back(nid);
        while (!stack.empty()) {
            int32_t v = stack.back();
            stack.pop_back();
            new_id[v] = (int32_t)order.size();
            order.push_back(v);
            for (int s = 7; s >= 0; --s) {
                int32_t e = child[(int64_t)v * 8 + s];
                if (e >= 0) stack.push_back(e);
            }
        }
    }
    const int64_t n_packed = (int64_t)order.size();

    // SH records in depth-first (Morton) order of the leaves.
    std::vector<uint32_t> rec_of_leaf(desc->n_leaves > 0 ? desc->n_leaves : 1, NO_SH_RECORD);
    std::vector<uint8_t> emits_of_leaf(desc->n_leaves > 0 ? desc->n_leaves : 1, 0);
    parallel_ranges(desc->n_leaves, [&](int64_t b, int64_t e) {
        for (int64_t leaf = b; leaf < e; ++leaf) {
            const float* c = desc->sh + leaf * 3 * K;
            bool emits = false;
            for (int k = 0; k < 3 * K; ++k) emits |= c[k] != 0.0f;
            emits_of_leaf[leaf] = emits ? 1 : 0;
        }
    });
    int64_t n_sh = 0;
    {
        std::vector<int32_t> st{0};
        while (!st.empty()) {
            int32_t v = st.back();
            st.pop_back();
            for (int s = 7; s >= 0; --s) {
                int32_t e = child[(int64_t)v * 8 + s];
                if (e >= 0) st.push_back(e);
            }
            for (int s = 0; s < 8; ++s) {
                int32_t e = child[(int64_t)v * 8 + s];
                if (e <= -2) {
                    int64_t leaf = -(int64_t)e - 2;
                    if (rec_of_leaf[leaf] != NO_SH_RECORD) continue;  // root leaf repeated in 8 slots
                    if (emits_of_leaf[leaf]) rec_of_leaf[leaf] = (uint32_t)n_sh++;
                }
            }
        }
    }
    // Note: the depth-first walk above visits a node's leaves after pushing its
    // children, so records follow pre-order of nodes; within a node, slot order.

    const int stride = sh_stride_bytes(K, precision);
    std::vector<uint32_t> nodes;
    std::vector<int32_t> leaf_ids;
    // every record is written whole (coefficients and zero padding) below,
    // so the buffer is not cleared first
    std::unique_ptr<uint8_t[]> sh;
    try {
        nodes.assign(n_packed * 16, 0);
        leaf_ids.assign(n_packed * 8, -1);
        sh.reset(new uint8_t[(size_t)(n_sh > 0 ? n_sh : 1) * stride]);
        if (n_sh == 0) std::memset(sh.get(), 0, (size_t)stride);
    } catch (const std::bad_alloc&) {
        return set_error(PLO_ERR_OOM, "host allocation for the packed tree failed");
    }
    std::vector<int8_t> scale_exp(desc->n_leaves > 0 ? desc->n_leaves : 1, 0);
    parallel_ranges(desc->n_leaves, [&](int64_t lb, int64_t le) {
        for (int64_t leaf = lb; leaf < le; ++leaf) {
            uint32_t r = rec_of_leaf[leaf];
            if (r == NO_SH_RECORD) continue;
            const float* c = desc->sh + leaf * 3 * K;
            uint8_t* dst = sh.get() + (size_t)r * stride;
            if (precision == PLO_PREC_FP32) {
                std::memcpy(dst, c, sizeof(float) * 3 * K);
                std::memset(dst + sizeof(float) * 3 * K, 0, (size_t)stride - sizeof(float) * 3 * K);
                continue;
            }
            float m = 0.0f;
            for (int k = 0; k < 3 * K; ++k) m = std::fmax(m, std::fabs(c[k]));
            int e;
            std::frexp(m, &e);  // m = f * 2^e, f in [0.5, 1)
            // FP16: map the largest coefficient into [2^14, 2^15) so that the
            // leaf's smaller coefficients keep binary16's normal range (down to
            // 2^-29 of the largest); BF16 has FP32's range and uses [0.5, 1).
            if (precision == PLO_PREC_FP16) e -= 15;
            if (e < -126) e = -126;
            if (e > 127) e = 127;
            float inv = std::ldexp(1.0f, -e);
            uint16_t* h = reinterpret_cast<uint16_t*>(dst);
            for (int k = 0; k < 3 * K; ++k) {
                float v = c[k] * inv;
                h[k] = precision == PLO_PREC_FP16 ? half_bits(v) : bf16_bits(v);
            }
            std::memset(dst + 2 * 3 * K, 0, (size_t)stride - 2 * 3 * K);
            scale_exp[leaf] = (int8_t)e;
        }
    });
    for (int64_t i = 0; i < n_packed; ++i) {
        int32_t v = order[i];
        for (int s = 0; s < 8; ++s) {
            int32_t e = child[(int64_t)v * 8 + s];
            uint32_t x = ENTRY_EMPTY, y = 0;
            if (e >= 0) {
                x = (uint32_t)new_id[e];
            } else if (e <= -2) {
                int64_t leaf = -(int64_t)e - 2;
                leaf_ids[i * 8 + s] = (int32_t)leaf;
                x = LEAF_BIT | rec_of_leaf[leaf];
                float sg = desc->sigma[leaf];
                if (precision == PLO_PREC_FP32) {
                    std::memcpy(&y, &sg, 4);
                } else {
                    uint32_t eb = rec_of_leaf[leaf] == NO_SH_RECORD ? 0u : (uint32_t)(scale_exp[leaf] + 127);
                    y = sigma24_bits(sg) | (eb << 24);
                }
            }
            nodes[i * 16 + 2 * s] = x;
            nodes[i * 16 + 2 * s + 1] = y;
        }
    }

    // Brick layout: the octree above level B = depth - s (top nodes keep the
    // packed order; a child at level B that has children is a brick), and
    // below it one dense (2^s)^3 array of cell entries per brick, in Morton
    // order, each finest cell holding the entry of the leaf that covers it.
    const bool bricks = opt->layout == PLO_LAYOUT_BRICKS;
    const int blog = bricks ? std::min(opt->brick_log > 0 ? opt->brick_log : 3, depth - 1) : 0;
    const int B = depth - blog;
    std::vector<uint32_t> top_tab;
    std::vector<uint32_t> brick_cells;
    int64_t n_top_nodes = 0, n_bricks = 0;
    int32_t n_top_staged = 0;
    if (bricks) {
        std::vector<int32_t> top_id(n_nodes, -1), brick_id(n_nodes, -1), top_order, brick_nodes;
        for (int32_t v : order) {
            if (level[v] < B) {
                top_id[v] = (int32_t)top_order.size();
                top_order.push_back(v);
                if (level[v] < std::min(top, B)) ++n_top_staged;
            } else if (level[v] == B) {
                brick_id[v] = (int32_t)brick_nodes.size();
                brick_nodes.push_back(v);
            }
        }
        n_top_nodes = (int64_t)top_order.size();
        n_bricks = (int64_t)brick_nodes.size();
        top_tab.assign(n_top_nodes * 16, 0);
        for (int64_t i = 0; i < n_top_nodes; ++i) {
            const int32_t v = top_order[i];
            const int64_t src = (int64_t)new_id[v] * 16;
            for (int sl = 0; sl < 8; ++sl) {
                const int32_t e = child[(int64_t)v * 8 + sl];
                uint32_t x = nodes[src + 2 * sl], y = nodes[src + 2 * sl + 1];
                if (e >= 0) x = (uint32_t)(level[e] < B ? top_id[e] : brick_id[e]), y = 0;
                top_tab[i * 16 + 2 * sl] = x;
                top_tab[i * 16 + 2 * sl + 1] = y;
            }
        }
        const int S = 1 << blog;
        const int64_t cells = (int64_t)S * S * S;
        brick_cells.assign(n_bricks * cells * 2, 0);
        parallel_ranges(n_bricks, [&](int64_t b0, int64_t b1) {
            struct Item {
                int32_t v;
                int lev;
                uint32_t x, y, z;  // brick-local finest coordinates of the node's corner
            };
            std::vector<Item> st;
            for (int64_t b = b0; b < b1; ++b) {
                uint32_t* dst = brick_cells.data() + b * cells * 2;
                for (int64_t c = 0; c < cells; ++c) dst[2 * c] = ENTRY_EMPTY;
                st.clear();
                st.push_back({brick_nodes[b], B, 0, 0, 0});
                while (!st.empty()) {
                    Item it = st.back();
                    st.pop_back();
                    const uint32_t half = 1u << (depth - it.lev - 1);  // child size in finest cells
                    const int64_t src = (int64_t)new_id[it.v] * 16;
                    for (int sl = 0; sl < 8; ++sl) {
                        const int32_t e = child[(int64_t)it.v * 8 + sl];
                        const uint32_t cx = it.x + (sl & 1) * half, cy = it.y + ((sl >> 1) & 1) * half,
                                       cz = it.z + ((sl >> 2) & 1) * half;
                        if (e >= 0) {
                            st.push_back({e, it.lev + 1, cx, cy, cz});
                        } else if (e <= -2) {
                            const uint32_t ex = nodes[src + 2 * sl], ey = nodes[src + 2 * sl + 1];
                            for (uint32_t k = 0; k < half; ++k)
                                for (uint32_t j = 0; j < half; ++j)
                                    for (uint32_t i = 0; i < half; ++i) {
                                        const uint32_t m = spread3(cx + i) | (spread3(cy + j) << 1) |
                                                           (spread3(cz + k) << 2);
                                        dst[2 * m] = ex;
                                        dst[2 * m + 1] = ey;
                                    }
                        }
                    }
                }
            }
        });
    }

    plo_tree* t = new (std::nothrow) plo_tree();
    if (!t) return set_error(PLO_ERR_OOM, "host allocation failed");
    t->layout = bricks ? PLO_LAYOUT_BRICKS : PLO_LAYOUT_OCTREE;
    t->brick_log = blog;
    t->brick_level = bricks ? B : depth;
    t->n_top_nodes = n_top_nodes;
    t->n_top_staged = n_top_staged;
    t->n_bricks = n_bricks;
    t->top_bytes = n_top_nodes * 64;
    t->brick_bytes = (int64_t)brick_cells.size() * 4;
    t->depth = depth;
    t->sh_degree = desc->sh_degree;
    t->K = K;
    t->precision = precision;
    t->top_levels = top;
    t->n_top = n_top;
    t->n_nodes = n_packed;
    t->n_leaves = desc->n_leaves;
    t->n_sh = n_sh;
    t->sh_stride = stride;
    for (int a = 0; a < 3; ++a) {
        t->bbox_min[a] = desc->bbox_min[a];
        double inv = 1.0 / ((double)desc->bbox_max[a] - (double)desc->bbox_min[a]);
        t->inv_ext[a] = (float)inv;
        t->inv_ext_lo[a] = (float)(inv - (double)t->inv_ext[a]);
    }
    t->node_bytes = n_packed * 64;
    t->sh_bytes = (int64_t)n_sh * stride;
    cudaError_t err = cudaGetDevice(&t->device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, t->device);
    if (err != cudaSuccess) {
        delete t;
        return cuda_error(err, "cudaGetDevice");
    }
    size_t sh_alloc = (size_t)(n_sh > 0 ? n_sh : 1) * stride;
    if ((err = (cudaError_t)dev_malloc(&t->d_nodes, (size_t)t->node_bytes)) != cudaSuccess ||
        (err = (cudaError_t)dev_malloc((void**)&t->d_leaf_ids, (size_t)n_packed * 8 * sizeof(int32_t))) !=
            cudaSuccess ||
        (err = (cudaError_t)dev_malloc(&t->d_sh, sh_alloc)) != cudaSuccess ||
        (err = (cudaError_t)dev_malloc((void**)&t->d_flags, 256)) != cudaSuccess ||
        (bricks && (err = (cudaError_t)dev_malloc(&t->d_top, (size_t)t->top_bytes)) != cudaSuccess) ||
        (bricks && (err = (cudaError_t)dev_malloc(&t->d_bricks, (size_t)std::max<int64_t>(t->brick_bytes, 256))) !=
                       cudaSuccess)) {
        plo_tree_free(t);
        cudaGetLastError();
        return err == cudaErrorMemoryAllocation ? set_error(PLO_ERR_OOM, "device allocation for the tree failed")
                                                : cuda_error(err, "cudaMalloc");
    }
    if ((err = cudaMemcpy(t->d_nodes, nodes.data(), (size_t)t->node_bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMemcpy(t->d_leaf_ids, leaf_ids.data(), (size_t)n_packed * 8 * sizeof(int32_t),
                          cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMemcpy(t->d_sh, sh.get(), sh_alloc, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (err = cudaMemset(t->d_flags, 0, 256)) != cudaSuccess ||
        (bricks && (err = cudaMemcpy(t->d_top, top_tab.data(), (size_t)t->top_bytes, cudaMemcpyHostToDevice)) !=
                       cudaSuccess) ||
        (bricks && t->brick_bytes > 0 &&
         (err = cudaMemcpy(t->d_bricks, brick_cells.data(), (size_t)t->brick_bytes, cudaMemcpyHostToDevice)) !=
             cudaSuccess)) {
        plo_tree_free(t);
        return cuda_error(err, "upload of the packed tree");
    }
    *out = t;
    return PLO_OK;
}

}  // namespace

// Host allocations are large (the packed records alone are n_sh x stride
// bytes); none of them may escape the C ABI as an exception.
extern "C" plo_status plo_build_tree_ex(const plo_tree_desc* desc, const plo_build_options* options, plo_tree** out) {
    try {
        return build_tree(desc, options, out);
    } catch (const std::bad_alloc&) {
        if (out) *out = nullptr;
        return set_error(PLO_ERR_OOM, "host allocation while packing the tree failed");
    }
}

extern "C" plo_status plo_build_tree(const plo_tree_desc* desc, int32_t precision, plo_tree** out) {
    const plo_build_options opt = {precision, PLO_LAYOUT_DEFAULT, 0};
    return plo_build_tree_ex(desc, &opt, out);
}

extern "C" void plo_tree_free(plo_tree* t) {
    if (!t) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(t->device);
    cudaDeviceSynchronize();
    cudaFree(t->d_nodes);
    cudaFree(t->d_leaf_ids);
    cudaFree(t->d_sh);
    cudaFree(t->d_flags);
    cudaFree(t->d_top);
    cudaFree(t->d_bricks);
    if (prev >= 0) cudaSetDevice(prev);
    delete t;
}

extern "C" plo_status plo_tree_get_info(const plo_tree* t, plo_tree_info* out) {
    if (!t || !out) return set_error(PLO_ERR_INVALID_ARG, "tree or out is NULL");
    out->depth = t->depth;
    out->sh_degree = t->sh_degree;
    out->precision = t->precision;
    out->top_levels = t->top_levels;
    out->n_nodes = t->n_nodes;
    out->n_leaves = t->n_leaves;
    out->n_sh_records = t->n_sh;
    out->node_bytes = t->node_bytes;
    out->sh_bytes = t->sh_bytes;
    out->sh_record_stride = t->sh_stride;
    out->device = t->device;
    out->layout = t->layout;
    out->brick_log = t->brick_log;
    out->n_bricks = t->n_bricks;
    out->brick_bytes = t->brick_bytes;
    out->top_nodes = t->n_top_nodes;
    return PLO_OK;
}

extern "C" plo_status plo_tree_check(const plo_tree* t, void* stream) {
    if (!t) return set_error(PLO_ERR_INVALID_ARG, "tree is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int flags = 0;
    cudaError_t err = cudaMemcpyAsync(&flags, t->d_flags, sizeof(flags), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return cuda_error(err, "plo_tree_check");
    if (flags) {
        cudaMemsetAsync(t->d_flags, 0, sizeof(unsigned int), s);
        cudaStreamSynchronize(s);
        if (flags & 1u) return set_error(PLO_ERR_TRAVERSAL_LIMIT, "a ray exceeded its step cap (max_steps)");
    }
    return PLO_OK;
}
