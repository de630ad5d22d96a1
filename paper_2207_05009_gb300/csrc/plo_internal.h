// Internal definitions shared by the library's translation units.
//
// Device layout of a packed tree (built by tree.cpp from the canonical host
// format of include/plo.h):
//
//   nodes   uint2 [n_nodes][8]   one 8-byte entry per child slot
//             .x == ENTRY_EMPTY             empty octant
//             .x <  LEAF_BIT                internal node id
//             .x &  LEAF_BIT                leaf; low 31 bits = SH record id,
//                                           or NO_SH_RECORD when all of the
//                                           leaf's coefficients are zero
//             .y  (leaves only)  FP32 trees: sigma as float bits
//                               FP16/BF16:  bits 0..23 sigma as a 24-bit
//                               float (FP32 bits 30..7: exponent and 16
//                               mantissa bits, round-to-nearest-even),
//                               bits 24..31 biased exponent e+127 of the
//                               leaf's SH scale 2^e (FP16 maps the largest
//                               |coefficient| into [2^14, 2^15), BF16 into
//                               [0.5, 1))
//           A leaf's density travels with its parent's child entry, so a
//           non-emissive leaf costs no load beyond the descent itself.
//           Nodes of the top `top_levels` levels come first (breadth-first),
//           the rest follow in depth-first (Morton) order.
//   Brick layout (PLO_LAYOUT_BRICKS) adds, for the render kernels:
//   top     uint2 [n_top_nodes][8]  the nodes of levels < B = depth - s in
//           the same order and encoding, except that a child at level B
//           that has children is a brick id;
//   bricks  uint2 [n_bricks][2^3s]  per brick a dense array of the entries
//           of its (2^s)^3 finest cells, index = Morton interleave of the
//           brick-local coordinates (x lowest): the entry of the leaf that
//           covers the cell (a leaf above the finest level repeats over its
//           cells), or ENTRY_EMPTY.
//   leaf_ids int32 [n_nodes][8]  canonical leaf id per entry (-1 otherwise);
//           read only by the lookup and trace diagnostics.
//   sh      records of 3*K coefficients, channel-major, one per emissive
//           leaf, in depth-first order, `sh_stride` bytes apart (16-byte
//           aligned): FP32 12K bytes rounded up to 16; FP16/BF16 6K rounded
//           up to 16 (K=9: 64 B, K=16: 96 B).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/plo.h"

namespace plo {

constexpr uint32_t ENTRY_EMPTY = 0xFFFFFFFFu;
constexpr uint32_t LEAF_BIT = 0x80000000u;
constexpr uint32_t NO_SH_RECORD = 0x7FFFFFFEu;
constexpr int MAX_DEPTH = 16;
constexpr int MAX_TOP_NODES = 585;  // levels 0..3 of a full octree

inline int sh_K(int degree) { return (degree + 1) * (degree + 1); }
inline int sh_stride_bytes(int K, int precision) {
    int raw = precision == PLO_PREC_FP32 ? 12 * K : 6 * K;
    return (raw + 15) / 16 * 16;
}

// Thread-local error message, returned by plo_last_error().
plo_status set_error(plo_status s, const std::string& msg);
plo_status cuda_error(int err, const char* what);

// Every device allocation of the library goes through one of these two
// (cudaMalloc, and cudaMallocAsync on a stream), so that tests can make the
// n-th one fail (plo_debug_fail_alloc_after).
int dev_malloc(void** p, size_t bytes);
int dev_malloc_async(void** p, size_t bytes, cudaStream_t s);

// Exclusive prefix sum of n uint32 values on the device (async on s; its
// temporary goes through dev_malloc_async).  in == out is allowed.
cudaError_t device_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);

// Packs, on the device, the octree whose leaves are the voxels with the
// sorted Morton codes d_codes [nl] at level `depth` (<= 10): their entry
// words d_yword (sigma bits; for 16-bit trees sigma24 | scale exponent << 24)
// and emission flags d_emits, and their packed SH records d_records [nl]
// (record id = leaf id), which the tree takes over on success.  Same layout
// as plo_build_tree of the equivalent canonical tree (octree layout).
plo_status pack_voxel_tree(int depth, int sh_degree, int precision, const uint32_t* d_codes, int64_t nl,
                           uint32_t* d_yword, uint8_t* d_emits, void* d_records, cudaStream_t s, plo_tree** out);

}  // namespace plo

struct plo_tree {
    int32_t depth;       // depth of the packed tree (>= 1; a root leaf is re-rooted one level down)
    int32_t sh_degree, K, precision;
    int32_t top_levels;  // levels whose nodes are staged in shared memory
    int32_t n_top;       // number of nodes in those levels (ids 0..n_top-1)
    int64_t n_nodes, n_leaves, n_sh;
    int32_t sh_stride;
    int32_t device;
    float bbox_min[3], inv_ext[3], inv_ext_lo[3];  // 1/extent as a double-float
    void* d_nodes;       // uint2 [n_nodes][8]
    int32_t* d_leaf_ids; // [n_nodes][8]
    void* d_sh;
    unsigned int* d_flags;  // device error flags (bit 0: step limit)
    int64_t node_bytes, sh_bytes;
    int32_t sm_count;
    // brick layout (PLO_LAYOUT_BRICKS): the octree above brick_level with
    // brick ids at that level, and the dense bricks below it
    int32_t layout;
    int32_t brick_log;     // brick side 2^brick_log finest cells
    int32_t brick_level;   // level of the brick cells (= depth for the octree layout)
    int32_t n_top_staged;  // top-tree nodes of levels < min(4, brick_level)
    int64_t n_top_nodes, n_bricks;
    int64_t top_bytes, brick_bytes;
    void* d_top = nullptr;     // uint2 [n_top_nodes][8]
    void* d_bricks = nullptr;  // uint2 [n_bricks][2^(3 brick_log)], Morton order
};
