// Fused plenoctree render kernel for sm_103a: proxy clip -> octree walk ->
// per-leaf SH emission -> front-to-back emission/absorption compositing
// (paper Sec. 4.1, Eq. 3-5; plenoctree of Sec. 4.2 / Sec. 5).
//
// One thread renders one ray at a time.  The grid is persistent: warps take
// rays from a shared counter (32 at a time; small launches give each warp a
// contiguous chunk) and a lane that finishes its ray takes the next one, so
// a warp does not idle behind its longest ray; each iteration of a warp
// moves every live lane past the cell it is in (advance, then composite),
// then descends every lane towards its next cell, at most 4 levels per
// iteration.  Child slots come from the bits of the point's integer
// coordinates on the finest grid.
//
// Numerics (all FP32, no FP64 on the device):
//   * The ray position is kept as an unevaluated sum hi + lo of two floats
//     per axis ("double-float").  Segment lengths come from exact dyadic cell
//     planes minus that position, so every segment length has ~1e-7 relative
//     error however far the ray origin is, and the cell sequence matches an
//     FP64 walk except for rays passing within ~1e-13 of a cell edge.
//   * The exit coordinate is snapped onto the exact plane; the next cell is
//     found by re-descending from the deepest common ancestor (kept on a
//     per-ray stack) with the tie rule "on a plane, go where the direction
//     points", so progress is guaranteed.
//   * Optical depth is accumulated as a compensated (two-float) sum;
//     T = exp(-OD) or max(0, 1 - OD) is recomputed from it after each leaf.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "plo_internal.h"
#include "sh.cuh"

namespace plo {
namespace {

constexpr int BLOCK = 256;
#ifndef PLO_RENDER_MIN_BLOCKS
#define PLO_RENDER_MIN_BLOCKS 4  // resident blocks per SM the register budget is sized for (measured best)
#endif
#ifndef PLO_BRICK_MIN_BLOCKS
#define PLO_BRICK_MIN_BLOCKS 3  // the same for the brick-layout kernels
#endif
constexpr int WARPS = BLOCK / 32;
constexpr int64_t RENDER_CLAIM = 32;  // rays a warp claims at a time from the shared cursor (32 measured best of 32-128)
#ifndef PLO_DESCEND_LEVELS
#define PLO_DESCEND_LEVELS 4  // tree levels a descent goes down per step (measured best of 2, 3, 4, 5, all)
#endif

// One packed tree as the kernels see it.
struct TreeParams {
    const uint2* nodes;   // node table walked by the descent (the brick layout's top tree)
    const int32_t* leaf_ids;
    const uint8_t* sh;
    unsigned int* flags;
    const uint2* bricks;  // brick layout: dense bricks below top_depth (NULL: octree layout)
    int32_t brick_log;    // brick side 2^brick_log finest cells
    int32_t top_depth;    // level of the brick cells (= depth for the octree layout)
    int32_t sh_stride;
    int32_t depth;
    int32_t n_top;   // nodes staged in shared memory (ids 0 .. n_top-1)
    int32_t s_off;   // their offset in the block's shared node table (entries)
    int32_t K, prec;
    int32_t max_steps;
    float bmin[3], inv_ext[3], inv_ext_lo[3];  // 1/extent as a double-float
};

struct KParams {
    TreeParams tree;
    int32_t transmittance, activation;
    float l_max, t_stop, sigma_min;
    int32_t saturate, proxy;
    float sphere[4];  // sphere proxy: centre, radius (world space)
    const float* rays;
    unsigned long long* cursor;  // shared claim counter (NULL: static chunks per warp)
    int64_t n;
    int64_t chunk;  // rays per warp
    float* rgb;
    float* T;
    int32_t* status;
    // trace mode
    int32_t trace_max;
    int64_t* tr_leaf;
    float* tr_t;
    int32_t* tr_count;
};

// ---------------------------------------------------------------- double-float
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// (a_hi + a_lo) * (r_hi + r_lo) with r = 1/d in double-float.
__device__ __forceinline__ DF df_mul(DF a, float rh, float rl) {
    float p = __fmul_rn(a.hi, rh);
    float e = __fmaf_rn(a.hi, rh, -p);
    e = __fmaf_rn(a.hi, rl, e);
    e = __fmaf_rn(a.lo, rh, e);
    return fast_two_sum(p, e);
}
// double-float reciprocal of d = dh + dl (dh finite, non-zero)
__device__ __forceinline__ void df_recip(float dh, float dl, float& rh, float& rl) {
    rh = __frcp_rn(dh);
    float r = __fmaf_rn(-rh, dh, 1.0f);  // exact residual of the rounded reciprocal
    r = __fmaf_rn(-rh, dl, r);
    rl = __fmul_rn(r, rh);
}
// p + t * d, all double-float
__device__ __forceinline__ DF df_axpy(DF p, DF t, float dh, float dl) {
    float m = __fmul_rn(t.hi, dh);
    float me = __fmaf_rn(t.hi, dh, -m);
    me = __fmaf_rn(t.lo, dh, me);
    me = __fmaf_rn(t.hi, dl, me);
    DF s = two_sum(p.hi, m);
    float lo = __fadd_rn(__fadd_rn(s.lo, p.lo), me);
    return fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ DF df_sub(DF a, DF b) {
    DF s = two_sum(a.hi, -b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}
// a * b exactly, as a double-float
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_mul_df(DF a, DF b) {
    DF p = two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, p.lo);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
// a / b (b.hi != 0): quotient of the high parts plus one correction step
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const DF r = df_sub(a, df_mul_df(b, DF{q1, 0.0f}));
    return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
// sqrt(a) for a >= 0: one Newton correction of the FP32 root
__device__ __forceinline__ DF df_sqrt(DF a) {
    const float s = __fsqrt_rn(a.hi);
    if (s == 0.0f) return {0.0f, 0.0f};
    const float e = __fadd_rn(__fmaf_rn(-s, s, a.hi), a.lo);
    return fast_two_sum(s, __fdiv_rn(e, __fmul_rn(2.0f, s)));
}
// (P - p) for an exact float plane P
__device__ __forceinline__ DF df_from_plane(float P, DF p) {
    DF n = two_sum(P, -p.hi);
    return two_sum(n.hi, __fsub_rn(n.lo, p.lo));
}
__device__ __forceinline__ bool df_less(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool df_eq(DF a, DF b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ float pow2i(int e) { return __int_as_float((127 + e) << 23); }  // e in [-126, 127]
// Finest-grid coordinate of p (depth D, scale = 2^D): floor(p 2^D), except
// that a point exactly on a grid plane belongs to the cell below it when the
// direction is negative (the tie rule), clamped to [0, 2^D - 1] (the root box
// is closed).  Bit D-1-l of the result is the child bit at level l: the same
// decision as comparing p with every mid-plane on the way down.
__device__ __forceinline__ uint32_t quantize(DF p, float scale, uint32_t qmax, float d) {
    const float h = p.hi * scale;  // exact: scale is a power of two
    const float f = floorf(h);
    int q = (int)f;
    if (h == f && (p.lo < 0.0f || (p.lo == 0.0f && d < 0.0f))) --q;
    q = max(q, 0);
    return min((uint32_t)q, qmax);
}

// Loads one SH record and returns sum_k c_{ch,k} Y_k for the three channels.
template <int K, int PREC>
__device__ __forceinline__ void sh_eval(const uint8_t* rec, uint32_t yword, const float* Y, float& r, float& g,
                                        float& b) {
    float acc[3] = {0.0f, 0.0f, 0.0f};
    if (PREC == PLO_PREC_FP32) {
        constexpr int NV = (3 * K + 3) / 4;
        const float4* v = reinterpret_cast<const float4*>(rec);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            float4 q = __ldg(v + j);
            float e[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int gi = 4 * j + u;
                if (gi < 3 * K) acc[gi / K] = __fmaf_rn(e[u], Y[gi % K], acc[gi / K]);
            }
        }
    } else {
        constexpr int NV = (3 * K + 7) / 8;
        const uint4* v = reinterpret_cast<const uint4*>(rec);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            uint4 q = __ldg(v + j);
            uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                int gi = 8 * j + u;
                if (gi < 3 * K) {
                    uint16_t bits = (uint16_t)(w[u >> 1] >> (16 * (u & 1)));
                    float f = PREC == PLO_PREC_FP16 ? __half2float(__ushort_as_half(bits))
                                                    : __uint_as_float((uint32_t)bits << 16);
                    acc[gi / K] = __fmaf_rn(f, Y[gi % K], acc[gi / K]);
                }
            }
        }
        float s = pow2i((int)(yword >> 24) - 127);
        acc[0] *= s;
        acc[1] *= s;
        acc[2] *= s;
    }
    r = acc[0];
    g = acc[1];
    b = acc[2];
}

template <int PREC>
__device__ __forceinline__ float decode_sigma(uint32_t y, int prec) {
    if (PREC == PLO_PREC_FP32 || (PREC < 0 && prec == PLO_PREC_FP32)) return __uint_as_float(y);
    return __uint_as_float((y & 0xFFFFFFu) << 7);  // 24-bit float: exponent + 16 mantissa bits
}

// SH emission of one record; K / PREC given at compile time, or read from
// the tree when K == 0 (the batch kernel mixes trees).
template <int K, int PREC>
__device__ __forceinline__ void sh_emission(const TreeParams& tp, uint32_t rec, uint32_t yword, const float* dirn,
                                            float& r, float& g, float& b, const float* sY = nullptr) {
    const uint8_t* p = tp.sh + (size_t)rec * tp.sh_stride;
    if (K > 0) {  // the per-lane basis in shared memory (sY, set at the ray's start)
        float Y[K > 0 ? K : 1];
#pragma unroll
        for (int k = 0; k < (K > 0 ? K : 1); ++k) Y[k] = sY[k * BLOCK];
        sh_eval<(K > 0 ? K : 1), PREC>(p, yword, Y, r, g, b);
        return;
    }
    // each degree builds only its own basis, so that the registers of the
    // larger bases are taken only in their branches
#define PLO_SH_CASE(KK, PP)                                  \
    if (tp.K == KK && tp.prec == PP) {                       \
        float Y[KK];                                         \
        sh_basis<KK>(dirn[0], dirn[1], dirn[2], Y);          \
        return sh_eval<KK, PP>(p, yword, Y, r, g, b);        \
    }
    PLO_SH_CASE(16, PLO_PREC_FP32) PLO_SH_CASE(9, PLO_PREC_FP32) PLO_SH_CASE(16, PLO_PREC_FP16)
    PLO_SH_CASE(9, PLO_PREC_FP16) PLO_SH_CASE(16, PLO_PREC_BF16) PLO_SH_CASE(9, PLO_PREC_BF16)
    PLO_SH_CASE(4, PLO_PREC_FP32) PLO_SH_CASE(4, PLO_PREC_FP16) PLO_SH_CASE(4, PLO_PREC_BF16)
    PLO_SH_CASE(1, PLO_PREC_FP32) PLO_SH_CASE(1, PLO_PREC_FP16) PLO_SH_CASE(1, PLO_PREC_BF16)
    PLO_SH_CASE(25, PLO_PREC_FP32) PLO_SH_CASE(25, PLO_PREC_FP16) PLO_SH_CASE(25, PLO_PREC_BF16)
#undef PLO_SH_CASE
    r = g = b = 0.0f;
}

__device__ __forceinline__ float act_fn(float s, int act, float l_max) {
    return act == PLO_ACT_RELU ? fmaxf(s, 0.0f) : l_max / (1.0f + expf(-s));
}

// ---------------------------------------------------------------- per-ray state
// Lane states: idle (no ray), descending to the cell at its current point,
// at a leaf cell waiting to composite it, or walking a brick cell by cell.
enum : int { ST_IDLE = 0, ST_DESCEND = 1, ST_LEAF = 2, ST_BRICK = 3 };

struct Ray {
    DF p[3];
    float d[3];         // unit-cube direction (high part; the low part is in low_parts())
    float dirn[3];      // normalised world direction for the SH basis
    float T, r, g, b;
    DF od;
    DF t;               // ray parameter at the current cell entry (trace only)
    DF rem;             // ray parameter left inside the sphere proxy (sphere only)
    uint32_t q[3];      // integer coordinates of the current point on the finest (depth-D) grid
                        // (ST_BRICK: of the point where the ray entered the brick)
    uint32_t node;      // node whose child is looked up next (ST_DESCEND); the brick (ST_BRICK)
    DF tn[3];           // ST_BRICK: ray parameter, from the brick entry point, of the next
                        // finest-grid plane crossed on each axis
    DF tb;              // ST_BRICK: the same parameter at the current cell's entry
    uint32_t loc;       // ST_BRICK: brick-local finest coordinates x | y << 4 | z << 8
    uint32_t entry_x, entry_y;
    int level;
    int steps;
    int slot;           // slot of the current cell in its parent (trace only)
    int state;
    int status;
    int tree;           // index into the batch's tree table (batch kernel only)
};

// Per-ray constants read once per cell, kept in shared memory to leave
// registers to the hot state: the low-order part of the double-float
// direction (dl, zero for the unit box) at [a * BLOCK], the reciprocal 1/d
// as a double-float, low part rl at [(3 + a) * BLOCK] and high part rh at
// [(6 + a) * BLOCK].  Column per thread.
__device__ __forceinline__ float* low_parts() {
    __shared__ float s_low[9 * BLOCK];
    return s_low + threadIdx.x;
}

__device__ __forceinline__ uint2 load_entry(const TreeParams& tp, const uint2* s_nodes, uint32_t node, int slot) {
    if (node < (uint32_t)tp.n_top) return s_nodes[tp.s_off + node * 8 + slot];
    return __ldg(tp.nodes + (size_t)node * 8 + slot);
}

// Brick-local cell index: Morton interleave of the local coordinates
// (loc = x | y << 4 | z << 8, each < 8), x lowest.
__device__ __forceinline__ uint32_t spread3(uint32_t x) { return (x & 1u) | ((x & 2u) << 2) | ((x & 4u) << 4); }
__device__ __forceinline__ uint2 brick_entry(const TreeParams& tp, uint32_t brick, uint32_t loc) {
    const uint32_t m = spread3(loc & 15u) | (spread3((loc >> 4) & 15u) << 1) | (spread3(loc >> 8) << 2);
    return __ldg(tp.bricks + ((size_t)brick << (3 * tp.brick_log)) + m);
}

// Enters brick `brick`, the level-top_depth cell that holds the current
// point: the brick-local coordinates of the finest cell R.q, and per axis the
// parameter of the next finest plane from the current point,
// (P - p) / d in double-float (as the octree step computes its exits).  The
// first cell's entry is loaded here, for the next iteration.
__device__ __forceinline__ void brick_enter(const TreeParams& tp, Ray& R, uint32_t brick) {
    const uint32_t smask = (1u << tp.brick_log) - 1u;
    R.node = brick;
    R.loc = (R.q[0] & smask) | ((R.q[1] & smask) << 4) | ((R.q[2] & smask) << 8);
    const float cell = pow2i(-tp.depth);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        DF v = {INFINITY, 0.0f};
        if (R.d[a] != 0.0f) {
            const float P = (float)(R.q[a] + (R.d[a] > 0.0f ? 1u : 0u)) * cell;  // exact
            v = df_mul(df_from_plane(P, R.p[a]), low_parts()[(6 + a) * BLOCK], low_parts()[(3 + a) * BLOCK]);
            if (v.hi < 0.0f) v = {0.0f, 0.0f};
        }
        R.tn[a] = v;
    }
    R.tb = {0.0f, 0.0f};
    const uint2 e = brick_entry(tp, brick, R.loc);
    R.entry_x = e.x;
    R.entry_y = e.y;
    R.state = ST_BRICK;
}

// Descends from R.node (level R.level) towards the leaf or empty octant that
// holds the point, taking the child bits from the finest-grid coordinates
// R.q, and ends in ST_LEAF (or, in the brick layout, in ST_BRICK when it
// reaches a brick).  A step goes down at most PLO_DESCEND_LEVELS levels; a
// longer descent goes on in the next step while the other lanes composite.
// A lane needs 2 levels per step on average but the warp ran the longest
// descent among its lanes, 5.7 levels (depth-10 luminaire, 16M room rays):
// 4 levels per step measured 348 -> 365 Mrays/s with FP32 leaves, 390 ->
// 397 with FP16; 2 levels gained nothing and 1 level lost.
template <bool BRICKS, int PREC>
__device__ __forceinline__ void descend_step(const TreeParams& tp, const uint2* s_nodes, Ray& R, uint32_t* stack) {
    for (int guard = 0; guard < PLO_DESCEND_LEVELS; ++guard) {
        const int sh = tp.depth - 1 - R.level;
        R.slot = (int)(((R.q[0] >> sh) & 1u) | (((R.q[1] >> sh) & 1u) << 1) | (((R.q[2] >> sh) & 1u) << 2));
        uint2 e = load_entry(tp, s_nodes, R.node, R.slot);
        ++R.level;
        if ((e.x & LEAF_BIT) || R.level >= tp.top_depth) {  // leaf, empty octant, brick (or a malformed table)
            if (BRICKS && tp.bricks && !(e.x & LEAF_BIT) && R.level == tp.top_depth) {
                brick_enter(tp, R, e.x);
                return;
            }
            if (!(e.x & LEAF_BIT)) e = make_uint2(ENTRY_EMPTY, 0u);
            R.entry_x = e.x;
            R.entry_y = e.y;
            R.state = ST_LEAF;
            // the SH record is read in the next iteration: start pulling it
            // into L2 now, for 16-bit records (measured on the depth-10
            // workload: FP16 427 -> 436 Mrays/s with it, FP32 410 -> 404,
            // so FP32 records are left to the load itself; before the leaf
            // step advanced ahead of its compositing FP32 gained, 366 ->
            // 379).  The choice is made at compile time: as a run-time test
            // it cost the FP16 kernel 9%.
            const uint32_t rec = e.x & ~LEAF_BIT;
            constexpr bool always = PREC > 0, never = PREC == PLO_PREC_FP32;
            if (!never && (always || tp.prec != PLO_PREC_FP32) && e.x != ENTRY_EMPTY && rec != NO_SH_RECORD) {
                const char* a = reinterpret_cast<const char*>(tp.sh) + (size_t)rec * tp.sh_stride;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a + tp.sh_stride - 1));
            }
            return;
        }
        stack[R.level * BLOCK] = e.x;
        R.node = e.x;
    }
}

__device__ __forceinline__ void ray_store(const KParams& kp, int64_t i, const Ray& R) {
    kp.rgb[3 * i + 0] = R.r;
    kp.rgb[3 * i + 1] = R.g;
    kp.rgb[3 * i + 2] = R.b;
    kp.T[i] = kp.saturate && R.T < kp.t_stop ? 0.0f : R.T;  // a saturated ray is opaque (Sec. 6.2)
    if (kp.status) kp.status[i] = R.status;
    if (kp.tr_count) kp.tr_count[i] = R.steps;
}

// Proxy clip.  On a hit the lane enters ST_DESCEND at the root; on a miss or
// an invalid ray the outputs are written and the lane stays ST_IDLE.
template <bool TRACE, bool SPHERE>
__device__ void ray_begin(const KParams& kp, const TreeParams& tp, int64_t i, Ray& R, uint32_t* stack) {
    const float* q = kp.rays + 6 * i;
    float o[3], dw[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = __ldg(q + a);
        dw[a] = __ldg(q + 3 + a);
    }
    R.T = 1.0f;
    R.r = R.g = R.b = 0.0f;
    R.od = {0.0f, 0.0f};
    R.t = {0.0f, 0.0f};
    R.status = PLO_RAY_OK;
    R.steps = 0;
    R.state = ST_IDLE;
    bool bad = dw[0] == 0.0f && dw[1] == 0.0f && dw[2] == 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) bad |= !isfinite(o[a]) || !isfinite(dw[a]);
    if (bad) {
        R.status = PLO_RAY_INVALID;
        R.r = R.g = R.b = R.T = __int_as_float(0x7fc00000);
        ray_store(kp, i, R);
        return;
    }
    const float inv_n = rsqrtf(__fadd_rn(__fadd_rn(__fmul_rn(dw[0], dw[0]), __fmul_rn(dw[1], dw[1])),
                                         __fmul_rn(dw[2], dw[2])));
    DF ou[3];  // origin in unit-cube coordinates, (o - bmin) / extent in double-float
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R.dirn[a] = __fmul_rn(dw[a], inv_n);
        ou[a] = df_mul(two_sum(o[a], -tp.bmin[a]), tp.inv_ext[a], tp.inv_ext_lo[a]);
        DF du = df_mul(DF{dw[a], 0.0f}, tp.inv_ext[a], tp.inv_ext_lo[a]);
        R.d[a] = du.hi;
        low_parts()[a * BLOCK] = du.lo;
    }
    // slab test in double-float
    DF tn = {-INFINITY, 0.0f}, tf = {INFINITY, 0.0f};
    DF near_a[3];
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        near_a[a] = {-INFINITY, 0.0f};
        if (R.d[a] == 0.0f) {
            if (ou[a].hi < 0.0f || ou[a].hi > 1.0f || (ou[a].hi == 0.0f && ou[a].lo < 0.0f) ||
                (ou[a].hi == 1.0f && ou[a].lo > 0.0f))
                miss = true;
            continue;
        }
        float rh, rl;
        df_recip(R.d[a], low_parts()[a * BLOCK], rh, rl);
        low_parts()[(6 + a) * BLOCK] = rh;
        low_parts()[(3 + a) * BLOCK] = rl;
        DF t0 = df_mul(df_from_plane(0.0f, ou[a]), rh, rl);
        DF t1 = df_mul(df_from_plane(1.0f, ou[a]), rh, rl);
        if (df_less(t1, t0)) {
            DF s = t0;
            t0 = t1;
            t1 = s;
        }
        near_a[a] = t0;
        if (df_less(tn, t0)) tn = t0;
        if (df_less(t1, tf)) tf = t1;
    }
    if (miss || !df_less(tn, tf) || !(tf.hi > 0.0f || (tf.hi == 0.0f && tf.lo > 0.0f))) {
        ray_store(kp, i, R);
        return;
    }
    if (SPHERE) {
        // sphere proxy (Sec. 5): keep the part of [tn, tf] inside the ball
        // |o + t d - c| <= r, solved once per ray in world space with
        // double-float arithmetic (about 44 significant bits; no FP64 on the
        // device).  With oc = o - c: a t^2 + 2 b t + q = 0, a = d.d,
        // b = oc.d, q = oc.oc - r^2; the root away from -b comes from
        // m = -(b + sign(b) sqrt(b^2 - a q)) as m / a, the other as q / m, so
        // neither subtracts nearly equal numbers.
        DF a2 = {0.0f, 0.0f}, b = {0.0f, 0.0f}, q = {0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const DF oc = two_sum(o[a], -kp.sphere[a]);
            const DF dd = {dw[a], 0.0f};
            a2 = df_add(a2, two_prod(dw[a], dw[a]));
            b = df_add(b, df_mul_df(oc, dd));
            q = df_add(q, df_mul_df(oc, oc));
        }
        q = df_sub(q, two_prod(kp.sphere[3], kp.sphere[3]));
        const DF disc = df_sub(df_mul_df(b, b), df_mul_df(a2, q));
        if (!(disc.hi > 0.0f || (disc.hi == 0.0f && disc.lo > 0.0f))) {
            ray_store(kp, i, R);
            return;
        }
        const DF sq = df_sqrt(disc);
        const DF m = df_neg(b.hi >= 0.0f ? df_add(b, sq) : df_sub(b, sq));
        const DF r_far = df_div(m, a2), r_near = df_div(q, m);
        const bool mneg = m.hi < 0.0f;
        const DF s0 = mneg ? r_far : r_near, s1 = mneg ? r_near : r_far;
        if (df_less(tn, s0)) tn = s0;
        if (df_less(s1, tf)) tf = s1;
        if (!df_less(tn, tf) || !(tf.hi > 0.0f || (tf.hi == 0.0f && tf.lo > 0.0f))) {
            ray_store(kp, i, R);
            return;
        }
    }
    bool outside = tn.hi > 0.0f || (tn.hi == 0.0f && tn.lo > 0.0f);
    if (SPHERE) R.rem = outside ? df_sub(tf, tn) : tf;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R.p[a] = outside ? df_axpy(ou[a], tn, R.d[a], low_parts()[a * BLOCK]) : ou[a];
        if (outside && R.d[a] != 0.0f && df_eq(near_a[a], tn)) R.p[a] = {R.d[a] > 0.0f ? 0.0f : 1.0f, 0.0f};
        if (R.p[a].hi < 0.0f) R.p[a] = {0.0f, 0.0f};  // rounding guard
        if (R.p[a].hi > 1.0f || (R.p[a].hi == 1.0f && R.p[a].lo > 0.0f)) R.p[a] = {1.0f, 0.0f};
    }
    if (TRACE) R.t = outside ? tn : DF{0.0f, 0.0f};
    const float scale = pow2i(tp.depth);
    const uint32_t qmax = (1u << tp.depth) - 1u;
#pragma unroll
    for (int a = 0; a < 3; ++a) R.q[a] = quantize(R.p[a], scale, qmax, R.d[a]);
    stack[0] = 0;
    R.node = 0;
    R.level = 0;
    R.state = ST_DESCEND;
}

// Composites the current cell's entry over a segment of length `seg` (Eq.
// 3-5): optical depth as a compensated sum, weight T_in (1 - e^{-sigma seg})
// or the linear model's, SH emission of emitting leaves.  Returns true when
// the ray is finished (T below t_stop) and its outputs are written.
template <int K, int PREC>
__device__ __forceinline__ bool composite(const KParams& kp, const TreeParams& tp, int64_t i, Ray& R, float seg,
                                          const float* sY) {
    if (R.entry_x == ENTRY_EMPTY) return false;
    float sigma = decode_sigma<PREC>(R.entry_y, tp.prec);
    if (sigma < kp.sigma_min) sigma = 0.0f;
    if (!(sigma > 0.0f)) return false;
    // the emission first: its record loads are then in flight during the
    // transmittance arithmetic (measured +1.5% with FP32 leaves)
    const uint32_t rec = R.entry_x & ~LEAF_BIT;
    float cr = 0.0f, cg = 0.0f, cb = 0.0f;
    const bool emits = rec != NO_SH_RECORD;
    if (emits) sh_emission<K, PREC>(tp, rec, R.entry_y, R.dirn, cr, cg, cb, sY);
    const float a = sigma * seg;
    const float Tin = R.T;
    const DF s = two_sum(R.od.hi, a);
    R.od = fast_two_sum(s.hi, __fadd_rn(s.lo, R.od.lo));
    float w, Tout;
    if (kp.transmittance == PLO_TRANS_EXP) {
        w = Tin * (-expm1f(-a));
        Tout = expf(-(R.od.hi + R.od.lo));
    } else {
        Tout = fmaxf(0.0f, __fsub_rn(__fsub_rn(1.0f, R.od.hi), R.od.lo));
        const float dT = fminf(Tin, a);
        w = kp.transmittance == PLO_TRANS_LINEAR ? dT : 0.5f * dT * (Tin + Tout);
    }
    if (emits || kp.activation != PLO_ACT_RELU) {
        R.r = __fmaf_rn(w, act_fn(cr, kp.activation, kp.l_max), R.r);
        R.g = __fmaf_rn(w, act_fn(cg, kp.activation, kp.l_max), R.g);
        R.b = __fmaf_rn(w, act_fn(cb, kp.activation, kp.l_max), R.b);
    }
    R.T = Tout;
    if (R.T < kp.t_stop || R.T <= 0.0f) {
        ray_store(kp, i, R);
        R.state = ST_IDLE;
        return true;
    }
    return false;
}

// One cell: segment length, advance to the next cell, compositing.  Leaves
// the lane in ST_DESCEND (next cell) or ST_IDLE (ray finished, outputs
// written).
template <int K, int PREC, bool TRACE, bool SPHERE>
__device__ void leaf_step(const KParams& kp, const TreeParams& tp, int64_t i, Ray& R, uint32_t* stack,
                          const float* sY = nullptr) {
    // segment: exit parameter of the current cell along each axis.  An FP32
    // estimate (error below 6e-8 |1/d| + 2e-7 v) picks the candidate exit
    // axes; only those get the double-float value.  Nearly always there is
    // one candidate: its operands are picked by selects so that the
    // double-float work is issued once per warp instead of once per axis.
    const int L = R.level;
    const int down = tp.depth - L;
    const float size = pow2i(-L);
    uint32_t c[3];
    float planes[3], va[3], rh[3];
    float vmin = INFINITY, rmin = 0.0f;
    int ax = 0;  // axis of the smallest estimate
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        rh[a] = low_parts()[(6 + a) * BLOCK];
        c[a] = R.q[a] >> down;
        planes[a] = (float)(c[a] + (R.d[a] > 0.0f ? 1u : 0u)) * size;
        va[a] = INFINITY;
        if (R.d[a] == 0.0f) continue;
        va[a] = fmaxf(__fmul_rn(__fsub_rn(planes[a], R.p[a].hi), rh[a]), 0.0f);
        if (va[a] < vmin) {
            vmin = va[a];
            rmin = fabsf(rh[a]);
            ax = a;
        }
    }
    DF dt = {INFINITY, 0.0f};
    DF dts[3];
    bool cand[3];
    int n_cand = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dts[a] = {INFINITY, 0.0f};
        cand[a] = va[a] <= vmin + 2.5e-7f * (fabsf(rh[a]) + rmin) + 1e-6f * vmin;
        n_cand += cand[a] ? 1 : 0;
    }
    if (n_cand == 1) {
        // the usual case: one candidate axis, gathered by selects so that the
        // double-float work runs once for every lane whatever its axis
        const float P = ax == 0 ? planes[0] : (ax == 1 ? planes[1] : planes[2]);
        const DF pa = ax == 0 ? R.p[0] : (ax == 1 ? R.p[1] : R.p[2]);
        const float rha = ax == 0 ? rh[0] : (ax == 1 ? rh[1] : rh[2]);
        DF v = df_mul(df_from_plane(P, pa), rha, low_parts()[(3 + ax) * BLOCK]);
        if (v.hi < 0.0f) v = {0.0f, 0.0f};
        dt = v;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a == ax) dts[a] = v;
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!cand[a]) continue;
            DF v = df_mul(df_from_plane(planes[a], R.p[a]), rh[a], low_parts()[(3 + a) * BLOCK]);
            if (v.hi < 0.0f) v = {0.0f, 0.0f};
            dts[a] = v;
            if (df_less(v, dt)) dt = v;
        }
    }
    bool last = false;  // the sphere proxy ends inside this cell
    if (SPHERE) {
        if (df_less(dt, R.rem)) {
            R.rem = df_sub(R.rem, dt);
        } else {
            dt = R.rem;
            last = true;
        }
    }
    const float seg = dt.hi;
    ++R.steps;

    if (TRACE) {
        int k = R.steps - 1;
        DF t1 = two_sum(R.t.hi, dt.hi);
        t1 = fast_two_sum(t1.hi, __fadd_rn(t1.lo, __fadd_rn(R.t.lo, dt.lo)));
        if (k < kp.trace_max) {
            size_t o = (size_t)i * kp.trace_max + k;
            kp.tr_leaf[o] = R.entry_x == ENTRY_EMPTY ? -1
                                                     : __ldg(tp.leaf_ids + (size_t)stack[(L - 1) * BLOCK] * 8 + R.slot);
            kp.tr_t[2 * o] = R.t.hi;
            kp.tr_t[2 * o + 1] = t1.hi;
        }
        R.t = t1;
    }

    // advance to the exit point; snap the exit axes onto their planes.  Axes
    // whose exit lies within 2^-36 (relative) of the first one count as exits
    // too, so a ray through a shared edge or corner crosses it in one step
    // instead of leaving a sliver segment behind.  The advance comes before
    // the compositing, which does not depend on it: its double-float work
    // then overlaps the wait for the SH record (measured on the depth-10
    // luminaire: 379 -> 406 Mrays/s with FP32 leaves, 399 -> 436 with FP16;
    // a finished ray drops the advanced position).
    int l_anc = L;
    const float tie = __fmaf_rn(dt.hi, 1.4551915228366852e-11f, dt.hi);
    const float scale = pow2i(tp.depth);
    const uint32_t qmax = (1u << tp.depth) - 1u;
    bool left = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (R.d[a] != 0.0f && (df_eq(dts[a], dt) || dts[a].hi <= tie)) {
            R.p[a] = {planes[a], 0.0f};
            const uint32_t cn = R.d[a] > 0.0f ? c[a] + 1u : c[a] - 1u;
            left |= (cn >> L) != 0u;  // left the root cube (also catches 0 - 1)
            // first (d > 0) or last (d < 0) finest cell of the neighbour
            R.q[a] = R.d[a] > 0.0f ? cn << down : (c[a] << down) - 1u;
            const int diff = 32 - __clz(cn ^ c[a]);
            if (L - diff < l_anc) l_anc = L - diff;
        } else {
            R.p[a] = df_axpy(R.p[a], dt, R.d[a], low_parts()[a * BLOCK]);
            R.q[a] = quantize(R.p[a], scale, qmax, R.d[a]);
        }
    }

    // composite the leaf (Eq. 3-5)
    if (composite<K, PREC>(kp, tp, i, R, seg, sY)) return;
    if (last) {
        ray_store(kp, i, R);
        R.state = ST_IDLE;
        return;
    }
    if (R.steps >= tp.max_steps) {
        R.status = PLO_RAY_STEP_LIMIT;
        atomicOr(tp.flags, 1u);
        ray_store(kp, i, R);
        R.state = ST_IDLE;
        return;
    }
    if (left) {
        ray_store(kp, i, R);
        R.state = ST_IDLE;
        return;
    }
    R.level = l_anc;
    R.node = stack[l_anc * BLOCK];
    R.state = ST_DESCEND;
}

// Leaves a brick across the face of axis `ax` at parameter tx (from the
// brick entry point R.p): the exit point, snapped onto the planes it lies on
// (the face, and any other axis whose next plane is crossed within 2^-36
// of tx, so that a ray through an edge steps diagonally), its finest-grid
// cell from the walk's own coordinates (no rounding: the walk counted every
// plane crossed), then a descent from the deepest common ancestor of the
// brick and that cell.
__device__ __forceinline__ void brick_exit(const KParams& kp, const TreeParams& tp, int64_t i, Ray& R,
                                           uint32_t* stack, int ax, DF tx) {
    const int s = tp.brick_log;
    const uint32_t S = 1u << s;
    const int Bl = tp.top_depth;
    const float cell = pow2i(-tp.depth);
    const float tie = __fmaf_rn(tx.hi, 1.4551915228366852e-11f, tx.hi);
    bool left = false;
    int l_anc = Bl;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const uint32_t base = R.q[a] & ~(S - 1u);  // the brick's corner on this axis
        const uint32_t l = (R.loc >> (4 * a)) & 15u;
        if (R.d[a] != 0.0f && (a == ax || R.tn[a].hi <= tie)) {
            const bool up = R.d[a] > 0.0f;
            const uint32_t qn = up ? base + l + 1u : base + l - 1u;  // wraps below 0: outside the cube
            R.p[a] = {(float)(up ? qn : qn + 1u) * cell, 0.0f};
            const uint32_t cb = base >> s, cn = qn >> s;
            left |= (cn >> Bl) != 0u;
            if (cn != cb) {
                const int diff = 32 - __clz(cn ^ cb);
                if (Bl - diff < l_anc) l_anc = Bl - diff;
            }
            R.q[a] = qn;
        } else {
            R.p[a] = df_axpy(R.p[a], tx, R.d[a], low_parts()[a * BLOCK]);
            R.q[a] = base + l;
        }
    }
    if (left || l_anc < 0) {
        ray_store(kp, i, R);
        R.state = ST_IDLE;
        return;
    }
    R.level = l_anc;
    R.node = stack[l_anc * BLOCK];
    R.state = ST_DESCEND;
}

// One finest cell of a brick: the exit parameter is the smallest of the
// three next-plane parameters (a digital differential analyser); composite
// the cell over [tb, exit], then step one cell along the exit axis and load
// that cell's entry for the next iteration.
template <int K, int PREC, bool SPHERE>
__device__ void brick_step(const KParams& kp, const TreeParams& tp, int64_t i, Ray& R, uint32_t* stack,
                           const float* sY = nullptr) {
    int ax = 0;
    DF tx = R.tn[0];
    if (df_less(R.tn[1], tx)) {
        ax = 1;
        tx = R.tn[1];
    }
    if (df_less(R.tn[2], tx)) {
        ax = 2;
        tx = R.tn[2];
    }
    DF dt = df_sub(tx, R.tb);
    if (dt.hi < 0.0f) dt = {0.0f, 0.0f};
    bool last = false;  // the sphere proxy ends inside this cell
    if (SPHERE) {
        if (df_less(dt, R.rem)) {
            R.rem = df_sub(R.rem, dt);
        } else {
            dt = R.rem;
            last = true;
        }
    }
    ++R.steps;
    if (composite<K, PREC>(kp, tp, i, R, dt.hi, sY)) return;
    if (last) {
        ray_store(kp, i, R);
        R.state = ST_IDLE;
        return;
    }
    if (R.steps >= tp.max_steps) {
        R.status = PLO_RAY_STEP_LIMIT;
        atomicOr(tp.flags, 1u);
        ray_store(kp, i, R);
        R.state = ST_IDLE;
        return;
    }
    // the next plane on the exit axis is one finest cell further: add
    // 2^-D |1/d| (a power-of-two scaling of the double-float 1/d, exact)
    const float sc = pow2i(-tp.depth);
    const float rh = low_parts()[(6 + ax) * BLOCK], rl = low_parts()[(3 + ax) * BLOCK];
    const DF step = rh > 0.0f ? DF{rh * sc, rl * sc} : DF{-rh * sc, -rl * sc};
    const DF tnew = df_add(tx, step);
    const bool up = ax == 0 ? R.d[0] > 0.0f : (ax == 1 ? R.d[1] > 0.0f : R.d[2] > 0.0f);
    const int sh = 4 * ax;
    const uint32_t l = (R.loc >> sh) & 15u;
    if (up ? l + 1u < (1u << tp.brick_log) : l > 0u) {
        R.tb = tx;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a == ax) R.tn[a] = tnew;
        R.loc = up ? R.loc + (1u << sh) : R.loc - (1u << sh);
        const uint2 e = brick_entry(tp, R.node, R.loc);
        R.entry_x = e.x;
        R.entry_y = e.y;
        return;
    }
    brick_exit(kp, tp, i, R, stack, ax, tx);
}

// The trace and sphere-proxy kernels keep more per-ray state, and degree-4
// leaves (K = 25) a larger basis: 3 blocks per SM (80 registers) beats 4
// with spills for them (measured; K = 25 on the depth-10 luminaire: 217 ->
// 285 Mrays/s with FP32 leaves, 287 -> 326 with FP16).
template <int K, int PREC, bool TRACE, bool SPHERE, bool BRICKS>
__global__ void __launch_bounds__(BLOCK, (TRACE || SPHERE || K >= 25)
                                              ? 3
                                              : (BRICKS ? PLO_BRICK_MIN_BLOCKS : PLO_RENDER_MIN_BLOCKS))
    k_render(KParams kp) {
    // nodes of the top levels, staged once per (persistent) block, then the
    // node id per level of the current cell's path (top_depth + 1 rows, one
    // column per thread): dynamic shared memory sized by the tree, so that a
    // shallow tree leaves more of the SM's memory to L1
    extern __shared__ uint2 s_nodes[];
    const TreeParams& tp = kp.tree;
    for (int j = threadIdx.x; j < tp.n_top * 8; j += BLOCK) s_nodes[j] = tp.nodes[j];
    __syncthreads();
    uint32_t* stack = reinterpret_cast<uint32_t*>(s_nodes + tp.n_top * 8) + threadIdx.x;
    __shared__ float s_Y[K * BLOCK];
    float* sY = s_Y + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    const int64_t warp = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    int64_t next = 0, end = 0;  // warp-uniform range of rays being handed out
    if (!kp.cursor) {
        next = warp * kp.chunk;
        if (next >= kp.n) return;  // whole warp exits together
        end = min(next + kp.chunk, kp.n);
    }
    bool drained = false;

    Ray R;
    R.state = ST_IDLE;
    int64_t my = 0;
    for (;;) {
        // idle lanes take the next rays; rays that miss the proxy finish at
        // once, so repeat while lanes are idle and rays remain
        for (;;) {
            unsigned idle = __ballot_sync(0xffffffffu, R.state == ST_IDLE);
            // refill in groups: ray setup runs with at least 4 lanes (or when
            // no ray is left in flight; 4 measured faster than 8 and 16)
            if (idle == 0u || (__popc(idle) < 4 && idle != 0xffffffffu)) break;
            if (next >= end) {
                if (!kp.cursor || drained) break;
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(kp.cursor, (unsigned long long)RENDER_CLAIM);
                b = __shfl_sync(0xffffffffu, b, 0);
                if ((int64_t)b >= kp.n) {
                    drained = true;
                    break;
                }
                next = (int64_t)b;
                end = min(next + RENDER_CLAIM, kp.n);
            }
            int64_t cand = next + __popc(idle & lanes_below);
            next += __popc(idle);
            if (R.state == ST_IDLE && cand < end) {
                my = cand;
                ray_begin<TRACE, SPHERE>(kp, tp, my, R, stack);
                if (R.state != ST_IDLE) {
                    float Y[K];
                    sh_basis<K>(R.dirn[0], R.dirn[1], R.dirn[2], Y);
#pragma unroll
                    for (int k = 0; k < K; ++k) sY[k * BLOCK] = Y[k];
                }
            }
        }
        const unsigned live = __ballot_sync(0xffffffffu, R.state != ST_IDLE);
        if (live == 0u) break;
        // every live lane is at a leaf, in a brick, or part-way down a
        // descent longer than one step allows
        if (BRICKS && R.state == ST_BRICK) brick_step<K, PREC, SPHERE>(kp, tp, my, R, stack, sY);
        if (R.state == ST_LEAF) leaf_step<K, PREC, TRACE, SPHERE>(kp, tp, my, R, stack, sY);
        if (R.state == ST_DESCEND) descend_step<BRICKS, PREC>(tp, s_nodes, R, stack);
    }
}

// ---------------------------------------------------------------- batched render
// Several luminaires in one launch: rays of tree t occupy [off[t], off[t+1])
// of one concatenated array.  Persistent warps claim `claim` rays at a time
// from a global cursor (one queue for all trees, so uneven ray counts
// balance themselves); lanes refill from the warp's claim as in k_render.
// Leaf precision and SH degree are read from the tree table per ray.
constexpr int MAX_BATCH = 16;
constexpr int BATCH_TOP_NODES = 73;  // levels 0..2 of a full octree

struct BatchParams {
    KParams base;  // render parameters and outputs (base.tree unused)
    TreeParams trees[MAX_BATCH];
    int64_t off[MAX_BATCH + 1];
    int32_t n_trees;
    int32_t claim;
    int32_t stack_off;           // entries (uint2) of staged nodes before the node stack
    unsigned long long* cursor;  // zeroed before each launch
};

template <bool BRICKS>
__global__ void __launch_bounds__(BLOCK, BRICKS ? PLO_BRICK_MIN_BLOCKS : PLO_RENDER_MIN_BLOCKS)
    k_render_batch(BatchParams bp) {
    extern __shared__ uint2 s_nodes[];
    __shared__ TreeParams s_tp[MAX_BATCH];
    __shared__ long long s_off[MAX_BATCH + 1];
    if (threadIdx.x < bp.n_trees) s_tp[threadIdx.x] = bp.trees[threadIdx.x];
    if (threadIdx.x <= bp.n_trees) s_off[threadIdx.x] = bp.off[threadIdx.x];
    for (int t = 0; t < bp.n_trees; ++t) {
        const TreeParams& tp = bp.trees[t];
        for (int j = threadIdx.x; j < tp.n_top * 8; j += BLOCK) s_nodes[tp.s_off + j] = tp.nodes[j];
    }
    __syncthreads();
    const KParams& kp = bp.base;
    const long long total = s_off[bp.n_trees];
    // per-thread node stack after the staged nodes (bp.stack_rows rows)
    uint32_t* stack = reinterpret_cast<uint32_t*>(s_nodes + bp.stack_off) + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const unsigned lanes_below = (1u << lane) - 1u;

    Ray R;
    R.state = ST_IDLE;
    R.tree = 0;
    int64_t my = 0;
    long long next = 0, end = 0;  // the warp's current claim (warp-uniform)
    bool drained = false;
    for (;;) {
        for (;;) {
            unsigned idle = __ballot_sync(0xffffffffu, R.state == ST_IDLE);
            // refill in groups of at least 8 lanes
            if (idle == 0u || (__popc(idle) < 8 && idle != 0xffffffffu)) break;
            if (next >= end) {
                if (drained) break;
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(bp.cursor, (unsigned long long)bp.claim);
                base = __shfl_sync(0xffffffffu, base, 0);
                if ((long long)base >= total) {
                    drained = true;
                    break;
                }
                next = (long long)base;
                end = min((long long)base + bp.claim, total);
            }
            const long long cand = next + __popc(idle & lanes_below);
            next += __popc(idle);
            if (R.state == ST_IDLE && cand < end) {
                my = cand;
                int t = 0;
                while (t + 1 < bp.n_trees && s_off[t + 1] <= cand) ++t;
                R.tree = t;
                ray_begin<false, false>(kp, s_tp[t], my, R, stack);
            }
        }
        const unsigned live = __ballot_sync(0xffffffffu, R.state != ST_IDLE);
        if (live == 0u) break;
        const TreeParams& tp = s_tp[R.tree];
        if (BRICKS && R.state == ST_BRICK) brick_step<0, -1, false>(kp, tp, my, R, stack);
        if (R.state == ST_LEAF) leaf_step<0, -1, false, false>(kp, tp, my, R, stack);
        if (R.state == ST_DESCEND) descend_step<BRICKS, -1>(tp, s_nodes, R, stack);
    }
}

// Point -> leaf lookup: descent from the root with the same tie rule.
__global__ void k_lookup(const uint2* nodes, const int32_t* leaf_ids, int depth, const float* pts, const float* dirs,
                         int64_t n, int64_t* out_leaf, int32_t* out_level) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float p[3], d[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p[a] = pts[3 * i + a];
        if (dirs) d[a] = dirs[3 * i + a];
    }
    int64_t res = -2;
    int lev = 0;
    if (p[0] >= 0.0f && p[0] <= 1.0f && p[1] >= 0.0f && p[1] <= 1.0f && p[2] >= 0.0f && p[2] <= 1.0f) {
        uint32_t node = 0, c[3] = {0, 0, 0};
        for (lev = 0; lev < depth;) {
            float sc = pow2i(-(lev + 1));
            int slot = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float m = (float)(2u * c[a] + 1u) * sc;
                int up = p[a] > m || (p[a] == m && d[a] >= 0.0f);
                c[a] = 2u * c[a] + up;
                slot |= up << a;
            }
            uint2 e = __ldg(nodes + (size_t)node * 8 + slot);
            ++lev;
            if (e.x == ENTRY_EMPTY) {
                res = -1;
                break;
            }
            if (e.x & LEAF_BIT) {
                res = __ldg(leaf_ids + (size_t)node * 8 + slot);
                break;
            }
            node = e.x;
        }
    }
    out_leaf[i] = res;
    if (out_level) out_level[i] = lev;
}

// Persistent grid: as many blocks as fit on the device at once (occupancy
// API), each warp owning a contiguous chunk of the rays.
template <int K, int PREC, bool TRACE, bool SPHERE, bool BRICKS>
cudaError_t launch_k(KParams kp, int sm_count, size_t smem, cudaStream_t s) {
    auto fn = k_render<K, PREC, TRACE, SPHERE, BRICKS>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BLOCK, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t warps_needed = (kp.n + 31) / 32;
    int64_t grid = (warps_needed + WARPS - 1) / WARPS;
    int64_t max_grid = (int64_t)sm_count * per_sm;
    if (grid > max_grid) grid = max_grid;
    int64_t total_warps = grid * WARPS;
    kp.chunk = (kp.n + total_warps - 1) / total_warps;
    fn<<<(unsigned)grid, BLOCK, smem, s>>>(kp);
    return cudaGetLastError();
}

template <bool TRACE, bool SPHERE, bool BRICKS>
cudaError_t dispatch(const plo_tree* t, const KParams& kp, size_t smem, cudaStream_t s) {
#define PLO_CASE(KK, PP)                                                   \
    if (t->K == KK && t->precision == PP) return launch_k<KK, PP, TRACE, SPHERE, BRICKS>(kp, t->sm_count, smem, s);
    PLO_CASE(1, PLO_PREC_FP32) PLO_CASE(4, PLO_PREC_FP32) PLO_CASE(9, PLO_PREC_FP32) PLO_CASE(16, PLO_PREC_FP32)
    PLO_CASE(1, PLO_PREC_FP16) PLO_CASE(4, PLO_PREC_FP16) PLO_CASE(9, PLO_PREC_FP16) PLO_CASE(16, PLO_PREC_FP16)
    PLO_CASE(1, PLO_PREC_BF16) PLO_CASE(4, PLO_PREC_BF16) PLO_CASE(9, PLO_PREC_BF16) PLO_CASE(16, PLO_PREC_BF16)
    PLO_CASE(25, PLO_PREC_FP32) PLO_CASE(25, PLO_PREC_FP16) PLO_CASE(25, PLO_PREC_BF16)
#undef PLO_CASE
    return cudaErrorInvalidValue;
}

// Kernel view of a tree.  `walk_bricks`: the brick layout's top tree and
// bricks (render kernels); otherwise the octree node table (trace, and
// trees packed with the octree layout).
void fill_tree_params(const plo_tree* t, const plo_render_params* p, TreeParams* tp, bool walk_bricks = true) {
    const bool bricks = walk_bricks && t->layout == PLO_LAYOUT_BRICKS;
    tp->nodes = static_cast<const uint2*>(bricks ? t->d_top : t->d_nodes);
    tp->bricks = bricks ? static_cast<const uint2*>(t->d_bricks) : nullptr;
    tp->brick_log = bricks ? t->brick_log : 0;
    tp->top_depth = bricks ? t->brick_level : t->depth;
    tp->leaf_ids = t->d_leaf_ids;
    tp->sh = static_cast<const uint8_t*>(t->d_sh);
    tp->flags = t->d_flags;
    tp->sh_stride = t->sh_stride;
    tp->depth = t->depth;
    tp->n_top = bricks ? t->n_top_staged : t->n_top;
    tp->s_off = 0;
    tp->K = t->K;
    tp->prec = t->precision;
    tp->max_steps = p->max_steps > 0 ? p->max_steps : 4 * (1 << t->depth) + 64;
    for (int a = 0; a < 3; ++a) {
        tp->bmin[a] = t->bbox_min[a];
        tp->inv_ext[a] = t->inv_ext[a];
        tp->inv_ext_lo[a] = t->inv_ext_lo[a];
    }
}

plo_status check_params(const plo_render_params* p) {
    if (!p) return set_error(PLO_ERR_INVALID_ARG, "params is NULL");
    if (p->transmittance < PLO_TRANS_EXP || p->transmittance > PLO_TRANS_LINEAR_LITERAL)
        return set_error(PLO_ERR_INVALID_ARG, "unknown transmittance model");
    if (p->activation != PLO_ACT_RELU && p->activation != PLO_ACT_SIGMOID)
        return set_error(PLO_ERR_INVALID_ARG, "unknown activation");
    if (!(p->t_stop >= 0.0f && p->t_stop <= 1.0f)) return set_error(PLO_ERR_INVALID_ARG, "t_stop must be in [0, 1]");
    if (!(p->sigma_min >= 0.0f) || !std::isfinite(p->sigma_min))
        return set_error(PLO_ERR_INVALID_ARG, "sigma_min must be finite and >= 0");
    if (p->activation == PLO_ACT_SIGMOID && !std::isfinite(p->l_max))
        return set_error(PLO_ERR_INVALID_ARG, "l_max must be finite");
    if (p->max_steps < 0) return set_error(PLO_ERR_INVALID_ARG, "max_steps must be >= 0");
    if (p->saturate != 0 && p->saturate != 1) return set_error(PLO_ERR_INVALID_ARG, "saturate must be 0 or 1");
    if (p->proxy != PLO_PROXY_BOX && p->proxy != PLO_PROXY_SPHERE)
        return set_error(PLO_ERR_INVALID_ARG, "unknown proxy");
    if (p->proxy == PLO_PROXY_SPHERE) {
        for (int a = 0; a < 4; ++a)
            if (!std::isfinite(p->sphere[a])) return set_error(PLO_ERR_INVALID_ARG, "sphere must be finite");
        if (!(p->sphere[3] > 0.0f)) return set_error(PLO_ERR_INVALID_ARG, "sphere radius must be > 0");
    }
    return PLO_OK;
}


// ---------------------------------------------------------------- ray order
// Large wavefronts are rendered in an order that groups rays entering the
// proxy box near each other: a counting sort by the Morton code of the
// entry point's cell on a 32^3 grid of the box (rays that miss it or are
// invalid are spread over the bins) moves the rays into a scratch copy, the render
// kernel runs on the copy unchanged, and its outputs are moved back.
// Neighbouring rays then walk neighbouring cells, so a warp's lanes share
// node and record loads in L1 and L2 (measured on the 16M room rays of the
// depth-10 tree, rays pre-sorted: 336.6 -> 356.6 Mrays/s with FP32 leaves,
// 386.7 -> 400.8 with FP16; finer keys gained no more).  The sort keeps its
// histograms in shared memory: one block per SM counts its contiguous chunk
// of rays, a scan of the (bin, block) table gives every block its slot in
// every bin, and the block scatters its chunk with shared-memory counters
// (a sort with global atomics cost 2.5 ms per 16M rays, more than it
// saved).  Each ray's result does not depend on the order.
constexpr int ORDER_BITS = 5;                       // cells per axis: 2^5
constexpr int ORDER_BINS = 1 << (3 * ORDER_BITS);  // 32768
constexpr int ORDER_THREADS = 1024;
constexpr size_t ORDER_SMEM = (size_t)ORDER_BINS * 4;  // one counter per bin

__device__ __forceinline__ uint32_t order_spread(uint32_t x) {
    uint32_t r = 0;
#pragma unroll
    for (int b = 0; b < ORDER_BITS; ++b) r |= ((x >> b) & 1u) << (3 * b);
    return r;
}

// Bin of a world-space ray: Morton code of the cell where it enters the
// unit cube of the tree (its origin's cell if it starts inside).  Rays that
// miss it (or are invalid) finish at once wherever they are, so they are
// spread over the bins by their index instead of piling into one shared
// counter (a path tracer's wavefront is mostly misses).
__device__ __forceinline__ uint32_t order_bin(const float* q, int64_t i, float3 bmin, float3 inv_ext) {
    const float bm[3] = {bmin.x, bmin.y, bmin.z}, ie[3] = {inv_ext.x, inv_ext.y, inv_ext.z};
    float u[3], du[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = (__ldg(q + a) - bm[a]) * ie[a];
        du[a] = __ldg(q + 3 + a) * ie[a];
        ok &= isfinite(u[a]) && isfinite(du[a]);
    }
    float tn = 0.0f, tf = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (du[a] == 0.0f) {
            ok &= u[a] >= 0.0f && u[a] <= 1.0f;
            continue;
        }
        const float t0 = -u[a] / du[a], t1 = (1.0f - u[a]) / du[a];
        tn = fmaxf(tn, fminf(t0, t1));
        tf = fminf(tf, fmaxf(t0, t1));
    }
    if (!ok || !(tn <= tf)) return (uint32_t)i & (uint32_t)(ORDER_BINS - 1);
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float e = fminf(fmaxf(__fmaf_rn(tn, du[a], u[a]), 0.0f), 1.0f) * (float)(1 << ORDER_BITS);
        c[a] = min((uint32_t)e, (1u << ORDER_BITS) - 1u);
    }
    return order_spread(c[0]) | (order_spread(c[1]) << 1) | (order_spread(c[2]) << 2);
}

// Block b counts the bins of rays [b chunk, (b+1) chunk): bins[i], and
// table[bin * gridDim.x + b] = its count of that bin.
__global__ void __launch_bounds__(ORDER_THREADS) k_order_count(const float* rays, int64_t n, int64_t chunk,
                                                               float3 bmin, float3 inv_ext, uint16_t* bins,
                                                               uint32_t* table) {
    extern __shared__ uint32_t s_cnt[];
    for (int j = threadIdx.x; j < ORDER_BINS; j += ORDER_THREADS) s_cnt[j] = 0u;
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(beg + chunk, n);
    for (int64_t i = beg + threadIdx.x; i < end; i += ORDER_THREADS) {
        const uint32_t b = order_bin(rays + 6 * i, i, bmin, inv_ext);
        bins[i] = (uint16_t)b;
        atomicAdd(s_cnt + b, 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < ORDER_BINS; j += ORDER_THREADS) table[(size_t)j * gridDim.x + blockIdx.x] = s_cnt[j];
}

// After the exclusive scan of the table: block b gives each ray of its chunk
// the next free position of its bin's slot: order[pos] = i, inv[i] = pos.
__global__ void __launch_bounds__(ORDER_THREADS) k_order_scatter(int64_t n, int64_t chunk, const uint16_t* bins,
                                                                 const uint32_t* table, uint32_t* order,
                                                                 uint32_t* inv) {
    extern __shared__ uint32_t s_pos[];
    for (int j = threadIdx.x; j < ORDER_BINS; j += ORDER_THREADS) s_pos[j] = table[(size_t)j * gridDim.x + blockIdx.x];
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(beg + chunk, n);
    for (int64_t i = beg + threadIdx.x; i < end; i += ORDER_THREADS) {
        const uint32_t pos = atomicAdd(s_pos + bins[i], 1u);
        order[pos] = (uint32_t)i;
        inv[i] = pos;
    }
}

// The rays in order: rays_s[pos] = rays[order[pos]] (writes in order, so
// only the reads are scattered).
__global__ void k_order_rays(const float* rays, int64_t n, const uint32_t* order, float* rays_s) {
    const int64_t pos = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (pos >= n) return;
    const float* src = rays + 6 * (int64_t)__ldg(order + pos);  // the caller's rays are only 4-byte aligned
    float* dst = rays_s + 6 * pos;
#pragma unroll
    for (int k = 0; k < 6; ++k) dst[k] = __ldg(src + k);
}

// The outputs back in ray order: ray i's from position inv[i] (writes in
// ray order, reads scattered).
__global__ void k_order_outputs(const uint32_t* inv, int64_t n, const float* rgb_s, const float* T_s,
                                const int32_t* st_s, float* rgb, float* T, int32_t* st) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const int64_t pos = __ldg(inv + i);
    rgb[3 * i] = __ldg(rgb_s + 3 * pos);
    rgb[3 * i + 1] = __ldg(rgb_s + 3 * pos + 1);
    rgb[3 * i + 2] = __ldg(rgb_s + 3 * pos + 2);
    T[i] = __ldg(T_s + pos);
    if (st) st[i] = __ldg(st_s + pos);
}

// ---------------------------------------------------------------- work distribution
// Large wavefronts are handed out dynamically: warps claim RENDER_CLAIM rays
// at a time from a counter allocated for the call, so a warp whose rays are
// long does not hold up the end of the launch (static per-warp chunks are
// kept below DYNAMIC_MIN_RAYS, where a call must not allocate).
constexpr int64_t DYNAMIC_MIN_RAYS = (int64_t)1 << 20;
// Wavefronts of at least this many rays are also put in entry-cell order
// (above): its fixed cost (a 5M-entry table per call) outweighs the gain on
// smaller ones (measured on 2M rays of the depth-9 tree: 497 -> 468
// Mrays/s with the order).
constexpr int64_t ORDER_MIN_RAYS = (int64_t)1 << 23;

template <bool TRACE>
plo_status render_common(const plo_tree* t, const float* d_rays, int64_t n, const plo_render_params* p,
                         float* d_rgb, float* d_T, int32_t* d_status, int32_t trace_max, int64_t* tr_leaf,
                         float* tr_t, int32_t* tr_count, void* stream) {
    if (!t) return set_error(PLO_ERR_INVALID_ARG, "tree is NULL");
    plo_status st = check_params(p);
    if (st != PLO_OK) return st;
    if (n < 0) return set_error(PLO_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return PLO_OK;
    if (!d_rays || !d_rgb || !d_T) return set_error(PLO_ERR_INVALID_ARG, "rays, rgb or T is NULL");
    if (TRACE && (trace_max <= 0 || !tr_leaf || !tr_t || !tr_count))
        return set_error(PLO_ERR_INVALID_ARG, "trace buffers are NULL or max_cells <= 0");
    if (TRACE && p->proxy != PLO_PROXY_BOX)
        return set_error(PLO_ERR_UNSUPPORTED, "plo_trace_rays follows the box proxy only");
    KParams kp{};
    fill_tree_params(t, p, &kp.tree, !TRACE);
    kp.transmittance = p->transmittance;
    kp.activation = p->activation;
    kp.l_max = p->l_max;
    kp.t_stop = p->t_stop;
    kp.sigma_min = p->sigma_min;
    kp.saturate = p->saturate;
    kp.proxy = p->proxy;
    for (int a = 0; a < 4; ++a) kp.sphere[a] = p->sphere[a];
    kp.rays = d_rays;
    kp.n = n;
    kp.rgb = d_rgb;
    kp.T = d_T;
    kp.status = d_status;
    kp.trace_max = trace_max;
    kp.tr_leaf = tr_leaf;
    kp.tr_t = tr_t;
    kp.tr_count = tr_count;
    // stage only the nodes of levels 0..2 (measured: the shared memory left
    // over goes to L1, which serves the deeper node loads better)
    if (kp.tree.n_top > BATCH_TOP_NODES) kp.tree.n_top = BATCH_TOP_NODES;
    size_t smem = (size_t)kp.tree.n_top * 8 * sizeof(uint2) + (size_t)(kp.tree.top_depth + 1) * BLOCK * 4;
    cudaError_t e = cudaSuccess;
    cudaStream_t cs = (cudaStream_t)stream;
    unsigned long long* cursor = nullptr;
    uint32_t* inv = nullptr;
    float *rgb_s = nullptr, *T_s = nullptr;
    int32_t* st_s = nullptr;
    const bool ordered = !TRACE && n >= ORDER_MIN_RAYS;
    if (!TRACE && n >= DYNAMIC_MIN_RAYS && !ordered) {
        e = (cudaError_t)dev_malloc_async((void**)&cursor, sizeof(unsigned long long), cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), cs);
        if (e != cudaSuccess) {
            if (cursor) cudaFreeAsync(cursor, cs);
            return cuda_error(e, "render work counter");
        }
        kp.cursor = cursor;
    }
    if (ordered) {
        // one scratch block: the claim counter, the (bin, block) table, the
        // order and its inverse, the rays and outputs in that order, each
        // ray's bin
        const int nblk = t->sm_count;
        const int64_t chunk = (n + nblk - 1) / nblk;
        auto up = [](size_t b) { return (b + 255) / 256 * 256; };
        const size_t o_table = 256, o_order = o_table + up((size_t)ORDER_BINS * nblk * 4);
        const size_t o_inv = o_order + up((size_t)n * 4);
        const size_t o_rays = o_inv + up((size_t)n * 4), o_rgb = o_rays + up((size_t)n * 24);
        const size_t o_T = o_rgb + up((size_t)n * 12), o_st = o_T + up((size_t)n * 4);
        const size_t o_bins = o_st + (d_status ? up((size_t)n * 4) : 0), total = o_bins + up((size_t)n * 2);
        e = (cudaError_t)dev_malloc_async((void**)&cursor, total, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, 256, cs);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_order_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)ORDER_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_order_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)ORDER_SMEM);
        if (e == cudaSuccess) {
            uint8_t* base = reinterpret_cast<uint8_t*>(cursor);
            uint32_t* table = reinterpret_cast<uint32_t*>(base + o_table);
            uint32_t* order = reinterpret_cast<uint32_t*>(base + o_order);
            inv = reinterpret_cast<uint32_t*>(base + o_inv);
            float* rays_s = reinterpret_cast<float*>(base + o_rays);
            rgb_s = reinterpret_cast<float*>(base + o_rgb);
            T_s = reinterpret_cast<float*>(base + o_T);
            st_s = d_status ? reinterpret_cast<int32_t*>(base + o_st) : nullptr;
            uint16_t* bins = reinterpret_cast<uint16_t*>(base + o_bins);
            const float3 bmin = make_float3(t->bbox_min[0], t->bbox_min[1], t->bbox_min[2]);
            const float3 iext = make_float3(t->inv_ext[0], t->inv_ext[1], t->inv_ext[2]);
            k_order_count<<<nblk, ORDER_THREADS, ORDER_SMEM, cs>>>(d_rays, n, chunk, bmin, iext, bins, table);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = device_exclusive_scan(table, table, (int64_t)ORDER_BINS * nblk, cs);
            if (e == cudaSuccess) {
                k_order_scatter<<<nblk, ORDER_THREADS, ORDER_SMEM, cs>>>(n, chunk, bins, table, order, inv);
                k_order_rays<<<(unsigned)((n + 255) / 256), 256, 0, cs>>>(d_rays, n, order, rays_s);
                e = cudaGetLastError();
            }
            kp.rays = rays_s;
            kp.rgb = rgb_s;
            kp.T = T_s;
            kp.status = st_s;
        }
        if (e != cudaSuccess) {
            if (cursor) cudaFreeAsync(cursor, cs);
            return cuda_error(e, "render work counter and ray order");
        }
        kp.cursor = cursor;
    }
    const bool bricks = !TRACE && t->layout == PLO_LAYOUT_BRICKS;
    if (TRACE)
        e = dispatch<TRACE, false, false>(t, kp, smem, (cudaStream_t)stream);
    else if (kp.proxy == PLO_PROXY_SPHERE)
        e = bricks ? dispatch<false, true, true>(t, kp, smem, (cudaStream_t)stream)
                   : dispatch<false, true, false>(t, kp, smem, (cudaStream_t)stream);
    else
        e = bricks ? dispatch<false, false, true>(t, kp, smem, (cudaStream_t)stream)
                   : dispatch<false, false, false>(t, kp, smem, (cudaStream_t)stream);
    if (e == cudaSuccess && inv) {
        k_order_outputs<<<(unsigned)((n + 255) / 256), 256, 0, cs>>>(inv, n, rgb_s, T_s, st_s, d_rgb, d_T, d_status);
        e = cudaGetLastError();
    }
    if (cursor) cudaFreeAsync(cursor, cs);
    if (e != cudaSuccess) return cuda_error(e, "render kernel launch");
    return PLO_OK;
}

}  // namespace
}  // namespace plo

using namespace plo;

extern "C" plo_status plo_render_rays(const plo_tree* tree, const float* d_rays, int64_t n,
                                      const plo_render_params* params, float* d_rgb, float* d_T, int32_t* d_status,
                                      void* stream) {
    return render_common<false>(tree, d_rays, n, params, d_rgb, d_T, d_status, 0, nullptr, nullptr, nullptr,
                                stream);
}

extern "C" plo_status plo_trace_rays(const plo_tree* tree, const float* d_rays, int64_t n,
                                     const plo_render_params* params, int32_t max_cells, int64_t* d_leaf,
                                     float* d_t, int32_t* d_count, void* stream) {
    // The trace runs the render kernel itself (trace instantiation); its
    // radiance goes to a stream-ordered temporary and is discarded.
    if (!tree) return set_error(PLO_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0) return set_error(PLO_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return PLO_OK;
    float* rgbT = nullptr;
    cudaError_t e = (cudaError_t)dev_malloc_async((void**)&rgbT, (size_t)n * 4 * sizeof(float), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_error(e, "trace scratch allocation");
    plo_status st = render_common<true>(tree, d_rays, n, params, rgbT, rgbT + 3 * n, nullptr, max_cells, d_leaf,
                                        d_t, d_count, stream);
    cudaFreeAsync(rgbT, (cudaStream_t)stream);
    return st;
}

extern "C" plo_status plo_lookup_points(const plo_tree* t, const float* d_points, const float* d_dirs, int64_t n,
                                        int64_t* d_leaf, int32_t* d_level, void* stream) {
    if (!t) return set_error(PLO_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0) return set_error(PLO_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return PLO_OK;
    if (!d_points || !d_leaf) return set_error(PLO_ERR_INVALID_ARG, "points or leaf output is NULL");
    int64_t grid = (n + 255) / 256;
    k_lookup<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(static_cast<const uint2*>(t->d_nodes), t->d_leaf_ids,
                                                               t->depth, d_points, d_dirs, n, d_leaf, d_level);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "lookup kernel launch");
    return PLO_OK;
}

// ---------------------------------------------------------------- allocation-free host path
// plo_render_rays_host_noalloc: the host-buffer render for callers that must
// not allocate device memory (see include/plo.h).  Its device staging for
// rays and results is the file-scope array below, so the call itself makes
// no cudaMalloc/cudaFree and no allocating library call.
namespace {

constexpr int64_t kNoAllocMaxRays = 262144;  // 10 floats per ray: 10 MiB in all
// plo_render_rays takes a stream-ordered work counter from DYNAMIC_MIN_RAYS
// rays up; every call of this path stays below that, so it never allocates.
static_assert(kNoAllocMaxRays < DYNAMIC_MIN_RAYS,
              "the allocation-free path must stay below the ray count at which plo_render_rays allocates");
// rays [max][6], then rgb [max][3], then T [max].  Every GPU that loads the
// library holds this array until the process exits.  All calls share it.
__device__ __align__(256) float g_noalloc_stage[kNoAllocMaxRays * 10];

// Device addresses of the staging array, one per CUDA context seen: a new
// primary context (after cudaDeviceReset, say) gets its own lookup instead
// of a stale address.
constexpr int kNoAllocMaxContexts = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ctx[kNoAllocMaxContexts] = {};
float* g_noalloc_ptr[kNoAllocMaxContexts] = {};
int g_noalloc_used = 0;

using CtxGetCurrentFn = int (*)(void**);  // cuCtxGetCurrent(CUcontext*)

CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    return fn;
}

// Device address of the staging array in the current context.  In host
// code g_noalloc_stage names a host-side stand-in, never the device memory,
// so only this address may be used.
plo_status noalloc_stage(float** out) {
    CtxGetCurrentFn get = ctx_get_current();
    if (!get) return set_error(PLO_ERR_CUDA, "cuCtxGetCurrent is not available from the driver");
    void* ctx = nullptr;
    if (get(&ctx) != 0 || !ctx) return set_error(PLO_ERR_CUDA, "no current CUDA context");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    for (int k = 0; k < g_noalloc_used; ++k)
        if (g_noalloc_ctx[k] == ctx) {
            *out = g_noalloc_ptr[k];
            return PLO_OK;
        }
    if (g_noalloc_used == kNoAllocMaxContexts)
        return set_error(PLO_ERR_UNSUPPORTED, "too many CUDA contexts for the allocation-free path's table");
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_stage);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress of the no-allocation staging array");
    g_noalloc_ctx[g_noalloc_used] = ctx;
    g_noalloc_ptr[g_noalloc_used] = static_cast<float*>(p);
    ++g_noalloc_used;
    *out = static_cast<float*>(p);
    return PLO_OK;
}

}  // namespace

extern "C" plo_status plo_render_rays_host_noalloc(const plo_tree* tree, const float* h_rays, int64_t n,
                                                   const plo_render_params* params, float* h_rgb, float* h_T,
                                                   void* stream) {
    if (!tree) return set_error(PLO_ERR_INVALID_ARG, "tree is NULL");
    if (n < 0) return set_error(PLO_ERR_INVALID_ARG, "n must be >= 0");
    if (n > kNoAllocMaxRays)
        return set_error(PLO_ERR_INVALID_ARG, "n = " + std::to_string(n) +
                                                  " exceeds the allocation-free path's maximum of " +
                                                  std::to_string(kNoAllocMaxRays) + " rays per call");
    if (n == 0) return PLO_OK;
    if (!h_rays || !h_rgb || !h_T) return set_error(PLO_ERR_INVALID_ARG, "rays, rgb or T is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev != tree->device)
        return set_error(PLO_ERR_INVALID_ARG, "the tree lives on another device than the current one");
    float* base = nullptr;
    plo_status st = noalloc_stage(&base);
    if (st != PLO_OK) return st;
    float* d_rays = base;
    float* d_rgb = base + 6 * kNoAllocMaxRays;
    float* d_T = base + 9 * kNoAllocMaxRays;
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(d_rays, h_rays, (size_t)n * 6 * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "host-to-device ray copy");
    st = plo_render_rays(tree, d_rays, n, params, d_rgb, d_T, nullptr, stream);
    if (st != PLO_OK) return st;
    e = cudaMemcpyAsync(h_rgb, d_rgb, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_T, d_T, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "plo_render_rays_host_noalloc");
    return PLO_OK;
}

// ---------------------------------------------------------------- batch handle
struct plo_batch {
    BatchParams bp;
    int32_t n_trees;
    int64_t n_rays;
    size_t smem;
    int sm_count;
    int device;
    plo_batch_config cfg;
    int32_t full_top[MAX_BATCH];  // stageable top nodes per tree (<= BATCH_TOP_NODES)
    bool bricks;                  // some tree uses the brick layout
    unsigned long long* d_cursor;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

void apply_config(plo_batch* b) {
    int32_t off = 0;
    for (int t = 0; t < b->n_trees; ++t) {
        const int32_t n = b->cfg.top_nodes > 0 ? std::min(b->full_top[t], b->cfg.top_nodes) : 0;
        b->bp.trees[t].n_top = n;
        b->bp.trees[t].s_off = off;
        off += n * 8;
    }
    int rows = 1;
    for (int t = 0; t < b->n_trees; ++t) rows = std::max(rows, b->bp.trees[t].top_depth + 1);
    b->bp.stack_off = off;
    b->smem = (size_t)off * sizeof(uint2) + (size_t)rows * BLOCK * 4;
    b->bp.claim = b->cfg.claim_rays;
}

void (*batch_kernel(const plo_batch* b))(BatchParams) {
    return b->bricks ? k_render_batch<true> : k_render_batch<false>;
}

cudaError_t launch_batch(plo_batch* b, cudaStream_t s) {
    auto fn = batch_kernel(b);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BLOCK, b->smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int bps = b->cfg.blocks_per_sm > 0 && b->cfg.blocks_per_sm < per_sm ? b->cfg.blocks_per_sm : per_sm;
    int64_t warps_needed = (b->n_rays + 31) / 32;
    int64_t grid = std::min<int64_t>((warps_needed + WARPS - 1) / WARPS, (int64_t)b->sm_count * bps);
    if (grid < 1) return cudaSuccess;
    e = cudaMemsetAsync(b->d_cursor, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    fn<<<(unsigned)grid, BLOCK, b->smem, s>>>(b->bp);
    return cudaGetLastError();
}

void set_buffers(plo_batch* b, const float* d_rays, float* d_rgb, float* d_T, int32_t* d_status) {
    b->bp.base.rays = d_rays;
    b->bp.base.rgb = d_rgb;
    b->bp.base.T = d_T;
    b->bp.base.status = d_status;
}

void drop_graph(plo_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

}  // namespace

extern "C" plo_status plo_batch_create(const plo_tree* const* trees, int32_t n_trees, const int64_t* ray_offsets,
                                       const plo_render_params* params, plo_batch** out) {
    if (!out) return set_error(PLO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!trees || !ray_offsets) return set_error(PLO_ERR_INVALID_ARG, "trees or ray_offsets is NULL");
    if (n_trees < 1 || n_trees > MAX_BATCH)
        return set_error(PLO_ERR_INVALID_ARG, "n_trees must be in [1, " + std::to_string(MAX_BATCH) + "]");
    plo_status st = check_params(params);
    if (st != PLO_OK) return st;
    if (params->proxy != PLO_PROXY_BOX)
        return set_error(PLO_ERR_UNSUPPORTED, "the batch render clips to each tree's box (PLO_PROXY_BOX only)");
    if (ray_offsets[0] != 0) return set_error(PLO_ERR_INVALID_ARG, "ray_offsets[0] must be 0");
    for (int t = 0; t < n_trees; ++t) {
        if (!trees[t]) return set_error(PLO_ERR_INVALID_ARG, "a tree is NULL");
        if (ray_offsets[t + 1] < ray_offsets[t]) return set_error(PLO_ERR_INVALID_ARG, "ray_offsets must not decrease");
        if (t > 0 && trees[t]->device != trees[0]->device)
            return set_error(PLO_ERR_INVALID_ARG, "all trees must live on one device");
    }
    plo_batch* b = new (std::nothrow) plo_batch();
    if (!b) return set_error(PLO_ERR_OOM, "host allocation failed");
    b->n_trees = n_trees;
    b->n_rays = ray_offsets[n_trees];
    b->device = trees[0]->device;
    b->sm_count = trees[0]->sm_count;
    KParams& kp = b->bp.base;
    kp.transmittance = params->transmittance;
    kp.activation = params->activation;
    kp.l_max = params->l_max;
    kp.t_stop = params->t_stop;
    kp.sigma_min = params->sigma_min;
    kp.saturate = params->saturate;
    kp.proxy = PLO_PROXY_BOX;
    kp.n = b->n_rays;
    for (int t = 0; t < n_trees; ++t) {
        fill_tree_params(trees[t], params, &b->bp.trees[t]);
        b->bricks |= trees[t]->layout == PLO_LAYOUT_BRICKS;
        b->full_top[t] = std::min<int32_t>(b->bp.trees[t].n_top, BATCH_TOP_NODES);
    }
    for (int t = 0; t <= n_trees; ++t) b->bp.off[t] = ray_offsets[t];
    b->bp.n_trees = n_trees;
    b->cfg = {256, 0, BATCH_TOP_NODES};
    apply_config(b);
    int e = dev_malloc((void**)&b->d_cursor, 256);
    if (e != 0) {
        delete b;
        return cuda_error(e, "batch cursor allocation");
    }
    b->bp.cursor = b->d_cursor;
    *out = b;
    return PLO_OK;
}

extern "C" void plo_batch_free(plo_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    drop_graph(b);
    cudaFree(b->d_cursor);
    delete b;
}

extern "C" plo_status plo_batch_set_config(plo_batch* b, const plo_batch_config* cfg) {
    if (!b || !cfg) return set_error(PLO_ERR_INVALID_ARG, "batch or config is NULL");
    if (cfg->claim_rays < 32 || cfg->claim_rays > (1 << 20) || cfg->claim_rays % 32)
        return set_error(PLO_ERR_INVALID_ARG, "claim_rays must be a multiple of 32 in [32, 2^20]");
    if (cfg->blocks_per_sm < 0 || cfg->top_nodes < 0 || cfg->top_nodes > BATCH_TOP_NODES)
        return set_error(PLO_ERR_INVALID_ARG, "blocks_per_sm must be >= 0, top_nodes in [0, 73]");
    b->cfg = *cfg;
    apply_config(b);
    drop_graph(b);
    return PLO_OK;
}

extern "C" plo_status plo_batch_get_config(const plo_batch* b, plo_batch_config* cfg) {
    if (!b || !cfg) return set_error(PLO_ERR_INVALID_ARG, "batch or config is NULL");
    *cfg = b->cfg;
    return PLO_OK;
}

extern "C" plo_status plo_batch_render(plo_batch* b, const float* d_rays, float* d_rgb, float* d_T,
                                       int32_t* d_status, void* stream) {
    if (!b) return set_error(PLO_ERR_INVALID_ARG, "batch is NULL");
    if (b->n_rays == 0) return PLO_OK;
    if (!d_rays || !d_rgb || !d_T) return set_error(PLO_ERR_INVALID_ARG, "rays, rgb or T is NULL");
    set_buffers(b, d_rays, d_rgb, d_T, d_status);
    cudaError_t e = launch_batch(b, (cudaStream_t)stream);
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "batch render launch");
}

extern "C" plo_status plo_batch_capture(plo_batch* b, const float* d_rays, float* d_rgb, float* d_T,
                                        int32_t* d_status, void* stream) {
    if (!b) return set_error(PLO_ERR_INVALID_ARG, "batch is NULL");
    if (!d_rays || !d_rgb || !d_T) return set_error(PLO_ERR_INVALID_ARG, "rays, rgb or T is NULL");
    drop_graph(b);
    set_buffers(b, d_rays, d_rgb, d_T, d_status);
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_error(e, "capture stream");
    // the occupancy query and attribute set happen outside the capture
    e = cudaFuncSetAttribute(batch_kernel(b), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = launch_batch(b, cs);
        e = cudaStreamEndCapture(cs, &b->graph);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    (void)stream;
    if (e != cudaSuccess) {
        drop_graph(b);
        return cuda_error(e, "batch graph capture");
    }
    return PLO_OK;
}

extern "C" plo_status plo_batch_replay(plo_batch* b, void* stream) {
    if (!b) return set_error(PLO_ERR_INVALID_ARG, "batch is NULL");
    if (!b->exec) return set_error(PLO_ERR_INVALID_ARG, "no captured graph: call plo_batch_capture first");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? PLO_OK : cuda_error(e, "batch graph launch");
}

extern "C" plo_status plo_batch_autotune(plo_batch* b, const float* d_rays, float* d_rgb, float* d_T, int32_t reps,
                                         void* stream, plo_batch_config* best_out, float* best_ms) {
    if (!b || !best_out) return set_error(PLO_ERR_INVALID_ARG, "batch or output is NULL");
    if (!d_rays || !d_rgb || !d_T) return set_error(PLO_ERR_INVALID_ARG, "rays, rgb or T is NULL");
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    set_buffers(b, d_rays, d_rgb, d_T, nullptr);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const plo_batch_config saved = b->cfg;
    plo_batch_config best = saved;
    float best_t = 1e30f;
    const int claims[] = {32, 64, 128, 256, 1024};
    const int bpss[] = {0, 1, 2};
    const int tops[] = {0, BATCH_TOP_NODES};
    cudaError_t err = cudaSuccess;
    for (int ci = 0; ci < 5 && err == cudaSuccess; ++ci)
        for (int bi = 0; bi < 3 && err == cudaSuccess; ++bi)
            for (int ti = 0; ti < 2 && err == cudaSuccess; ++ti) {
                b->cfg = {claims[ci], bpss[bi], tops[ti]};
                apply_config(b);
                err = launch_batch(b, s);  // warm-up
                if (err != cudaSuccess) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && err == cudaSuccess; ++r) err = launch_batch(b, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= (float)reps;
                if (ms < best_t) {
                    best_t = ms;
                    best = b->cfg;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cfg = err == cudaSuccess ? best : saved;
    apply_config(b);
    drop_graph(b);
    if (err != cudaSuccess) return cuda_error(err, "batch autotune");
    *best_out = best;
    if (best_ms) *best_ms = best_t;
    return PLO_OK;
}
