// Layer-fused forward of the network's trunk (Sec. 4.2: eight fully
// connected layers of 256 with ReLU) on sm_103a: a 128-row tile's
// activations stay in shared memory from the encoded input to the eighth
// layer's output; only what the backward pass needs leaves the SM (each
// layer's bf16 output, stored by TMA straight from the shared-memory tile,
// and its ReLU bits).
//
// Per CTA (persistent, one per SM) two tiles are in flight, in slots 0 and
// 1, each with its own 64 KB activation buffer and 256 TMEM columns; the
// jobs (slot, layer) run in the order A0 B0 A1 B1 ... A7 B7, so the
// epilogue of one slot overlaps the MMAs of the other.  The weights stream
// from L2 through a ring of three 32 KB stages (one K-block of 64 inputs of
// the 256 x K matrix each), in the same job order.
//
// Warp roles: 0 lane 0 TMA loads (input tiles, weights), 1 TMEM owner and
// MMA issuer (lane 0), 2 lane 0 TMA stores of the finished activation
// tiles, 4..19 the epilogue (warp w reads TMEM lanes 32 (w % 4) .. +31 and
// a quarter of the 32-column chunks; 16 warps measured 2.60 -> 2.54 ms per
// training step against 8).  The epilogue writes its bf16 results into
// the activation buffer in the layout a 128-byte-swizzled TMA load would
// produce (row r's 16-byte chunk c at r * 128 + ((c ^ (r & 7)) * 16) of
// its 64-column block), so the next layer's MMA and the TMA store read it
// as they read TMA-loaded tiles.  Every mbarrier wait is bounded, as in
// k_gemm: a wait that gives up raises the abort flag and bit 1 of the error
// word, and every role drains what it has in flight.
#pragma once

#include "gemm.cuh"

namespace plo {
namespace gemm {

constexpr int TR_LAYERS = 8;
constexpr int TR_N = 256;
constexpr int TR_WSTAGES = 3;
constexpr int TR_WBYTES = TR_N * 128;          // one K-block of a weight matrix: 256 rows x 128 B
constexpr int TR_KBYTES = BM * 128;            // one K-block of an activation tile: 128 rows x 128 B
constexpr int TR_ABYTES = 4 * TR_KBYTES;       // a 128 x 256 bf16 activation tile
constexpr int TR_EPI_WARP0 = 4;
constexpr int TR_EPI_GROUPS = 4;                      // epilogue warps per TMEM lane quadrant
constexpr int TR_CHUNKS = TR_N / 32 / TR_EPI_GROUPS;  // 32-column chunks per epilogue warp
constexpr int TR_THREADS = 32 * TR_EPI_WARP0 + 128 * TR_EPI_GROUPS;
__host__ __device__ constexpr size_t trunk_smem_bytes() {
    return 1024 + 2 * (size_t)TR_ABYTES + (size_t)TR_WSTAGES * TR_WBYTES + 256;
}

// Indexed by job j of a tile: the forward's layer j (j = 0..7), or in the
// backward chain the data gradient through layer l = 7 - j (j = 0..6).
struct TrunkMaps {
    CUtensorMap x;                 // input tile, boxes 64 x 128, 128-byte swizzle: the encoded
                                   // samples [M][64] (forward), d loss / d Z_7 [M][256] (backward)
    CUtensorMap w[TR_LAYERS];      // B operand [256][K], boxes 64 x 256: W_j (forward), W_l^T (backward)
    CUtensorMap h[TR_LAYERS];      // job j's output [M][256], boxes 64 x 128 (TMA stores)
};

struct TrunkArgs {
    const float* bias[TR_LAYERS];  // forward: layer j's bias
    uint32_t* bits[TR_LAYERS];     // [M][8] words: forward, layer j's ReLU bits (written, nullable);
                                   // backward, the ReLU bits of H_l (read: the mask of the gradient)
    uint32_t store;                // bit j: store job j's output through h[j]
    unsigned int* err;          // bit 1: a pipeline wait gave up
    uint32_t wait_limit;        // polls per wait (0: sm100::WAIT_LIMIT)
    int M;
};

struct TrCtl {
    uint64_t wfull[TR_WSTAGES], wempty[TR_WSTAGES];
    uint64_t xfull[2], tfull[2], aready[2], sdone[2];
    uint64_t drain;
    uint32_t tmem;
    uint32_t limit;
    int abort;
};

__device__ __forceinline__ bool tr_wait(uint64_t* bar, uint32_t ph, TrCtl* ctl, unsigned int* err) {
    const uint32_t a = sm100::smem_addr(bar);
    const uint32_t limit = ctl->limit;
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(ph)
            : "memory");
        if (done) return true;
        if ((it & 1023u) == 1023u && *(volatile int*)&ctl->abort) return false;
    }
    *(volatile int*)&ctl->abort = 1;
    atomicOr(err, 2u);
    return false;
}

// The CTA's tiles are blockIdx.x + k gridDim.x; tiles 2j and 2j + 1 of that
// list form pair j (slots 0 and 1).  Every role walks the same job list.
__device__ __forceinline__ int tr_tile(int pair, int slot, int n_tiles) {
    const int t = blockIdx.x + (2 * pair + slot) * (int)gridDim.x;
    return t < n_tiles ? t : -1;
}

// BWD: the data-gradient chain instead of the forward: per job
// dZ_{l-1} = (dZ_l W_l) masked by the ReLU bits of H_l, l = 7 .. 1, starting
// from the head's dZ_7 (four input K-blocks) with no bias.
template <bool BWD>
__global__ void __launch_bounds__(TR_THREADS, 1) k_trunk(const __grid_constant__ TrunkMaps maps, TrunkArgs a) {
    constexpr uint32_t IDESC = sm100::idesc_bf16(BM, TR_N, 0, 0);
    constexpr int NJ = BWD ? TR_LAYERS - 1 : TR_LAYERS;  // jobs per tile
    constexpr int XKB = BWD ? 4 : 1;                      // K-blocks of the input tile
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* act[2] = {smem, smem + TR_ABYTES};
    uint8_t* wbuf = smem + 2 * TR_ABYTES;
    TrCtl* ctl = reinterpret_cast<TrCtl*>(wbuf + TR_WSTAGES * TR_WBYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TR_WSTAGES; ++s) {
            sm100::mbar_init(&ctl->wfull[s], 1);
            sm100::mbar_init(&ctl->wempty[s], 1);
        }
        for (int p = 0; p < 2; ++p) {
            sm100::mbar_init(&ctl->xfull[p], 1);
            sm100::mbar_init(&ctl->tfull[p], 1);
            sm100::mbar_init(&ctl->aready[p], 32 * (TR_THREADS / 32 - TR_EPI_WARP0));
            sm100::mbar_init(&ctl->sdone[p], 1);
        }
        sm100::mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        ctl->limit = a.wait_limit ? a.wait_limit : sm100::WAIT_LIMIT;
        sm100::fence_mbar_init();
    }
    if (warp == 1) sm100::tmem_alloc(&ctl->tmem, 2 * TR_N);
    sm100::tc_fence_before();
    __syncthreads();
    sm100::tc_fence_after();
    const uint32_t tmem = ctl->tmem;
    const int n_tiles = (a.M + BM - 1) / BM;
    const int mine = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int n_pairs = (mine + 1) / 2;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA loads: input tiles and weight K-blocks, in job order
        sm100::prefetch_tmap(&maps.x);
        int ws = 0;
        uint32_t wph = 0, armed = 0, armed_ph = 0;
        int jobs[2] = {0, 0}, xs[2] = {0, 0};
        bool ok = true;
        for (int pr = 0; ok && pr < n_pairs; ++pr)
            for (int l = 0; ok && l < NJ; ++l)
                for (int p = 0; ok && p < 2; ++p) {
                    const int tile = tr_tile(pr, p, n_tiles);
                    if (tile < 0) continue;
                    if (l == 0) {
                        // the slot's buffer is free once the last store of its previous tile has read it
                        if (jobs[p] > 0 && !tr_wait(&ctl->sdone[p], (uint32_t)(jobs[p] - 1) & 1u, ctl, a.err)) {
                            ok = false;
                            break;
                        }
                        sm100::mbar_arrive_expect_tx(&ctl->xfull[p], (uint32_t)(XKB * TR_KBYTES));
                        for (int kb = 0; kb < XKB; ++kb)
                            sm100::tma_load_2d(act[p] + (size_t)kb * TR_KBYTES, &maps.x, kb * 64, tile * BM,
                                               &ctl->xfull[p]);
                        ++xs[p];
                    }
                    const int nkb = (!BWD && l == 0) ? 1 : 4;
                    for (int kb = 0; kb < nkb; ++kb) {
                        if (!tr_wait(&ctl->wempty[ws], wph ^ 1u, ctl, a.err)) {
                            ok = false;
                            break;
                        }
                        sm100::mbar_arrive_expect_tx(&ctl->wfull[ws], (uint32_t)TR_WBYTES);
                        sm100::tma_load_2d(wbuf + (size_t)ws * TR_WBYTES, &maps.w[l], kb * 64, 0, &ctl->wfull[ws]);
                        armed |= 1u << ws;
                        armed_ph = (armed_ph & ~(1u << ws)) | (wph << ws);
                        if (++ws == TR_WSTAGES) {
                            ws = 0;
                            wph ^= 1u;
                        }
                    }
                    ++jobs[p];
                }
        if (!ok) {  // drain the loads still in flight before the CTA exits
            for (int s = 0; s < TR_WSTAGES; ++s)
                if (armed & (1u << s)) sm100::mbar_wait(&ctl->wfull[s], (armed_ph >> s) & 1u);
            for (int p = 0; p < 2; ++p)
                if (xs[p] > 0) sm100::mbar_wait(&ctl->xfull[p], (uint32_t)(xs[p] - 1) & 1u);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        int ws = 0;
        uint32_t wph = 0;
        int jobs[2] = {0, 0}, xs[2] = {0, 0};
        bool ok = true, issued = false;
        for (int pr = 0; ok && pr < n_pairs; ++pr)
            for (int l = 0; ok && l < NJ; ++l)
                for (int p = 0; ok && p < 2; ++p) {
                    const int tile = tr_tile(pr, p, n_tiles);
                    if (tile < 0) continue;
                    // the input: the loaded tile, or the previous layer's output
                    const bool in = l == 0 ? tr_wait(&ctl->xfull[p], (uint32_t)(xs[p]++) & 1u, ctl, a.err)
                                           : tr_wait(&ctl->aready[p], (uint32_t)(jobs[p] - 1) & 1u, ctl, a.err);
                    if (!in) {
                        ok = false;
                        break;
                    }
                    sm100::tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(p * TR_N);
                    const int nkb = (!BWD && l == 0) ? 1 : 4;
                    for (int kb = 0; kb < nkb; ++kb) {
                        if (!tr_wait(&ctl->wfull[ws], wph, ctl, a.err)) {
                            ok = false;
                            break;
                        }
                        sm100::tc_fence_after();
                        const uint32_t a0 = sm100::smem_addr(act[p] + (size_t)kb * TR_KBYTES);
                        const uint32_t b0 = sm100::smem_addr(wbuf + (size_t)ws * TR_WBYTES);
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k) {
                            const uint64_t adesc = sm100::smem_desc_sw128(a0 + 32 * k, 16, 1024);
                            const uint64_t bdesc = sm100::smem_desc_sw128(b0 + 32 * k, 16, 1024);
                            sm100::mma_bf16(d, adesc, bdesc, IDESC, (kb | k) != 0);
                        }
                        issued = true;
                        sm100::mma_commit(&ctl->wempty[ws]);
                        if (++ws == TR_WSTAGES) {
                            ws = 0;
                            wph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    sm100::mma_commit(&ctl->tfull[p]);
                    ++jobs[p];
                }
        if (!ok && issued) {  // let issued MMAs finish before TMEM is freed
            sm100::mma_commit(&ctl->drain);
            sm100::mbar_wait(&ctl->drain, 0);
        }
    } else if (warp == 2 && lane == 0) {
        // ---------------- TMA stores of finished activation tiles
        int jobs[2] = {0, 0};
        bool ok = true;
        for (int pr = 0; ok && pr < n_pairs; ++pr)
            for (int l = 0; ok && l < NJ; ++l)
                for (int p = 0; ok && p < 2; ++p) {
                    const int tile = tr_tile(pr, p, n_tiles);
                    if (tile < 0) continue;
                    if (!tr_wait(&ctl->aready[p], (uint32_t)jobs[p] & 1u, ctl, a.err)) {
                        ok = false;
                        break;
                    }
                    if ((a.store >> l) & 1u) {
                        for (int kb = 0; kb < 4; ++kb)
                            sm100::tma_store_2d(&maps.h[l], kb * 64, tile * BM, act[p] + (size_t)kb * TR_KBYTES);
                        sm100::bulk_commit();
                        sm100::bulk_wait_read_0();
                    }
                    sm100::mbar_arrive(&ctl->sdone[p]);
                    ++jobs[p];
                }
        sm100::bulk_wait_all();  // the stores are complete before the CTA exits
    } else if (warp >= TR_EPI_WARP0) {
        // ---------------- epilogue: bias + ReLU -> bf16 into the slot's buffer, ReLU bits
        const int q = warp & 3;
        const int grp = (warp - TR_EPI_WARP0) >> 2;
        const int rl = q * 32 + lane;  // row within the tile
        int jobs[2] = {0, 0};
        bool ok = true;
        for (int pr = 0; ok && pr < n_pairs; ++pr)
            for (int l = 0; ok && l < NJ; ++l)
                for (int p = 0; ok && p < 2; ++p) {
                    const int tile = tr_tile(pr, p, n_tiles);
                    if (tile < 0) continue;
                    if (!tr_wait(&ctl->tfull[p], (uint32_t)jobs[p] & 1u, ctl, a.err) ||
                        (l > 0 && !tr_wait(&ctl->sdone[p], (uint32_t)(jobs[p] - 1) & 1u, ctl, a.err))) {
                        ok = false;
                        break;
                    }
                    sm100::tc_fence_after();
                    const int row = tile * BM + rl;
                    const float* bias = a.bias[l];
                    uint32_t* bits = a.bits[l];
                    uint8_t* A = act[p];
#pragma unroll 1
                    for (int c = grp * TR_CHUNKS; c < (grp + 1) * TR_CHUNKS; ++c) {
                        float v[32];
                        sm100::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(p * TR_N + c * 32), v);
                        uint32_t packed[16], pos = 0u;
                        if (BWD) {  // keep the gradient where the forward pre-activation was > 0
                            const uint32_t mw = row < a.M ? __ldg(bits + (size_t)row * 8 + c) : 0u;
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const float x0 = ((mw >> (2 * j)) & 1u) ? v[2 * j] : 0.0f;
                                const float x1 = ((mw >> (2 * j + 1)) & 1u) ? v[2 * j + 1] : 0.0f;
                                __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
                                packed[j] = *reinterpret_cast<uint32_t*>(&h);
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 8 && !BWD; ++j) {
                            const float4 b4 = __ldg(reinterpret_cast<const float4*>(bias + c * 32) + j);
                            const float x0 = v[4 * j] + b4.x, x1 = v[4 * j + 1] + b4.y;
                            const float x2 = v[4 * j + 2] + b4.z, x3 = v[4 * j + 3] + b4.w;
                            __nv_bfloat162 h0 = __floats2bfloat162_rn(fmaxf(x0, 0.0f), fmaxf(x1, 0.0f));
                            __nv_bfloat162 h1 = __floats2bfloat162_rn(fmaxf(x2, 0.0f), fmaxf(x3, 0.0f));
                            packed[2 * j] = *reinterpret_cast<uint32_t*>(&h0);
                            packed[2 * j + 1] = *reinterpret_cast<uint32_t*>(&h1);
                            pos |= ((x0 > 0.0f ? 1u : 0u) | (x1 > 0.0f ? 2u : 0u) | (x2 > 0.0f ? 4u : 0u) |
                                    (x3 > 0.0f ? 8u : 0u))
                                   << (4 * j);
                        }
                        if (!BWD && bits && row < a.M) bits[(size_t)row * 8 + c] = pos;
                        uint8_t* blk = A + (size_t)(c >> 1) * TR_KBYTES + (size_t)rl * 128;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int ch = (c & 1) * 4 + u;
                            *reinterpret_cast<uint4*>(blk + ((ch ^ (rl & 7)) << 4)) =
                                make_uint4(packed[4 * u], packed[4 * u + 1], packed[4 * u + 2], packed[4 * u + 3]);
                        }
                    }
                    sm100::fence_proxy_async();
                    sm100::tc_fence_before();
                    sm100::mbar_arrive(&ctl->aready[p]);
                    ++jobs[p];
                }
    }
    sm100::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        sm100::tc_fence_after();
        sm100::tmem_dealloc(tmem, 2 * TR_N);
    }
}

}  // namespace gemm
}  // namespace plo
