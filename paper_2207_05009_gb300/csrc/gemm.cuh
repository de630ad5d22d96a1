// BF16 tensor-core GEMMs for the NeRF-SH network (Sec. 4.2) on sm_103a:
// tcgen05.mma with FP32 accumulators in TMEM, operands staged by TMA into
// 128-byte-swizzled shared memory.
//
// k_gemm:  C[M][N] = A[M][K] * B[N][K]^T  (both K-major), fused epilogue:
//          bias + ReLU -> bf16, bias -> fp32, (x mask>0) -> bf16, or a split
//          (columns below `split`: bias + ReLU -> bf16; the rest: bias -> fp32).
//          Persistent CTAs; B (the weights, N*K*2 <= 128 KB) stays resident
//          in shared memory; A streams through a 4-stage ring of 128x64
//          tiles; two TMEM accumulators let the epilogue of one 128-row tile
//          overlap the MMAs of the next.
// k_wgrad: dW[o][i] += sum_m dZ[m][o] * H[m][i] over a chunk of rows m
//          (both operands MN-major, read straight from the row-major
//          activations), split over CTAs and reduced with vector atomics.
//
// Warp roles: warp 0 lane 0 issues TMA, warp 1 owns TMEM and lane 0 issues
// MMAs, the rest run the epilogue (warp w reads TMEM lanes 32*(w%4) .. +31).
// k_gemm has two epilogue warpgroups (320 threads): the two warps of a lane
// quadrant take half of the tile's 32-column chunks each, so every
// sub-partition interleaves two epilogue warps; k_wgrad has one (192).  All mbarrier waits are bounded; a wait that gives up
// raises an abort flag in shared memory and a bit in the caller's error word,
// every role then drains what it has in flight and the CTA frees its TMEM.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sm100.cuh"

namespace plo {
namespace gemm {

constexpr int THREADS = 192;       // k_wgrad
constexpr int EPI_GROUPS = 2;      // k_gemm epilogue warpgroups
constexpr int GEMM_THREADS = 64 + 128 * EPI_GROUPS;
constexpr int BM = 128;
constexpr int BK = 64;  // one 128-byte swizzle row of bf16
constexpr int STAGES = 4;
constexpr int A_STAGE_BYTES = BM * BK * 2;  // 16 KB

enum Epi : int { EPI_RELU_BF16 = 0, EPI_BIAS_F32 = 1, EPI_MASK_BF16 = 2, EPI_SPLIT = 3, EPI_MASKBITS_BF16 = 4 };

struct EpiArgs {
    const float* bias;            // [N] (EPI_RELU_BF16, EPI_BIAS_F32, EPI_SPLIT)
    __nv_bfloat16* out_bf16;      // [M][ldo]
    float* out_f32;               // [M][ldo] (EPI_BIAS_F32); [M][ldo2] columns >= split (EPI_SPLIT)
    int ldo;
    const __nv_bfloat16* mask;    // [M][ldm] (EPI_MASK_BF16)
    int ldm;
    int split;                    // EPI_SPLIT: first fp32 column (a multiple of 32)
    int ldo2;                     // EPI_SPLIT: row stride of out_f32
    const float* col0_add;        // EPI_BIAS_F32: added to column 0 of each row (nullable)
    int ld_col0;                  // row stride of col0_add
    int tma_out;                  // bf16 outputs leave through the output tensor map (boxes of 32 x 32)
    uint32_t* bits_out;           // EPI_RELU_BF16 / EPI_SPLIT: [M][ldb] words, bit j of word c set iff
                                  // the pre-activation of column 32c + j is > 0 (nullable)
    const uint32_t* bits;         // EPI_MASKBITS_BF16: the mask as such words, [M][ldb]
    int ldb;                      // words per row of bits_out / bits
    unsigned int* err;            // device error word (bit 1: GEMM wait timeout)
    uint32_t wait_limit;          // polls per barrier wait (0: sm100::WAIT_LIMIT)
    int debug_skip_loads;         // test hook: the producer issues no loads, so the waits run out
};

__host__ __device__ constexpr int tmem_cols_for(int n) {
    return n * 2 <= 32 ? 32 : (n * 2 <= 64 ? 64 : (n * 2 <= 128 ? 128 : (n * 2 <= 256 ? 256 : 512)));
}
constexpr int OUT_STAGE_BYTES = 32 * 32 * 2;  // one 32 x 32 bf16 box, per epilogue warp and buffer
__host__ __device__ constexpr size_t gemm_smem_bytes(int N, int K) {
    return 1024 /*align*/ + (size_t)N * K * 2 + (size_t)STAGES * A_STAGE_BYTES +
           8 * EPI_GROUPS * OUT_STAGE_BYTES + 256 /*barriers*/;
}

struct Ctl {
    uint64_t full[STAGES], empty[STAGES], bfull, tfull[2], tempty[2], drain;
    uint32_t tmem;
    uint32_t limit;
    int abort;
};

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t ph, Ctl* ctl, unsigned int* err) {
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

template <int N>
// mk: the chunk's 32 mask values (EPI_MASK_BF16), or its mask word in mk[0].x
// (EPI_MASKBITS_BF16), loaded ahead by the caller;
// stage: where the 32 bf16 results go instead of global memory (nullable)
__device__ __forceinline__ void epilogue_chunk(const EpiArgs& ep, int epi, int row, int M, int col, const float* v,
                                               const uint4* mk, uint4* stage) {
    if (row >= M) return;
    if (epi == EPI_BIAS_F32 || (epi == EPI_SPLIT && col >= ep.split)) {
        const bool split = epi == EPI_SPLIT;
        float4* dst = reinterpret_cast<float4*>(split ? ep.out_f32 + (size_t)row * ep.ldo2 + (col - ep.split)
                                                      : ep.out_f32 + (size_t)row * ep.ldo + col);
        const float c0 = (!split && col == 0 && ep.col0_add) ? __ldg(ep.col0_add + (size_t)row * ep.ld_col0) : 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float4 b = *reinterpret_cast<const float4*>(ep.bias + col + 4 * j);
            dst[j] = make_float4(v[4 * j] + b.x + (j == 0 ? c0 : 0.0f), v[4 * j + 1] + b.y, v[4 * j + 2] + b.z,
                                 v[4 * j + 3] + b.w);
        }
        return;
    }
    uint32_t packed[16];
    if (epi == EPI_RELU_BF16 || epi == EPI_SPLIT) {
        uint32_t pos = 0u;  // bit j: pre-activation j is > 0 (the ReLU derivative)
        float bv[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 b4 = __ldg(reinterpret_cast<const float4*>(ep.bias + col) + j);
            bv[4 * j] = b4.x;
            bv[4 * j + 1] = b4.y;
            bv[4 * j + 2] = b4.z;
            bv[4 * j + 3] = b4.w;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float x0 = v[2 * j] + bv[2 * j];
            const float x1 = v[2 * j + 1] + bv[2 * j + 1];
            __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(x0, 0.0f), fmaxf(x1, 0.0f));
            packed[j] = *reinterpret_cast<uint32_t*>(&h);
            pos |= (x0 > 0.0f ? 1u : 0u) << (2 * j);
            pos |= (x1 > 0.0f ? 1u : 0u) << (2 * j + 1);
        }
        if (ep.bits_out) ep.bits_out[(size_t)row * ep.ldb + col / 32] = pos;
    } else if (epi == EPI_MASKBITS_BF16) {
        const uint32_t mw = mk[0].x;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float a = ((mw >> (2 * j)) & 1u) ? v[2 * j] : 0.0f;
            float b = ((mw >> (2 * j + 1)) & 1u) ? v[2 * j + 1] : 0.0f;
            __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            packed[j] = *reinterpret_cast<uint32_t*>(&h);
        }
    } else {  // EPI_MASK_BF16
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 mw = mk[q];
            uint32_t w[4] = {mw.x, mw.y, mw.z, mw.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                // bf16 pair (lo, hi): positive iff sign clear and not zero
                uint32_t lo = w[u] & 0xFFFFu, hi = w[u] >> 16;
                float a = (lo != 0u && !(lo & 0x8000u)) ? v[8 * q + 2 * u] : 0.0f;
                float b = (hi != 0u && !(hi & 0x8000u)) ? v[8 * q + 2 * u + 1] : 0.0f;
                __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                packed[4 * q + u] = *reinterpret_cast<uint32_t*>(&h);
            }
        }
    }
    uint4* dst = stage ? stage : reinterpret_cast<uint4*>(ep.out_bf16 + (size_t)row * ep.ldo + col);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
}

template <int N, int K>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
           const __grid_constant__ CUtensorMap tmO, EpiArgs ep, int epi, int M) {
    static_assert(K % BK == 0 && N % 32 == 0 && N <= 256, "tile shape");
    constexpr int KB = K / BK;
    constexpr int TMEM_COLS = tmem_cols_for(N);
    constexpr uint32_t IDESC = sm100::idesc_bf16(BM, N, 0, 0);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sB = smem;                    // KB blocks of [N rows][128 B]
    uint8_t* sA = sB + (size_t)N * K * 2;  // STAGES x [128 rows][128 B]
    uint8_t* sO = sA + STAGES * A_STAGE_BYTES;  // epilogue warps x 2 output boxes
    Ctl* ctl = reinterpret_cast<Ctl*>(sO + 8 * EPI_GROUPS * OUT_STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            sm100::mbar_init(&ctl->full[s], 1);
            sm100::mbar_init(&ctl->empty[s], 1);
        }
        sm100::mbar_init(&ctl->bfull, 1);
        for (int j = 0; j < 2; ++j) {
            sm100::mbar_init(&ctl->tfull[j], 1);
            sm100::mbar_init(&ctl->tempty[j], 128 * EPI_GROUPS);
        }
        sm100::mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        ctl->limit = ep.wait_limit ? ep.wait_limit : sm100::WAIT_LIMIT;
        sm100::fence_mbar_init();
    }
    if (warp == 1) sm100::tmem_alloc(&ctl->tmem, TMEM_COLS);
    sm100::tc_fence_before();
    __syncthreads();
    sm100::tc_fence_after();
    const uint32_t tmem = ctl->tmem;
    const int n_tiles = (M + BM - 1) / BM;

    if (warp == 0 && lane == 0 && !ep.debug_skip_loads) {
        // ---------------- TMA producer
        sm100::prefetch_tmap(&tmA);
        sm100::prefetch_tmap(&tmB);
        sm100::mbar_arrive_expect_tx(&ctl->bfull, (uint32_t)(N * K * 2));
        for (int kb = 0; kb < KB; ++kb) sm100::tma_load_2d(sB + (size_t)kb * N * 128, &tmB, kb * BK, 0, &ctl->bfull);
        int stage = 0;
        uint32_t ph = 0;
        uint32_t armed = 0, armed_ph = 0;  // stages with a load issued, and its parity
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
            for (int kb = 0; kb < KB; ++kb) {
                if (!wait_or_abort(&ctl->empty[stage], ph ^ 1u, ctl, ep.err)) {
                    ok = false;
                    break;
                }
                sm100::mbar_arrive_expect_tx(&ctl->full[stage], A_STAGE_BYTES);
                sm100::tma_load_2d(sA + stage * A_STAGE_BYTES, &tmA, kb * BK, tile * BM, &ctl->full[stage]);
                armed |= 1u << stage;
                armed_ph = (armed_ph & ~(1u << stage)) | (ph << stage);
                if (++stage == STAGES) {
                    stage = 0;
                    ph ^= 1u;
                }
            }
        }
        if (!ok) {  // drain the loads still in flight before the CTA exits
            for (int s = 0; s < STAGES; ++s)
                if (armed & (1u << s)) sm100::mbar_wait(&ctl->full[s], (armed_ph >> s) & 1u);
            sm100::mbar_wait(&ctl->bfull, 0);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        bool ok = wait_or_abort(&ctl->bfull, 0, ctl, ep.err);
        int stage = 0, acc = 0;
        uint32_t ph = 0, aph = 0;
        bool issued = false;
        for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
            if (!wait_or_abort(&ctl->tempty[acc], aph ^ 1u, ctl, ep.err)) {
                ok = false;
                break;
            }
            sm100::tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(acc * N);
            for (int kb = 0; kb < KB; ++kb) {
                if (!wait_or_abort(&ctl->full[stage], ph, ctl, ep.err)) {
                    ok = false;
                    break;
                }
                sm100::tc_fence_after();
                const uint32_t a0 = sm100::smem_addr(sA + stage * A_STAGE_BYTES);
                const uint32_t b0 = sm100::smem_addr(sB + (size_t)kb * N * 128);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k) {
                    uint64_t adesc = sm100::smem_desc_sw128(a0 + 32 * k, 16, 1024);
                    uint64_t bdesc = sm100::smem_desc_sw128(b0 + 32 * k, 16, 1024);
                    sm100::mma_bf16(d, adesc, bdesc, IDESC, (kb | k) != 0);
                }
                issued = true;
                sm100::mma_commit(&ctl->empty[stage]);
                if (++stage == STAGES) {
                    stage = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) break;
            sm100::mma_commit(&ctl->tfull[acc]);
            if (++acc == 2) {
                acc = 0;
                aph ^= 1u;
            }
        }
        if (!ok && issued) {  // let issued MMAs finish before TMEM is freed
            sm100::mma_commit(&ctl->drain);
            sm100::mbar_wait(&ctl->drain, 0);
        }
    } else if (warp >= 2) {
        // ---------------- epilogue
        const int q = warp & 3;                 // TMEM lane quadrant (rows q*32 .. +31 of the tile)
        const int grp = (warp - 2) >> 2;        // which half of the column chunks
        constexpr int CH = N / 32 / EPI_GROUPS;  // chunks per warp
        static_assert((N / 32) % EPI_GROUPS == 0, "chunks split evenly between the epilogue warpgroups");
        const int c_beg = grp * CH, c_end = c_beg + CH;
        uint8_t* sOw = sO + (size_t)(warp - 2) * 2 * OUT_STAGE_BYTES;  // this warp's two output boxes
        int acc = 0, sbuf = 0;
        uint32_t aph = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            const int row = tile * BM + q * 32 + lane;
            // the mask is read one chunk ahead, so its latency overlaps the
            // accumulator wait and the previous chunk's work
            const bool masked = epi == EPI_MASK_BF16 && row < M;
            const bool bitmask = epi == EPI_MASKBITS_BF16 && row < M;
            const uint4* mrow = masked ? reinterpret_cast<const uint4*>(ep.mask + (size_t)row * ep.ldm) : nullptr;
            const uint32_t* brow = bitmask ? ep.bits + (size_t)row * ep.ldb : nullptr;
            uint4 mk[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) mk[j] = masked ? __ldg(mrow + 4 * c_beg + j) : make_uint4(0u, 0u, 0u, 0u);
            if (bitmask) mk[0].x = __ldg(brow + c_beg);
            if (!wait_or_abort(&ctl->tfull[acc], aph, ctl, ep.err)) break;
            sm100::tc_fence_after();
#pragma unroll 1
            for (int c = c_beg; c < c_end; ++c) {
                float v[32];
                sm100::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * N + c * 32), v);
                uint4 nx[4];
                const bool more = masked && c + 1 < c_end;
#pragma unroll
                for (int j = 0; j < 4; ++j) nx[j] = more ? __ldg(mrow + 4 * (c + 1) + j) : make_uint4(0u, 0u, 0u, 0u);
                if (bitmask && c + 1 < c_end) nx[0].x = __ldg(brow + c + 1);
                const bool tma = ep.tma_out && epi != EPI_BIAS_F32 && !(epi == EPI_SPLIT && c * 32 >= ep.split);
                if (tma) {
                    // stage the warp's 32 x 32 box, then one thread stores it;
                    // a buffer is refilled once the store issued from it two
                    // chunks ago has read it (rows past M are clipped)
                    uint8_t* st = sOw + (size_t)sbuf * OUT_STAGE_BYTES;
                    if (lane == 0) sm100::bulk_wait_read_1();
                    __syncwarp();
                    epilogue_chunk<N>(ep, epi, row, M, c * 32, v, mk, reinterpret_cast<uint4*>(st + lane * 64));
                    sm100::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        sm100::tma_store_2d(&tmO, c * 32, tile * BM + q * 32, st);
                        sm100::bulk_commit();
                    }
                    sbuf ^= 1;
                } else {
                    epilogue_chunk<N>(ep, epi, row, M, c * 32, v, mk, nullptr);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) mk[j] = nx[j];
            }
            sm100::tc_fence_before();
            sm100::mbar_arrive(&ctl->tempty[acc]);
            if (++acc == 2) {
                acc = 0;
                aph ^= 1u;
            }
        }
        if (lane == 0) sm100::bulk_wait_all();  // the output stores are complete before the CTA exits
    }
    sm100::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        sm100::tc_fence_after();
        sm100::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- weight gradient
// dW[o][i] += sum_{m in chunk} dZ[m][o] * H[m][i]; o in [out_base, out_base+128).
// A' = dZ^T tile: two TMA boxes of 64 (o) x 64 (m) -> MN-major, LBO = 8 KB
// between the 64-wide o blocks, SBO = 1 KB between 8-row m groups.  B' = H^T
// tile: NIN/64 boxes of 64 (i) x 64 (m), same strides.
// With db: db[o] += sum_m dZ[m][o] (the bias gradient) as one more MMA per
// k-step, A' against a 16 x 64 tile of ones kept in shared memory, into 16
// spare accumulator columns: the column sums cost no extra pass over dZ.
template <int NIN>
__host__ __device__ constexpr size_t wgrad_stage_bytes() {
    return (size_t)(2 + NIN / 64) * 64 * 128;
}
constexpr int WGRAD_ONES_BYTES = 16 * 128;  // 16 rows (n) x 64 (k) bf16 ones, K-major
template <int NIN>
__host__ __device__ constexpr size_t wgrad_smem_bytes() {
    return 1024 + STAGES * wgrad_stage_bytes<NIN>() + 1024 /*barriers, padded*/ + WGRAD_ONES_BYTES;
}
template <int NIN>
__host__ __device__ constexpr int wgrad_tmem_cols() {  // NIN accumulator columns + 16 for the bias sums
    return NIN + 16 <= 32 ? 32 : (NIN + 16 <= 64 ? 64 : (NIN + 16 <= 128 ? 128 : (NIN + 16 <= 256 ? 256 : 512)));
}

template <int NIN>
__global__ void __launch_bounds__(THREADS, 1)
    k_wgrad(const __grid_constant__ CUtensorMap tmDZ, const __grid_constant__ CUtensorMap tmH, float* dW, int n_out,
            int M, int chunk, unsigned int* err, float* db) {
    constexpr int TMEM_COLS = wgrad_tmem_cols<NIN>();
    constexpr uint32_t IDESC = sm100::idesc_bf16(BM, NIN, 1, 1);
    constexpr uint32_t IDESC_ONES = sm100::idesc_bf16(BM, 16, 1, 0);
    constexpr uint32_t STAGE = (uint32_t)wgrad_stage_bytes<NIN>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    Ctl* ctl = reinterpret_cast<Ctl*>(smem + STAGES * STAGE);
    uint8_t* ones = smem + STAGES * STAGE + 1024;  // 1 KB aligned
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // blockIdx.x: output tile, so that the CTAs of one sample chunk run side
    // by side and the second read of their shared H tiles hits L2
    const int out_base = blockIdx.x * BM;
    const int m_beg = blockIdx.y * chunk;
    const int m_end = min(m_beg + chunk, M);
    const int n_kb = m_end > m_beg ? (m_end - m_beg + 63) / 64 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            sm100::mbar_init(&ctl->full[s], 1);
            sm100::mbar_init(&ctl->empty[s], 1);
        }
        sm100::mbar_init(&ctl->tfull[0], 1);
        sm100::mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        ctl->limit = sm100::WAIT_LIMIT;
        sm100::fence_mbar_init();
    }
    if (db) {  // bf16 1.0 everywhere, so the swizzle of the tile does not matter
        for (int j = threadIdx.x; j < WGRAD_ONES_BYTES / 4; j += THREADS)
            reinterpret_cast<uint32_t*>(ones)[j] = 0x3F803F80u;
        sm100::fence_proxy_async();  // visible to the tensor core
    }
    if (warp == 1) sm100::tmem_alloc(&ctl->tmem, TMEM_COLS);
    sm100::tc_fence_before();
    __syncthreads();
    sm100::tc_fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == 0 && lane == 0) {
        sm100::prefetch_tmap(&tmDZ);
        sm100::prefetch_tmap(&tmH);
        int stage = 0;
        uint32_t ph = 0, armed = 0, armed_ph = 0;
        bool ok = true;
        for (int kb = 0; kb < n_kb; ++kb) {
            if (!wait_or_abort(&ctl->empty[stage], ph ^ 1u, ctl, err)) {
                ok = false;
                break;
            }
            uint8_t* st = smem + stage * STAGE;
            const int m0 = m_beg + kb * 64;
            sm100::mbar_arrive_expect_tx(&ctl->full[stage], STAGE);
            sm100::tma_load_2d(st, &tmDZ, out_base, m0, &ctl->full[stage]);
            sm100::tma_load_2d(st + 8192, &tmDZ, out_base + 64, m0, &ctl->full[stage]);
#pragma unroll
            for (int j = 0; j < NIN / 64; ++j)
                sm100::tma_load_2d(st + 16384 + j * 8192, &tmH, j * 64, m0, &ctl->full[stage]);
            armed |= 1u << stage;
            armed_ph = (armed_ph & ~(1u << stage)) | (ph << stage);
            if (++stage == STAGES) {
                stage = 0;
                ph ^= 1u;
            }
        }
        if (!ok)
            for (int s = 0; s < STAGES; ++s)
                if (armed & (1u << s)) sm100::mbar_wait(&ctl->full[s], (armed_ph >> s) & 1u);
    } else if (warp == 1 && lane == 0) {
        int stage = 0;
        uint32_t ph = 0;
        bool ok = true, issued = false;
        for (int kb = 0; kb < n_kb; ++kb) {
            if (!wait_or_abort(&ctl->full[stage], ph, ctl, err)) {
                ok = false;
                break;
            }
            sm100::tc_fence_after();
            const uint32_t a0 = sm100::smem_addr(smem + stage * STAGE);
            const uint32_t b0 = a0 + 16384;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint64_t adesc = sm100::smem_desc_sw128(a0 + 2048 * k, 8192, 1024);
                uint64_t bdesc = sm100::smem_desc_sw128(b0 + 2048 * k, 8192, 1024);
                sm100::mma_bf16(tmem, adesc, bdesc, IDESC, (kb | k) != 0);
                if (db) {
                    uint64_t odesc = sm100::smem_desc_sw128(sm100::smem_addr(ones) + 32 * k, 16, 1024);
                    sm100::mma_bf16(tmem + NIN, adesc, odesc, IDESC_ONES, (kb | k) != 0);
                }
            }
            issued = true;
            sm100::mma_commit(&ctl->empty[stage]);
            if (++stage == STAGES) {
                stage = 0;
                ph ^= 1u;
            }
        }
        if (ok && issued) sm100::mma_commit(&ctl->tfull[0]);
        if (!ok && issued) {
            sm100::mma_commit(&ctl->drain);
            sm100::mbar_wait(&ctl->drain, 0);
        }
    } else if (warp >= 2 && n_kb > 0) {
        const int q = warp & 3;
        if (wait_or_abort(&ctl->tfull[0], 0, ctl, err)) {
            sm100::tc_fence_after();
            const int o = out_base + q * 32 + lane;
#pragma unroll 1
            for (int c = 0; c < NIN / 32; ++c) {
                float v[32];
                sm100::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 32), v);
                if (o < n_out) {
                    float4* dst = reinterpret_cast<float4*>(dW + (size_t)o * NIN + c * 32);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        atomicAdd(dst + j, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
                }
            }
            if (db) {  // the 16 ones-columns all hold the row sum; the first one is used
                float v[32];
                sm100::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)NIN, v);
                if (o < n_out) atomicAdd(db + o, v[0]);
            }
        }
    }
    sm100::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        sm100::tc_fence_after();
        sm100::tmem_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace gemm
}  // namespace plo
