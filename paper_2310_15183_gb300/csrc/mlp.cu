// mlp.cu -- tensor-core GEMM on tcgen05 (TMEM accumulators) for the surrogate network's
// forward and backward passes.
//
// gemm:  C[m, n] = sum_k A[m, k] B[n, k]  (+ bias[n]) (then SiLU)
//   A element (m, k) at A[m * a_sm + k * a_sk], B element (n, k) at B[n * b_sn + k * b_sk]
//   (bf16, or fp16 for both; any strides, so transposed operands need no copy), FP32
//   accumulation in TMEM; outputs any of: FP32 C (stored, or added for split-K), the FP32
//   pre-activation, a 16-bit copy and a transposed bf16 copy.
//
// Three kernels, chosen by operand layout:
//  * tc_gemm_ws_kernel (K-contiguous operands with encodable TMA tensor maps): persistent,
//    one CTA per SM walking (n, m, k-split) tiles; warp 0 loads A and B chunks with TMA
//    into S stages (mbarrier complete_tx), warp 1 issues the MMAs into one of two TMEM
//    accumulators, eight epilogue warps drain the other one -- bias, SiLU, swizzled
//    shared-memory boxes written back by TMA bulk tensor stores (FP32 add-reductions
//    for split-K) -- so loads, MMAs and stores of consecutive tiles overlap.
//  * tc_gemm_pipe_kernel (K-contiguous, no tensor map): one CTA per 128 x BN tile, a
//    three-stage cp.async pipeline, the MMA thread committing each stage to its mbarrier.
//  * tc_gemm_kernel (any strides): the same tile with register-staged loads.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>
#include <stdlib.h>
#include <string.h>

#include "../../include/geotrace.h"
#include "mlp.cuh"
#include "tc_gemm.cuh"

namespace gt {

namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr uint32_t WAIT_LIMIT = 1u << 24;

template <int BN>
struct GemmSmem {
    static constexpr uint32_t A_BYTES = BM * BK * 2;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr uint32_t TOTAL = 2 * STAGE + 64;
    static constexpr uint32_t A_LBO = (BM / 8) * 128; // K-direction core-matrix stride
    static constexpr uint32_t B_LBO = (BN / 8) * 128;
};

__device__ __forceinline__ void stage_tile(uint8_t *sm, const __nv_bfloat16 *__restrict__ src,
                                           int rows_total, int k_total, int64_t s_row,
                                           int64_t s_k, int row0, int k0, int nrows, uint32_t lbo,
                                           bool vec_ok)
{
    const int tid = threadIdx.x;
    if (vec_ok) {
        // 8 consecutive k per 16-byte vector
        const int nvec = nrows * (BK / 8);
        for (int v = tid; v < nvec; v += blockDim.x) {
            const int row = v / (BK / 8), kb = v % (BK / 8);
            const int gr = row0 + row, gk = k0 + kb * 8;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (gr < rows_total) {
                if (gk + 8 <= k_total) {
                    val = *reinterpret_cast<const uint4 *>(src + (int64_t)gr * s_row + gk);
                } else if (gk < k_total) {
                    __nv_bfloat16 tmp[8];
#pragma unroll
                    for (int e = 0; e < 8; e++)
                        tmp[e] = (gk + e < k_total) ? src[(int64_t)gr * s_row + gk + e]
                                                    : __float2bfloat16(0.0f);
                    val = *reinterpret_cast<const uint4 *>(tmp);
                }
            }
            *reinterpret_cast<uint4 *>(sm + tc::kmajor_offset(row, kb * 8, lbo)) = val;
        }
    } else {
        // generic strides: consecutive threads take consecutive rows (coalesced when the
        // source is row-contiguous, i.e. a transposed view)
        const int n = nrows * BK;
        for (int e = tid; e < n; e += blockDim.x) {
            const int row = e % nrows, k = e / nrows;
            const int gr = row0 + row, gk = k0 + k;
            __nv_bfloat16 val = __float2bfloat16(0.0f);
            if (gr < rows_total && gk < k_total) val = src[(int64_t)gr * s_row + (int64_t)gk * s_k];
            *reinterpret_cast<__nv_bfloat16 *>(sm + tc::kmajor_offset(row, k, lbo)) = val;
        }
    }
}

__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// 16-bit output element (bf16, or fp16 bits stored in the same slot) and a packed pair
__device__ __forceinline__ __nv_bfloat16 to_c16(float y, int f16)
{
    if (f16) {
        const __half h = __float2half_rn(y);
        return __ushort_as_bfloat16(__half_as_ushort(h));
    }
    return __float2bfloat16(y);
}
__device__ __forceinline__ uint32_t pack_c16(float lo, float hi, int f16)
{
    if (f16) {
        const __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// bf16 pair of y: hi = bf16(y) and lo = bf16(y - hi) (y - hi is exact in FP32), so that
// hi + lo carries y to about 2^-17 relative
__device__ __forceinline__ void split_bf16(float y, __nv_bfloat16 *hi, __nv_bfloat16 *lo)
{
    *hi = __float2bfloat16(y);
    *lo = __float2bfloat16(y - __bfloat162float(*hi));
}

// One 16-bit output value: plain, or split into [hi | lo | hi] columns (c16_split)
__device__ __forceinline__ void store_c16(const GemmArgs &g, int64_t row, int col, float y)
{
    __nv_bfloat16 *p = g.C16 + row * g.ldc16 + col;
    if (g.c16_split) {
        __nv_bfloat16 hi, lo;
        split_bf16(y, &hi, &lo);
        p[0] = hi;
        p[g.N] = lo;
        p[2 * g.N] = hi;
    } else {
        *p = to_c16(y, g.c16_f16);
    }
}

// Epilogue shared by both kernels: TMEM -> registers (thread = row) -> bias -> shared
// memory tile (32 columns at a time) -> coalesced stores where each warp writes
// 32 consecutive columns of one row.  The transposed bf16 copy is written straight from
// the row owner (consecutive lanes = consecutive rows, already coalesced).
__device__ __forceinline__ void gemm_epilogue(const GemmArgs &g, uint32_t tmem, int BN_, int m0,
                                              int n0, bool have_acc, float *stage /* 128 x 33 */)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row_own = m0 + warp * 32 + lane;
    for (int cc = 0; cc < BN_; cc += 32) {
        float v[32];
        if (have_acc) {
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
        } else {
#pragma unroll
            for (int i = 0; i < 32; i++) v[i] = 0.0f;
        }
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const int col = n0 + cc + i;
            float z = v[i];
            if (g.bias && blockIdx.z == 0 && col < g.N) z += g.bias[col];
            stage[(warp * 32 + lane) * 33 + i] = z;
            if (g.C16T && row_own < g.M && col < g.N)
                g.C16T[(int64_t)col * g.ldt + row_own] =
                    __float2bfloat16(g.act == 1 ? silu(z) : z);
        }
        __syncthreads();
        // 128 rows x 32 columns: warp w writes rows w, w + 4, ..., lane = column
        const int col = n0 + cc + lane;
        if (col < g.N && cc + lane < BN_) {
            for (int rr = warp; rr < 128; rr += 4) {
                const int row = m0 + rr;
                if (row >= g.M) break;
                const float z = stage[rr * 33 + lane];
                if (g.pre) g.pre[(int64_t)row * g.ld_pre + col] = z;
                const float y = g.act == 1 ? silu(z) : z;
                if (g.C32) {
                    float *p = g.C32 + (int64_t)row * g.ldc + col;
                    if (g.atomic)
                        atomicAdd(p, y);
                    else
                        *p = y;
                }
                if (g.C16) store_c16(g, row, col, y);
            }
        }
        __syncthreads();
    }
}

template <int BN>
__global__ void __launch_bounds__(128) tc_gemm_kernel(GemmArgs g)
{
    using L = GemmSmem<BN>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * L::STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 2 * L::STAGE + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    constexpr uint32_t NCOLS = BN < 32 ? 32 : BN;

    // K range of this split
    const int nk_total = (g.K + BK - 1) / BK;
    const int per = (nk_total + gridDim.z - 1) / gridDim.z;
    const int c_begin = blockIdx.z * per;
    const int c_end = min(nk_total, c_begin + per);
    const int nk = c_end > c_begin ? c_end - c_begin : 0;

    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), NCOLS);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
        tc::mbar_init(tc::smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    const bool a_vec = (g.a_sk == 1) && (g.a_sm % 8 == 0) && ((uintptr_t)g.A % 16 == 0);
    const bool b_vec = (g.b_sk == 1) && (g.b_sn % 8 == 0) && ((uintptr_t)g.B % 16 == 0);
    const uint32_t idesc = tc::idesc_f16_f32(BM, BN, g.f16_in == 0);

    for (int c = 0; c < nk; ++c) {
        const int s = c & 1;
        if (c >= 2) {
            ok = tc::mbar_wait(tc::smem_u32(&mbar[s]), (uint32_t)(((c - 2) >> 1) & 1), WAIT_LIMIT);
            tc::fence_after_sync();
        }
        uint8_t *As = smem + s * L::STAGE;
        uint8_t *Bs = As + L::A_BYTES;
        const int k0 = (c_begin + c) * BK;
        if (ok) {
            stage_tile(As, g.A, g.M, g.K, g.a_sm, g.a_sk, m0, k0, BM, L::A_LBO, a_vec);
            stage_tile(Bs, g.B, g.N, g.K, g.b_sn, g.b_sk, n0, k0, BN, L::B_LBO, b_vec);
        }
        tc::fence_proxy_async();
        ok = __syncthreads_and(ok ? 1 : 0) != 0; // uniform: every thread leaves together
        if (!ok) break;
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a_base = tc::smem_u32(As), b_base = tc::smem_u32(Bs);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t ad = tc::smem_desc(a_base + kk * 2 * L::A_LBO, L::A_LBO, 128);
                const uint64_t bd = tc::smem_desc(b_base + kk * 2 * L::B_LBO, L::B_LBO, 128);
                tc::mma_f16(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(tc::smem_u32(&mbar[s]));
        }
    }
    if (ok && nk > 0) {
        const int last = nk - 1;
        ok = tc::mbar_wait(tc::smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1), WAIT_LIMIT);
    }
    ok = __syncthreads_and(ok ? 1 : 0) != 0; // one outcome for the whole CTA
    tc::fence_after_sync();
    if (!ok) {
        if (tid == 0 && g.err) atomicExch(g.err, 1);
    } else {
        // the operand stages are free now: reuse them as the epilogue's staging tile
        gemm_epilogue(g, tmem, BN, m0, n0, nk > 0, reinterpret_cast<float *>(smem));
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}


// ---------------------------------------------------------------------------------
// Pipelined variant for K-contiguous operands (a_sk = b_sk = 1, 16-byte aligned rows):
// every thread moves 16-byte pieces straight into the K-major core-matrix layout with
// cp.async (zero-filled beyond the matrix edges), STAGES chunks in flight; one thread
// issues the MMAs of a chunk as soon as it has landed and commits them to the stage's
// mbarrier, which gates the stage's reuse.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

__device__ __forceinline__ void issue_tile(uint32_t s_base, const __nv_bfloat16 *__restrict__ src,
                                           int rows_total, int k_total, int64_t s_row, int row0,
                                           int k0, int nrows, uint32_t lbo)
{
    const int npieces = nrows * (BK / 8);
    for (int v = threadIdx.x; v < npieces; v += blockDim.x) {
        const int row = v >> 3, kb = v & 7; // BK / 8 == 8 pieces per row
        const int gr = row0 + row, gk = k0 + kb * 8;
        int bytes = 0;
        const __nv_bfloat16 *p = src;
        if (gr < rows_total && gk < k_total) {
            bytes = (k_total - gk) >= 8 ? 16 : (k_total - gk) * 2;
            p = src + (int64_t)gr * s_row + gk;
        }
        cp_async16(s_base + tc::kmajor_offset(row, kb * 8, lbo), p, (uint32_t)bytes);
    }
}

template <int BN, int STAGES>
__global__ void __launch_bounds__(128) tc_gemm_pipe_kernel(GemmArgs g)
{
    using L = GemmSmem<BN>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + STAGES * L::STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + STAGES * L::STAGE + 8 * STAGES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    constexpr uint32_t NCOLS = BN < 32 ? 32 : BN;
    const int nk_total = (g.K + BK - 1) / BK;
    const int per = (nk_total + gridDim.z - 1) / gridDim.z;
    const int c_begin = blockIdx.z * per;
    const int c_end = min(nk_total, c_begin + per);
    const int nk = c_end > c_begin ? c_end - c_begin : 0;

    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), NCOLS);
    if (tid == 0) {
        for (int st = 0; st < STAGES; st++) tc::mbar_init(tc::smem_u32(&mbar[st]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t sbase = tc::smem_u32(smem);
    const uint32_t idesc = tc::idesc_f16_f32(BM, BN, g.f16_in == 0);

    auto issue = [&](int c) {
        const uint32_t a_s = sbase + (c % STAGES) * L::STAGE;
        const int k0 = (c_begin + c) * BK;
        issue_tile(a_s, g.A, g.M, g.K, g.a_sm, m0, k0, BM, L::A_LBO);
        issue_tile(a_s + L::A_BYTES, g.B, g.N, g.K, g.b_sn, n0, k0, BN, L::B_LBO);
    };
#pragma unroll
    for (int c = 0; c < STAGES - 1; c++) {
        if (c < nk) issue(c);
        cp_async_commit();
    }
    bool ok = true;
    for (int c = 0; c < nk; ++c) {
        cp_async_wait<STAGES - 2>(); // this thread's pieces of chunk c have landed
        tc::fence_proxy_async();
        ok = __syncthreads_and(ok ? 1 : 0) != 0; // uniform: every thread leaves together
        if (!ok) break;
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a_base = sbase + (c % STAGES) * L::STAGE, b_base = a_base + L::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t ad = tc::smem_desc(a_base + kk * 2 * L::A_LBO, L::A_LBO, 128);
                const uint64_t bd = tc::smem_desc(b_base + kk * 2 * L::B_LBO, L::B_LBO, 128);
                tc::mma_f16(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(tc::smem_u32(&mbar[c % STAGES]));
        }
        const int nc = c + STAGES - 1;
        if (c >= 1 && nc < nk) { // chunk nc reuses the stage of chunk c - 1
            ok = tc::mbar_wait(tc::smem_u32(&mbar[(c - 1) % STAGES]),
                               (uint32_t)(((c - 1) / STAGES) & 1), WAIT_LIMIT);
        }
        if (ok && nc < nk) issue(nc);
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (ok && nk > 0) {
        const int last = nk - 1;
        ok = tc::mbar_wait(tc::smem_u32(&mbar[last % STAGES]), (uint32_t)((last / STAGES) & 1),
                           WAIT_LIMIT);
    }
    ok = __syncthreads_and(ok ? 1 : 0) != 0; // one outcome for the whole CTA
    tc::fence_after_sync();
    if (!ok) {
        if (tid == 0 && g.err) atomicExch(g.err, 1);
    } else {
        // the operand stages are free now: reuse them as the epilogue's staging tile
        gemm_epilogue(g, tmem, BN, m0, n0, nk > 0, reinterpret_cast<float *>(smem));
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}

template <int BN>
cudaError_t launch_pipe(const GemmArgs &g, int splits, cudaStream_t s)
{
    using L = GemmSmem<BN>;
    constexpr int STAGES = 3;
    const uint32_t bytes = STAGES * L::STAGE + 8 * STAGES + 64;
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_pipe_kernel<BN, STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, splits);
    tc_gemm_pipe_kernel<BN, STAGES><<<grid, 128, bytes, s>>>(g);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------------
// Persistent warp-specialised variant (K-contiguous operands with TMA tensor maps).
// 320 threads: warp 0 lane 0 loads A and B chunks with one 2-D TMA box of 64 elements x
// (128 | BN) rows each, 128-byte swizzled (the K-major SW128 operand layout), into S stages;
// warp 1 lane 0 issues the MMAs into one of two TMEM accumulators; warps 2-9 drain the
// other accumulator (bias, SiLU, stores) meanwhile, two warps per TMEM lane quarter
// taking alternate 32-column chunks.  Stage and accumulator hand-offs are
// mbarriers (TMA complete_tx, tcgen05.commit, epilogue arrivals); every wait is bounded.
constexpr int EPI_WARPS = 8;
constexpr int WS_THREADS = 64 + 32 * EPI_WARPS;

// Per-epilogue-warp staging of the TMA-store epilogue: a 32 x 32 FP32 box (128-byte
// swizzle), a 32 x 32 bf16 box (64-byte swizzle), a 32 x 32 transposed bf16 box (no
// swizzle) and 32 bias values.
constexpr uint32_t STG_F32 = 0, STG_B16 = 4096, STG_B16T = 6144, STG_BIAS = 8192, STG_WARP = 9216;

template <int BN, int S, bool TMA_OUT>
struct WsSmem {
    static constexpr uint32_t A_BYTES = BM * BK * 2;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr uint32_t EPI = TMA_OUT ? EPI_WARPS * STG_WARP : EPI_WARPS * 32 * 33 * 4;
    static constexpr uint32_t BAR = S * STAGE + EPI;
    static constexpr uint32_t NBAR = 2 * S + 5; // full[S], empty[S], acc_full[2], acc_empty[2], done
    // + 1 KB so that the base can be rounded up to the 1024-byte swizzle period
    static constexpr uint32_t TOTAL = BAR + 8 * NBAR + 16 + 1024;
    static constexpr uint32_t A_LBO = (BM / 8) * 128;
    static constexpr uint32_t B_LBO = (BN / 8) * 128;
    static constexpr uint32_t NCOLS = 2 * BN < 32 ? 32 : 2 * BN; // two accumulators
    static_assert(TOTAL <= 227 * 1024, "shared memory per CTA");
    static_assert(STAGE % 1024 == 0, "stage size keeps the staging boxes 1024-byte aligned");
};

struct OutMaps {
    CUtensorMap c32, pre, c16, c16t;
};

template <int BN, int S, bool TMA_OUT>
__global__ void __launch_bounds__(WS_THREADS, 1)
    tc_gemm_ws_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ OutMaps om, GemmArgs g, int splits)
{
    using L = WsSmem<BN, S, TMA_OUT>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = tc::smem_u32(smem);
    const uint32_t bar = sbase + L::BAR;
    auto FULL = [&](int s) { return bar + 8u * s; };
    auto EMPTY = [&](int s) { return bar + 8u * (S + s); };
    auto ACCF = [&](int b) { return bar + 8u * (2 * S + b); };
    auto ACCE = [&](int b) { return bar + 8u * (2 * S + 2 + b); };
    const uint32_t DONE = bar + 8u * (2 * S + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::BAR + 8 * L::NBAR);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int m_tiles = (g.M + BM - 1) / BM, n_tiles = (g.N + BN - 1) / BN;
    const int nk_total = (g.K + BK - 1) / BK;
    const int per = (nk_total + splits - 1) / splits;
    const int total = m_tiles * n_tiles * splits;

    if (warp == 1) tc::tmem_alloc(tc::smem_u32(tmem_slot), L::NCOLS);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            tc::mbar_init(FULL(s), 1);
            tc::mbar_init(EMPTY(s), 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(ACCF(b), 1);
            tc::mbar_init(ACCE(b), EPI_WARPS);
        }
        tc::mbar_init(DONE, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) { // ---- producer
            uint32_t q = 0;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const int nt = t % n_tiles, mt = (t / n_tiles) % m_tiles, ks = t / (m_tiles * n_tiles);
                const int c0 = ks * per, c1 = min(nk_total, c0 + per);
                for (int c = c0; c < c1; ++c, ++q) {
                    const int s = q % S;
                    if (q >= (uint32_t)S) {
                        ok = tc::mbar_wait(EMPTY(s), ((q / S) - 1) & 1, WAIT_LIMIT);
                        if (!ok) break;
                    }
                    tc::mbar_expect_tx(FULL(s), L::STAGE);
                    const uint32_t a_dst = sbase + s * L::STAGE, b_dst = a_dst + L::A_BYTES;
                    // one 64 x rows box per operand, 128-byte swizzled by the copy engine
                    tc::tma_load_2d(a_dst, &tmA, c * BK, mt * BM, FULL(s));
                    tc::tma_load_2d(b_dst, &tmB, c * BK, nt * BN, FULL(s));
                }
            }
            // copies still in flight (only after a failed wait) land before the CTA exits
            for (uint32_t j = q > (uint32_t)S ? q - S : 0; j < q; ++j)
                if (!tc::mbar_wait(FULL(j % S), (j / S) & 1, WAIT_LIMIT)) ok = false;
        }
    } else if (warp == 1) {
        if (lane == 0) { // ---- MMA issuer
            const uint32_t idesc = tc::idesc_f16_f32(BM, BN, g.f16_in == 0);
            uint32_t q = 0, tl = 0;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++tl) {
                const int ks = t / (m_tiles * n_tiles);
                const int c0 = ks * per, c1 = min(nk_total, c0 + per);
                const int b = tl & 1;
                if (tl >= 2) {
                    ok = tc::mbar_wait(ACCE(b), ((tl >> 1) - 1) & 1, WAIT_LIMIT);
                    if (!ok) break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int c = c0; c < c1; ++c, ++q) {
                    const int s = q % S;
                    ok = tc::mbar_wait(FULL(s), (q / S) & 1, WAIT_LIMIT);
                    if (!ok) break;
                    tc::fence_after_sync();
                    const uint32_t a_base = sbase + s * L::STAGE, b_base = a_base + L::A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t ad = tc::smem_desc_sw128(a_base + kk * 32);
                        const uint64_t bd = tc::smem_desc_sw128(b_base + kk * 32);
                        tc::mma_f16(d, ad, bd, idesc, (c > c0 || kk > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(EMPTY(s));
                }
                if (!ok) break;
                tc::mma_commit(ACCF(b));
            }
            // every issued MMA completes before the accumulators are freed
            tc::mma_commit(DONE);
            if (!tc::mbar_wait(DONE, 0, WAIT_LIMIT)) ok = false;
        }
    } else if (TMA_OUT) { // ---- epilogue warps 2..9 storing through TMA
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        uint8_t *stg = smem + S * L::STAGE + (warp - 2) * STG_WARP;
        const uint32_t s_f32 = tc::smem_u32(stg + STG_F32), s_b16 = tc::smem_u32(stg + STG_B16),
                       s_b16t = tc::smem_u32(stg + STG_B16T);
        float *sbias = reinterpret_cast<float *>(stg + STG_BIAS);
        uint32_t tl = 0;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++tl) {
            const int nt = t % n_tiles, mt = (t / n_tiles) % m_tiles, ks = t / (m_tiles * n_tiles);
            const int b = tl & 1;
            const int m0 = mt * BM + quarter * 32, n0 = nt * BN;
            // bias of this lane's column in each of the warp's chunks, fetched before the wait
            const bool has_bias = g.bias && ks == 0;
            constexpr int NCH = BN / 64 > 0 ? BN / 64 : 1;
            float bl[NCH];
#pragma unroll
            for (int j = 0; j < NCH; j++) {
                const int col = n0 + 32 * half + 64 * j + lane;
                bl[j] = (has_bias && 32 * half + 64 * j < BN && col < g.N) ? __ldg(g.bias + col) : 0.f;
            }
            ok = tc::mbar_wait(ACCF(b), (tl >> 1) & 1, WAIT_LIMIT);
            if (!ok) break;
            tc::fence_after_sync();
#pragma unroll
            for (int j = 0; j < NCH; j++) {
                const int cc = 32 * half + 64 * j;
                if (cc >= BN || m0 >= g.M || n0 + cc >= g.N) break;
                float v[32];
                tc::tmem_ld32(tmem + (uint32_t)(b * BN + cc) + ((uint32_t)(quarter * 32) << 16), v);
                // this warp's previous boxes have left shared memory before it is rewritten
                if (lane == 0) tc::bulk_wait_read();
                if (has_bias) sbias[lane] = bl[j];
                __syncwarp();
                if (has_bias) {
#pragma unroll
                    for (int i = 0; i < 32; i += 4) {
                        const float4 bb = *reinterpret_cast<const float4 *>(sbias + i);
                        v[i] += bb.x;
                        v[i + 1] += bb.y;
                        v[i + 2] += bb.z;
                        v[i + 3] += bb.w;
                    }
                }
                // FP32 box, row = lane, 16-byte chunk c at c ^ (row % 8)
                auto put_f32 = [&]() {
#pragma unroll
                    for (int c = 0; c < 8; c++)
                        *reinterpret_cast<float4 *>(stg + STG_F32 + lane * 128 + ((c ^ (lane & 7)) << 4)) =
                            make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                    tc::fence_proxy_async();
                    __syncwarp();
                };
                if (g.pre) {
                    put_f32();
                    if (lane == 0) {
                        tc::tma_store_2d(&om.pre, n0 + cc, m0, s_f32);
                        tc::bulk_commit();
                    }
                }
                if (g.act == 1) {
#pragma unroll
                    for (int i = 0; i < 32; i++) v[i] = silu(v[i]);
                }
                if (g.C32) {
                    if (g.pre) {
                        if (lane == 0) tc::bulk_wait_read();
                        __syncwarp();
                    }
                    put_f32();
                    if (lane == 0) {
                        if (g.atomic)
                            tc::tma_reduce_add_2d(&om.c32, n0 + cc, m0, s_f32);
                        else
                            tc::tma_store_2d(&om.c32, n0 + cc, m0, s_f32);
                        tc::bulk_commit();
                    }
                }
                // 16-bit box, row = lane (64 bytes), chunk c at c ^ ((row / 2) % 4); with
                // c16_split the hi halves first (the lo halves follow below)
                auto put_b16 = [&](bool lo_part) {
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        uint4 w;
                        uint32_t *wp = &w.x;
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const float a = v[8 * c + 2 * j], b = v[8 * c + 2 * j + 1];
                            if (g.c16_split) {
                                __nv_bfloat16 ha, la, hb, lb;
                                split_bf16(a, &ha, &la);
                                split_bf16(b, &hb, &lb);
                                const __nv_bfloat162 h2 = lo_part ? __halves2bfloat162(la, lb)
                                                                  : __halves2bfloat162(ha, hb);
                                wp[j] = *reinterpret_cast<const uint32_t *>(&h2);
                            } else {
                                wp[j] = pack_c16(a, b, g.c16_f16);
                            }
                        }
                        *reinterpret_cast<uint4 *>(stg + STG_B16 + lane * 64 +
                                                   ((c ^ ((lane >> 1) & 3)) << 4)) = w;
                    }
                };
                if (g.C16) put_b16(false);
                if (g.C16T) { // transposed bf16 box: row = column i, element = lane
#pragma unroll
                    for (int i = 0; i < 32; i++)
                        reinterpret_cast<__nv_bfloat16 *>(stg + STG_B16T)[i * 32 + lane] =
                            __float2bfloat16(v[i]);
                }
                if (g.C16 || g.C16T) {
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        if (g.C16) tc::tma_store_2d(&om.c16, n0 + cc, m0, s_b16);
                        if (g.C16 && g.c16_split) tc::tma_store_2d(&om.c16, 2 * g.N + n0 + cc, m0, s_b16);
                        if (g.C16T) tc::tma_store_2d(&om.c16t, m0, n0 + cc, s_b16t);
                        tc::bulk_commit();
                    }
                }
                if (g.C16 && g.c16_split) { // the lo halves into the middle N columns
                    if (lane == 0) tc::bulk_wait_read();
                    __syncwarp();
                    put_b16(true);
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        tc::tma_store_2d(&om.c16, g.N + n0 + cc, m0, s_b16);
                        tc::bulk_commit();
                    }
                }
                __syncwarp();
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(ACCE(b));
        }
        if (lane == 0) tc::bulk_wait_all();
        __syncwarp();
    } else { // ---- epilogue warps 2..9: TMEM lanes 32 * (warp % 4), column chunks by half
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        float *stg = reinterpret_cast<float *>(smem + S * L::STAGE) + (warp - 2) * 32 * 33;
        uint32_t tl = 0;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++tl) {
            const int nt = t % n_tiles, mt = (t / n_tiles) % m_tiles, ks = t / (m_tiles * n_tiles);
            const int b = tl & 1;
            ok = tc::mbar_wait(ACCF(b), (tl >> 1) & 1, WAIT_LIMIT);
            if (!ok) break;
            tc::fence_after_sync();
            const int m0 = mt * BM + quarter * 32, n0 = nt * BN;
            const int row_own = m0 + lane;
            for (int cc = 32 * half; cc < BN; cc += 64) {
                float v[32];
                tc::tmem_ld32(tmem + (uint32_t)(b * BN + cc) + ((uint32_t)(quarter * 32) << 16), v);
                // lane owns column n0 + cc + lane in the store phase below
                const int col = n0 + cc + lane;
                const bool col_ok = cc + lane < BN && col < g.N;
                const float bias = (g.bias && ks == 0 && col_ok) ? g.bias[col] : 0.f;
                if (g.C16T) { // transposed bf16 copy, written by the row owner
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        const float z = v[i] + __shfl_sync(0xffffffffu, bias, i);
                        const int c = n0 + cc + i;
                        if (row_own < g.M && cc + i < BN && c < g.N)
                            g.C16T[(int64_t)c * g.ldt + row_own] =
                                __float2bfloat16(g.act == 1 ? silu(z) : z);
                    }
                }
#pragma unroll
                for (int i = 0; i < 32; i++) stg[lane * 33 + i] = v[i];
                __syncwarp();
                if (col_ok) {
                    const int nrows = min(32, g.M - m0);
#pragma unroll
                    for (int rr = 0; rr < 32; rr++) {
                        if (rr < nrows) {
                            const int64_t row = m0 + rr;
                            const float z = stg[rr * 33 + lane] + bias;
                            if (g.pre) g.pre[row * g.ld_pre + col] = z;
                            const float y = g.act == 1 ? silu(z) : z;
                            if (g.C32) {
                                float *p = g.C32 + row * g.ldc + col;
                                if (g.atomic)
                                    atomicAdd(p, y);
                                else
                                    *p = y;
                            }
                            if (g.C16) store_c16(g, row, col, y);
                        }
                    }
                }
                __syncwarp();
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(ACCE(b));
        }
    }
    if (!ok && g.err) atomicExch(g.err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, L::NCOLS);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 16-bit matrix of `rows` x `cols` (row stride `ld` elements, K = cols contiguous), boxes
// of BK = 64 columns (128 bytes) x box_rows rows written 128-byte swizzled, zero fill
// outside.
bool make_map(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols, uint64_t ld,
              uint32_t box_rows)
{
    auto enc = tensor_map_encoder();
    if (!enc || rows == 0 || cols == 0 || rows > (1ull << 32) || cols > (1ull << 32)) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld * 2};
    cuuint32_t box[2] = {BK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_sm_count = 0;

// Output tensor map (2-D, row stride `ld` elements) with 32 x 32 boxes.
bool make_out_map(CUtensorMap *m, void *base, CUtensorMapDataType dt, int esize, uint64_t rows,
                  uint64_t cols, uint64_t ld, CUtensorMapSwizzle sw)
{
    auto enc = tensor_map_encoder();
    if (!enc || rows == 0 || cols == 0 || ((uintptr_t)base & 15) || (ld * esize) % 16) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld * esize};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int S, bool TMA_OUT>
cudaError_t launch_ws_kernel(const CUtensorMap &ta, const CUtensorMap &tb, const OutMaps &om,
                             const GemmArgs &g, int splits, int grid, cudaStream_t s)
{
    using L = WsSmem<BN, S, TMA_OUT>;
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_ws_kernel<BN, S, TMA_OUT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL);
    if (e != cudaSuccess) return e;
    tc_gemm_ws_kernel<BN, S, TMA_OUT><<<grid, WS_THREADS, L::TOTAL, s>>>(ta, tb, om, g, splits);
    return cudaGetLastError();
}

template <int BN>
cudaError_t launch_ws(const GemmArgs &g, int splits, cudaStream_t s, bool *used)
{
    *used = false;
    CUtensorMap ta, tb;
    if (!make_map(&ta, g.A, (uint64_t)g.M, (uint64_t)g.K, (uint64_t)g.a_sm, BM) ||
        !make_map(&tb, g.B, (uint64_t)g.N, (uint64_t)g.K, (uint64_t)g.b_sn, BN))
        return cudaSuccess; // caller falls back
    // TMA-store epilogue when every requested output has an encodable map
    OutMaps om;
    memset(&om, 0, sizeof(om));
    bool tma_out = BN >= 32;
    if (tma_out && g.C32)
        tma_out = make_out_map(&om.c32, g.C32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g.M, g.N, g.ldc,
                               CU_TENSOR_MAP_SWIZZLE_128B);
    if (tma_out && g.pre)
        tma_out = make_out_map(&om.pre, g.pre, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g.M, g.N,
                               g.ld_pre, CU_TENSOR_MAP_SWIZZLE_128B);
    if (tma_out && g.C16)
        tma_out = make_out_map(&om.c16, g.C16,
                               g.c16_f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                               2, g.M, g.c16_split ? 3 * (uint64_t)g.N : (uint64_t)g.N,
                               g.ldc16, CU_TENSOR_MAP_SWIZZLE_64B);
    if (tma_out && g.C16T)
        tma_out = make_out_map(&om.c16t, g.C16T, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.N, g.M, g.ldt,
                               CU_TENSOR_MAP_SWIZZLE_NONE);
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    }
    const int nk_total = (g.K + BK - 1) / BK;
    if (splits > nk_total) splits = nk_total;
    splits = (nk_total + ((nk_total + splits - 1) / splits) - 1) / ((nk_total + splits - 1) / splits);
    const int64_t total = (int64_t)((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * splits;
    const int grid = (int)(total < g_sm_count ? total : g_sm_count);
    constexpr int S = BN >= 256 ? 3 : 4;
    *used = true;
    return tma_out ? launch_ws_kernel<BN, S, true>(ta, tb, om, g, splits, grid, s)
                   : launch_ws_kernel<BN, S, false>(ta, tb, om, g, splits, grid, s);
}

template <int BN>
cudaError_t launch_bn(const GemmArgs &g, int splits, cudaStream_t s)
{
    using L = GemmSmem<BN>;
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL);
    if (e != cudaSuccess) return e;
    dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, splits);
    tc_gemm_kernel<BN><<<grid, 128, L::TOTAL, s>>>(g);
    return cudaGetLastError();
}

} // namespace

// The warp-specialised TMA kernel is the default for K-contiguous operands; setting
// GT_GEMM_NO_TMA in the environment selects the cp.async pipeline instead.
static const bool g_use_ws = getenv("GT_GEMM_NO_TMA") == nullptr;

cudaError_t launch_gemm(const GemmArgs &g, int bn, int splits, cudaStream_t s)
{
    if (splits < 1) splits = 1;
    const bool pipe = g.a_sk == 1 && g.b_sk == 1 && g.a_sm % 8 == 0 && g.b_sn % 8 == 0 &&
                      ((uintptr_t)g.A % 16) == 0 && ((uintptr_t)g.B % 16) == 0;
    if (pipe && g.K > 0 && g_use_ws) {
        bool used = false;
        cudaError_t e = cudaSuccess;
        switch (bn) {
        case 16: e = launch_ws<16>(g, splits, s, &used); break;
        case 32: e = launch_ws<32>(g, splits, s, &used); break;
        case 64: e = launch_ws<64>(g, splits, s, &used); break;
        case 128: e = launch_ws<128>(g, splits, s, &used); break;
        case 256: e = launch_ws<256>(g, splits, s, &used); break;
        default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess || used) return e;
    }
    if (pipe) {
        switch (bn) {
        case 16: return launch_pipe<16>(g, splits, s);
        case 32: return launch_pipe<32>(g, splits, s);
        case 64: return launch_pipe<64>(g, splits, s);
        case 128: return launch_pipe<128>(g, splits, s);
        case 256: return launch_pipe<256>(g, splits, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (bn) {
    case 16: return launch_bn<16>(g, splits, s);
    case 32: return launch_bn<32>(g, splits, s);
    case 64: return launch_bn<64>(g, splits, s);
    case 128: return launch_bn<128>(g, splits, s);
    case 256: return launch_bn<256>(g, splits, s);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace gt

extern "C" int gt_gemm_bf16(int device, void *cuda_stream, int M, int N, int K, const void *A,
                            int64_t a_sm, int64_t a_sk, const void *B, int64_t b_sn, int64_t b_sk,
                            const float *bias, int act, float *C, int64_t ldc, int accumulate,
                            int splits, int bn)
{
    if (M < 0 || N < 0 || K < 0 || !A || !B || !C || (act != 0 && act != 1)) return GT_ERR_INVALID_ARG;
    if (bn != 16 && bn != 32 && bn != 64 && bn != 128 && bn != 256) return GT_ERR_INVALID_ARG;
    if (splits < 1 || splits > 4096 || ldc < N) return GT_ERR_INVALID_ARG;
    if (M == 0 || N == 0) return GT_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return GT_ERR_CUDA;
    gt::GemmArgs g = {};
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = (const __nv_bfloat16 *)A;
    g.a_sm = a_sm;
    g.a_sk = a_sk;
    g.B = (const __nv_bfloat16 *)B;
    g.b_sn = b_sn;
    g.b_sk = b_sk;
    g.bias = bias;
    g.act = act;
    g.C32 = C;
    g.ldc = ldc;
    g.atomic = accumulate || splits > 1;
    cudaError_t e = gt::launch_gemm(g, bn, splits, (cudaStream_t)cuda_stream);
    if (prev >= 0) cudaSetDevice(prev);
    return e == cudaSuccess ? GT_OK : GT_ERR_CUDA;
}
