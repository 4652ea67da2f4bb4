// tc_gemm.cuh -- fifth-generation tensor-core (tcgen05) building blocks for sm_103a:
// TMEM allocation, UMMA shared-memory / instruction descriptors, kind::f16 MMA with
// BF16 or FP16 operands and FP32 accumulation in TMEM, commit to an mbarrier, TMEM
// loads, and the TMA bulk-tensor loads, stores and reductions with their mbarriers.
//
// Two operand layouts in shared memory, both K-major:
//   - the 128-byte swizzled layout of the warp-specialised TMA kernel (smem_desc_sw128),
//     written by one TMA box per operand per 64-wide K-chunk; and
//   - the no-swizzle core-matrix layout of the cp.async / register-staged fallback
//     kernels (smem_desc): 8x8 "core matrices" of 8 rows x 16 bytes, core matrix
//     (g, kb) -- row group g = row/8, column block kb = k/8 -- at kb * lbo + g * 128
//     bytes, so the leading byte offset (between core matrices along K) is `lbo` and
//     the stride byte offset (between 8-row groups) is 128.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gt {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 64-bit UMMA shared-memory descriptor: start >> 4 in [0,14), LBO >> 4 in [16,30),
// SBO >> 4 in [32,46), version 1 in [46,48), no swizzle in [61,64).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Descriptor of a K-major operand tile in the 128-byte swizzled layout: rows of 128 bytes
// (64 16-bit elements of K), the 16-byte chunk j of row r stored at chunk j ^ (r % 8), in
// 1024-byte atoms of 8 rows (stride byte offset 1024; the leading byte offset is unused
// for this layout and set to 16).  Swizzling mode 2 in bits 61-63.  K-slices of 16
// elements within the atom start 32 bytes apart; the atoms must be 1024-byte aligned.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

// 32-bit instruction descriptor of kind::f16: D = F32 (bits 4-5 = 1), A and B both BF16
// (bits 7-9 = 1, 10-12 = 1) or both FP16 (0), both K-major (bits 15, 16 = 0), N >> 3 at
// 17, M >> 4 at 24.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N, bool bf16)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) { return idesc_f16_f32(M, N, true); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar_smem)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        mbar_smem));
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar_smem, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_smem), "r"(count));
}

// Bounded wait for the mbarrier phase with parity `parity`; returns false if the
// iteration limit ran out (the caller records the error and unwinds).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar_smem, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}\n"
            : "=r"(done)
            : "r"(mbar_smem), "r"(parity));
        if (done) return true;
    }
    return false;
}

// 32 lanes x 32 consecutive FP32 columns: thread t of warp w receives TMEM lane
// 32 (w % 4) + t, columns [col, col + 32).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major no-swizzle tile whose K-direction
// core-matrix stride is `lbo` bytes.
__device__ __forceinline__ uint32_t kmajor_offset(int row, int k, uint32_t lbo)
{
    return (uint32_t)(k >> 3) * lbo + (uint32_t)(row >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

} // namespace tc
} // namespace gt

namespace gt {
namespace tc {

// ---------------------------------------------------------------- TMA and mbarriers
__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
                 : "memory");
}
// 2-D tiled TMA load of box {x .. x + box0, y .. y + box1} into shared memory; completes
// on `mbar` with the box's byte count.  x (the innermost coordinate) must keep x * 2
// bytes a multiple of 16 for bf16 -- callers pass multiples of 8 elements.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(tmap), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

} // namespace tc
} // namespace gt

namespace gt {
namespace tc {

// ---------------------------------------------------------------- TMA stores
// 2-D tiled store (or FP32 add-reduction) of a shared-memory box to global memory; rows
// and columns outside the tensor are clipped.  Issued by one thread after the box's
// writers fenced their shared-memory stores to the async proxy.
__device__ __forceinline__ void tma_store_2d(const void *tmap, int x, int y, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     tmap),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void tma_reduce_add_2d(const void *tmap, int x, int y, uint32_t src)
{
    asm volatile(
        "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
            tmap),
        "r"(x), "r"(y), "r"(src)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of all committed bulk stores have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// all committed bulk stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

} // namespace tc
} // namespace gt
