// mlp.cuh -- interface of the tensor-core GEMM used by the surrogate network.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gt {

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16 *A; // (m, k) at A[m * a_sm + k * a_sk]
    int64_t a_sm, a_sk;
    const __nv_bfloat16 *B; // (n, k) at B[n * b_sn + k * b_sk]
    int64_t b_sn, b_sk;
    const float *bias; // [N] or null
    int act;           // 0 identity, 1 SiLU
    float *pre;        // optional pre-activation output (fp32, ld_pre)
    int64_t ld_pre;
    float *C32;        // optional fp32 output (ldc)
    int64_t ldc;
    int atomic;        // accumulate into C32 with atomics (split-K)
    __nv_bfloat16 *C16; // optional bf16 output (ldc16)
    int64_t ldc16;
    __nv_bfloat16 *C16T; // optional transposed bf16 output: C16T[n * ldt + m]
    int64_t ldt;
    int *err;          // set to 1 when an mbarrier wait ran out
    int f16_in;        // A and B hold IEEE fp16 bit patterns instead of bf16 (both, never mixed)
    int c16_f16;       // C16 receives fp16 instead of bf16 (C16T stays bf16)
    int c16_split;     // C16 receives each value y as a bf16 pair (hi, lo), hi = bf16(y),
                       // lo = bf16(y - hi), laid out [hi | lo | hi] over 3 N columns
                       // (ldc16 >= 3 N): the A operand of a split-precision product
};

// bn in {16, 32, 64, 128, 256}; splits = K splits (gridDim.z).
cudaError_t launch_gemm(const GemmArgs &g, int bn, int splits, cudaStream_t s);

} // namespace gt
