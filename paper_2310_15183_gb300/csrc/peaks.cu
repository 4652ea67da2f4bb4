// peaks.cu -- FMA-pipe microbenchmarks that measure the chip's FP64 and FP32
// arithmetic peaks (the ray tracer is bound by plain ALU throughput, and these
// peaks are not otherwise on record).  Each thread runs 8 independent FMA chains
// so the pipes, not the FMA latency, limit the rate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/geotrace.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T *out, int iters, T a, T b)
{
    T x0 = (T)threadIdx.x, x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 16; u++) {
            x0 = x0 * a + b;
            x1 = x1 * a + b;
            x2 = x2 * a + b;
            x3 = x3 * a + b;
            x4 = x4 * a + b;
            x5 = x5 * a + b;
            x6 = x6 * a + b;
            x7 = x7 * a + b;
        }
    }
    const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == T(-12345.678)) out[0] = s; // never true; keeps the chains live
}

} // namespace

extern "C" int gt_measure_fma_peak(int device, int fp64, int iters, double *flops_per_s)
{
    if (!flops_per_s || iters < 1) return GT_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return GT_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int block = 256, grid = sms * 8;
    void *out = nullptr;
    cudaEvent_t e0, e1;
    cudaError_t err = cudaMalloc(&out, 16);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float ms = 0.f;
    if (err == cudaSuccess) {
        for (int rep = 0; rep < 2 && err == cudaSuccess; rep++) { // first pass warms up
            cudaEventRecord(e0, 0);
            if (fp64)
                fma_chain_kernel<double><<<grid, block>>>((double *)out, iters, 0.999999, 1e-7);
            else
                fma_chain_kernel<float><<<grid, block>>>((float *)out, iters, 0.999999f, 1e-7f);
            cudaEventRecord(e1, 0);
            err = cudaEventSynchronize(e1);
            if (err == cudaSuccess) err = cudaGetLastError();
        }
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (prev >= 0) cudaSetDevice(prev);
    if (err != cudaSuccess) return GT_ERR_CUDA;
    const double fmas = (double)grid * block * iters * 16.0 * 8.0;
    *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    return GT_OK;
}
