// noalloc.cu -- gt_trace_batch_noalloc: the batched trace without any device allocation.
//
// The ray-queue launch needs a little device scratch: the queue counter and watchdog
// words, and the per-camera descriptors the set-up kernel fills in.  gt_trace_batch
// keeps those in memory its context allocated with cudaMalloc.  Callers that cannot
// allocate device memory use this entry point instead; its scratch is the file-scope
// array below, which every device that loads the library holds until the process
// exits.  Inputs and outputs are still the caller's.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/geotrace.h"
#include "internal.cuh"

namespace {

constexpr size_t WORDS_BYTES = gt::SCR_WORDS * sizeof(unsigned long long);
constexpr size_t CAMS_OFFSET = (WORDS_BYTES + 255) / 256 * 256;
constexpr size_t SCRATCH_BYTES = CAMS_OFFSET + GT_NOALLOC_MAX_CAMS * sizeof(gt::CamDesc);

// Queue words at offset 0, camera descriptors at CAMS_OFFSET.  Shared by every call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_lock;
void *g_addr[MAX_DEVICES] = {};

// Device address of the array on `device` (which must be current); looked up once per
// device and kept for the life of the process, so the entry point must not be used on a
// device across a cudaDeviceReset of it (the module, and the array with it, is reloaded).
// In host code the symbol is only a stand-in, never a device address.
int scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= MAX_DEVICES) return GT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_lock);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return GT_ERR_CUDA;
        g_addr[device] = p;
    }
    *out = (unsigned char *)g_addr[device];
    return GT_OK;
}

struct DeviceRestore {
    int prev = -1;
    ~DeviceRestore()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

} // namespace

extern "C" int gt_trace_batch_noalloc(int device, void *cuda_stream, const gt_camera_desc *cams,
                                      int n_cams, int64_t n_steps, double step_precision,
                                      int mode, double *t, double *r, double *theta, double *phi,
                                      uint8_t *status, uint32_t *nsteps)
{
    if (!cams || n_cams < 1) return GT_ERR_INVALID_ARG;
    if (n_cams > GT_NOALLOC_MAX_CAMS) return GT_ERR_INVALID_ARG; // beyond the static scratch
    if (n_steps < 0 || n_steps > 0xffffffffLL) return GT_ERR_INVALID_ARG;
    if (!(step_precision > 0.0) || !isfinite(step_precision)) return GT_ERR_INVALID_ARG;
    if (mode != GT_MODE_FP64 && mode != GT_MODE_FP32_MIXED) return GT_ERR_INVALID_ARG;
    if (((uintptr_t)t | (uintptr_t)r | (uintptr_t)theta | (uintptr_t)phi) & 7u) return GT_ERR_INVALID_ARG;
    if ((uintptr_t)nsteps & 3u) return GT_ERR_INVALID_ARG;

    gt::CamDesc h[GT_NOALLOC_MAX_CAMS]; // host staging on the stack, not the heap
    int64_t total = 0;
    bool any_mn = false, any_kerr = false;
    for (int i = 0; i < n_cams; i++) {
        const gt_camera_desc &d = cams[i];
        if (!gt::valid_spacetime(d.M, d.S, d.Q) ||
            !gt::valid_camera(d.r0, d.theta0, d.fov_deg, d.res_x, d.res_y))
            return GT_ERR_INVALID_ARG;
        gt::fill_desc(h[i], d.M, d.S, d.Q, d.r0, d.theta0, d.fov_deg, d.res_x, d.res_y, total);
        total += (int64_t)d.res_x * d.res_y;
        if (d.Q != 0.0)
            any_mn = true;
        else
            any_kerr = true;
    }

    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev)
        return GT_ERR_INVALID_ARG;
    DeviceRestore restore;
    if (cudaGetDevice(&restore.prev) != cudaSuccess) restore.prev = -1;
    if (cudaSetDevice(device) != cudaSuccess) return GT_ERR_CUDA;
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (major != 10 || minor != 3) return GT_ERR_UNSUPPORTED;

    unsigned char *base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc != GT_OK) return rc;
    unsigned long long *words = (unsigned long long *)base;
    gt::CamDesc *d_cams = (gt::CamDesc *)(base + CAMS_OFFSET);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // descriptors in, device-side set-up, validity back (synchronous)
    cudaError_t e = cudaMemcpyAsync(d_cams, h, sizeof(gt::CamDesc) * n_cams,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = gt::launch_camera_setup(d_cams, n_cams, 0, 0.0, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, d_cams, sizeof(gt::CamDesc) * n_cams, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return GT_ERR_CUDA;
    for (int i = 0; i < n_cams; i++)
        if (!h[i].valid) return GT_ERR_INVALID_ARG;
    if (total == 0) return GT_OK;

    // the queue counter and watchdog word keep the previous call's values: clear them
    e = cudaMemsetAsync(words, 0, WORDS_BYTES, s);
    if (e != cudaSuccess) return GT_ERR_CUDA;

    gt::TraceArgs a;
    memset(&a, 0, sizeof a);
    a.cams = d_cams;
    a.n_cams = n_cams;
    a.n_rays = total;
    a.n_fresh = total;
    a.first = 0;
    a.n_steps = n_steps;
    a.sp = step_precision;
    a.w6 = 1.0 / 6.0;
    a.flags = 0;
    a.reproject_every = 4096; // the context's default interval
    a.timeout_ns = 0;
    a.t = t;
    a.r = r;
    a.th = theta;
    a.ph = phi;
    a.status = status;
    a.nsteps = nsteps;
    a.scratch = words;
    a.zone_df = 1; // the context's default zone (double-float Manko-Novikov field)
    const int kind = any_mn && any_kerr ? 2 : (any_mn ? gt::KIND_MN : gt::KIND_KERR);
    const int block = 128;
    const int fit = gt::max_blocks_per_sm(
        mode == GT_MODE_FP64 ? gt::KMODE_FP64 : gt::KMODE_MIXED_INLINE, kind, block);
    const int grid = (fit < 4 ? fit : 4) * sms;
    // FP32-mixed runs its zone inline here: the park lists of the context path
    // would need allocated memory
    e = gt::launch_trace(a, mode == GT_MODE_FP64 ? gt::KMODE_FP64 : gt::KMODE_MIXED_INLINE, kind,
                         block, grid, false, s);
    return e == cudaSuccess ? GT_OK : GT_ERR_CUDA;
}
