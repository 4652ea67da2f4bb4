// capi.cu -- the C ABI declared in include/geotrace.h: context, validation, launch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/geotrace.h"
#include "internal.cuh"

using gt::CamDesc;

struct gt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    bool st_set = false, cam_set = false;
    double M = 0, S = 0, Q = 0;
    double r0 = 0, th0 = 0, fov = 0;
    int res_x = 0, res_y = 0;
    gt_options opts = {};
    // single-camera descriptor (device) and its validity
    CamDesc *d_cam = nullptr;
    bool cam_dirty = true;
    int cam_valid = 0;
    int cam_flags = -1;
    double cam_rsw = -2.0;
    // batch descriptors (device)
    CamDesc *d_batch = nullptr;
    int batch_cap = 0;
    // launch scratch words
    unsigned long long *d_scratch = nullptr;
    // staging for gt_trace_host
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int cuda_code(cudaError_t e)
{
    if (e == cudaSuccess) return GT_OK;
    if (e == cudaErrorMemoryAllocation) return GT_ERR_OOM;
    return GT_ERR_CUDA;
}

bool valid_spacetime(double M, double S, double Q)
{
    if (!(M > 0.0) || !isfinite(M) || !isfinite(S) || !isfinite(Q)) return false;
    if (!(fabs(S) < M * M)) return false;
    if (Q != 0.0 && S == 0.0) return false;
    return true;
}

bool valid_camera(double r0, double th0, double fov, int rx, int ry)
{
    if (!(r0 > 0.0) || !isfinite(r0)) return false;
    if (!(th0 > 0.0 && th0 < M_PI)) return false;
    if (!(fov > 0.0 && fov < 180.0)) return false;
    if (rx < 1 || ry < 1) return false;
    return true;
}

void fill_desc(CamDesc &d, double M, double S, double Q, double r0, double th0, double fov,
               int rx, int ry, int64_t offset)
{
    memset(&d, 0, sizeof d);
    d.M = M;
    d.S = S;
    d.Q = Q;
    d.r0 = r0;
    d.th0 = th0;
    d.fov_deg = fov;
    d.res_x = rx;
    d.res_y = ry;
    d.offset = offset;
}

gt_options effective(const gt_options &o)
{
    gt_options e = o;
    if (e.block_size == 0) e.block_size = 128;
    if (e.blocks_per_sm == 0) e.blocks_per_sm = 4;
    if (e.reproject_every == 0) e.reproject_every = 64;
    return e;
}

// Upload + set up the single camera if it changed; synchronous (reads validity).
int prepare_camera(gt_ctx *c)
{
    const gt_options e = effective(c->opts);
    if (!c->cam_dirty && c->cam_flags == e.flags && c->cam_rsw == e.r_switch) return GT_OK;
    CamDesc d;
    fill_desc(d, c->M, c->S, c->Q, c->r0, c->th0, c->fov, c->res_x, c->res_y, 0);
    cudaError_t err = cudaMemcpyAsync(c->d_cam, &d, sizeof d, cudaMemcpyHostToDevice, c->stream);
    if (err == cudaSuccess) err = gt::launch_camera_setup(c->d_cam, 1, e.flags, e.r_switch, c->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(&d, c->d_cam, sizeof d, cudaMemcpyDeviceToHost, c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    c->cam_valid = d.valid;
    c->cam_dirty = false;
    c->cam_flags = e.flags;
    c->cam_rsw = e.r_switch;
    return GT_OK;
}

int run_trace(gt_ctx *c, const CamDesc *d_cams, int n_cams, int kind_hint, int64_t first,
              int64_t n_rays, int64_t n_steps, double sp, int mode, double *t, double *r, double *th, double *ph,
              uint8_t *status, uint32_t *nsteps)
{
    const gt_options e = effective(c->opts);
    if (n_rays == 0) return GT_OK;
    gt::TraceArgs a;
    memset(&a, 0, sizeof a);
    a.cams = d_cams;
    a.n_cams = n_cams;
    a.n_rays = n_rays;
    a.first = first;
    a.n_steps = n_steps;
    a.sp = sp;
    a.w6 = (e.flags & GT_FLAG_COMPAT_WEIGHTS) ? 0.1667 : 1.0 / 6.0;
    a.flags = e.flags;
    a.reproject_every = e.reproject_every;
    a.timeout_ns = e.timeout_seconds > 0.0 ? (uint64_t)(e.timeout_seconds * 1e9) : 0;
    a.t = t;
    a.r = r;
    a.th = th;
    a.ph = ph;
    a.status = status;
    a.nsteps = nsteps;
    a.scratch = c->d_scratch;
    cudaError_t err =
        cudaMemsetAsync(c->d_scratch, 0, gt::SCR_WORDS * sizeof(unsigned long long), c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    const bool one_shot = (e.flags & GT_FLAG_ONE_SHOT) != 0;
    int grid;
    if (one_shot) {
        const int64_t g = (n_rays + e.block_size - 1) / e.block_size;
        if (g > 0x7fffffff) return GT_ERR_INVALID_ARG;
        grid = (int)g;
    } else {
        // persistent grid: never more blocks than can be resident at once
        const int fit = gt::max_blocks_per_sm(mode, kind_hint, e.block_size);
        grid = (e.blocks_per_sm < fit ? e.blocks_per_sm : fit) * c->sm_count;
    }
    err = gt::launch_trace(a, mode, kind_hint, e.block_size, grid, one_shot, c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    if (a.timeout_ns) {
        unsigned long long flag = 0;
        err = cudaMemcpyAsync(&flag, c->d_scratch + gt::SCR_TIMEOUT, sizeof flag,
                              cudaMemcpyDeviceToHost, c->stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
        if (err != cudaSuccess) return cuda_code(err);
        if (flag) return GT_ERR_TIMEOUT;
    }
    return GT_OK;
}

bool aligned8(const void *p) { return ((uintptr_t)p & 7u) == 0; }

int check_common(gt_ctx *c, int64_t n_steps, double sp, int mode)
{
    if (!c) return GT_ERR_INVALID_ARG;
    if (n_steps < 0 || n_steps > 0xffffffffLL) return GT_ERR_INVALID_ARG;
    if (!(sp > 0.0) || !isfinite(sp)) return GT_ERR_INVALID_ARG;
    if (mode != GT_MODE_FP64 && mode != GT_MODE_FP32_MIXED) return GT_ERR_INVALID_ARG;
    return GT_OK;
}

} // namespace

extern "C" {

const char *gt_strerror(int code)
{
    switch (code) {
    case GT_OK: return "ok";
    case GT_ERR_INVALID_ARG: return "invalid argument";
    case GT_ERR_NOT_CONFIGURED: return "spacetime or camera not configured";
    case GT_ERR_CUDA: return "CUDA runtime error";
    case GT_ERR_OOM: return "device memory allocation failed";
    case GT_ERR_TIMEOUT: return "device watchdog stopped the launch";
    case GT_ERR_UNSUPPORTED: return "unsupported device or feature";
    default: return "unknown error code";
    }
}

int gt_create(gt_ctx **out, int device, void *cuda_stream)
{
    if (!out) return GT_ERR_INVALID_ARG;
    *out = nullptr;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) return GT_ERR_UNSUPPORTED;
    if (device < 0 || device >= n_dev) return GT_ERR_INVALID_ARG;
    DeviceGuard g(device);
    if (!g.ok) return GT_ERR_CUDA;
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (major != 10 || minor != 3) return GT_ERR_UNSUPPORTED;
    gt_ctx *c = new (std::nothrow) gt_ctx();
    if (!c) return GT_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->sm_count = sms;
    cudaError_t e = cudaMalloc(&c->d_cam, sizeof(CamDesc));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_scratch, gt::SCR_WORDS * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(c->d_cam);
        cudaFree(c->d_scratch);
        delete c;
        return cuda_code(e);
    }
    *out = c;
    return GT_OK;
}

int gt_destroy(gt_ctx *c)
{
    if (!c) return GT_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_cam);
    cudaFree(c->d_batch);
    cudaFree(c->d_scratch);
    cudaFree(c->d_stage);
    delete c;
    return GT_OK;
}

int gt_set_stream(gt_ctx *c, void *cuda_stream)
{
    if (!c) return GT_ERR_INVALID_ARG;
    c->stream = (cudaStream_t)cuda_stream;
    return GT_OK;
}

int gt_set_spacetime(gt_ctx *c, double M, double S, double Q)
{
    if (!c || !valid_spacetime(M, S, Q)) return GT_ERR_INVALID_ARG;
    c->M = M;
    c->S = S;
    c->Q = Q;
    c->st_set = true;
    c->cam_dirty = true;
    return GT_OK;
}

int gt_set_camera(gt_ctx *c, double r0, double theta0, double fov_deg, int res_x, int res_y)
{
    if (!c || !valid_camera(r0, theta0, fov_deg, res_x, res_y)) return GT_ERR_INVALID_ARG;
    c->r0 = r0;
    c->th0 = theta0;
    c->fov = fov_deg;
    c->res_x = res_x;
    c->res_y = res_y;
    c->cam_set = true;
    c->cam_dirty = true;
    return GT_OK;
}

int gt_set_options(gt_ctx *c, const gt_options *o)
{
    if (!c) return GT_ERR_INVALID_ARG;
    gt_options v = {};
    if (o) v = *o;
    if (v.block_size != 0 && (v.block_size < 32 || v.block_size > 256 || v.block_size % 32))
        return GT_ERR_INVALID_ARG;
    if (v.blocks_per_sm < 0 || v.blocks_per_sm > 64) return GT_ERR_INVALID_ARG;
    if (v.reproject_every < 0) return GT_ERR_INVALID_ARG;
    if (!isfinite(v.r_switch) || !(v.timeout_seconds >= 0.0) || !isfinite(v.timeout_seconds))
        return GT_ERR_INVALID_ARG;
    if (v.flags & ~(GT_FLAG_COMPAT_WEIGHTS | GT_FLAG_COMPAT_CAMERA | GT_FLAG_ONE_SHOT))
        return GT_ERR_INVALID_ARG;
    c->opts = v;
    return GT_OK;
}

int gt_trace(gt_ctx *c, int64_t n_steps, double sp, int mode, double *t, double *r, double *th,
             double *ph, uint8_t *status, uint32_t *nsteps)
{
    if (!c) return GT_ERR_INVALID_ARG;
    return gt_trace_range(c, 0, (int64_t)c->res_x * c->res_y, n_steps, sp, mode, t, r, th, ph,
                          status, nsteps);
}

int gt_trace_range(gt_ctx *c, int64_t first, int64_t count, int64_t n_steps, double sp, int mode,
                   double *t, double *r, double *th, double *ph, uint8_t *status,
                   uint32_t *nsteps)
{
    int rc = check_common(c, n_steps, sp, mode);
    if (rc != GT_OK) return rc;
    if (!c->st_set || !c->cam_set) return GT_ERR_NOT_CONFIGURED;
    if (!aligned8(t) || !aligned8(r) || !aligned8(th) || !aligned8(ph) ||
        ((uintptr_t)nsteps & 3u))
        return GT_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    rc = prepare_camera(c);
    if (rc != GT_OK) return rc;
    if (!c->cam_valid) return GT_ERR_INVALID_ARG;
    if (first < 0 || count < 0 || first + count > (int64_t)c->res_x * c->res_y)
        return GT_ERR_INVALID_ARG;
    const int kind = (c->Q != 0.0) ? gt::KIND_MN : gt::KIND_KERR;
    return run_trace(c, c->d_cam, 1, kind, first, count, n_steps, sp, mode, t, r, th, ph, status,
                     nsteps);
}

int gt_trace_host(gt_ctx *c, int64_t n_steps, double sp, int mode, double *t, double *r,
                  double *th, double *ph, uint8_t *status, uint32_t *nsteps)
{
    int rc = check_common(c, n_steps, sp, mode);
    if (rc != GT_OK) return rc;
    if (!c->st_set || !c->cam_set) return GT_ERR_NOT_CONFIGURED;
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    const size_t n = (size_t)c->res_x * (size_t)c->res_y;
    const size_t need = n * (4 * sizeof(double) + sizeof(uint32_t) + sizeof(uint8_t)) + 64;
    if (c->stage_bytes < need) {
        cudaFree(c->d_stage);
        c->d_stage = nullptr;
        c->stage_bytes = 0;
        cudaError_t e = cudaMalloc(&c->d_stage, need);
        if (e != cudaSuccess) return cuda_code(e);
        c->stage_bytes = need;
    }
    double *dt = (double *)c->d_stage;
    double *dr = dt + n, *dth = dr + n, *dph = dth + n;
    uint32_t *dn = (uint32_t *)(dph + n);
    uint8_t *ds = (uint8_t *)(dn + n);
    rc = gt_trace(c, n_steps, sp, mode, t ? dt : nullptr, r ? dr : nullptr, th ? dth : nullptr,
                  ph ? dph : nullptr, status ? ds : nullptr, nsteps ? dn : nullptr);
    if (rc != GT_OK && rc != GT_ERR_TIMEOUT) return rc;
    cudaError_t e = cudaSuccess;
    struct {
        void *h;
        const void *d;
        size_t b;
    } cp[6] = {{t, dt, n * 8}, {r, dr, n * 8}, {th, dth, n * 8}, {ph, dph, n * 8},
               {nsteps, dn, n * 4}, {status, ds, n}};
    for (auto &x : cp)
        if (x.h && e == cudaSuccess)
            e = cudaMemcpyAsync(x.h, x.d, x.b, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_code(e);
    return rc;
}

int gt_trace_batch(gt_ctx *c, const gt_camera_desc *cams, int n_cams, int64_t n_steps, double sp,
                   int mode, double *t, double *r, double *th, double *ph, uint8_t *status,
                   uint32_t *nsteps)
{
    int rc = check_common(c, n_steps, sp, mode);
    if (rc != GT_OK) return rc;
    if (!cams || n_cams < 1 || n_cams > (1 << 20)) return GT_ERR_INVALID_ARG;
    if (!aligned8(t) || !aligned8(r) || !aligned8(th) || !aligned8(ph) ||
        ((uintptr_t)nsteps & 3u))
        return GT_ERR_INVALID_ARG;
    std::vector<CamDesc> h(n_cams);
    int64_t off = 0;
    bool any_mn = false, any_kerr = false;
    for (int i = 0; i < n_cams; i++) {
        const gt_camera_desc &d = cams[i];
        if (!valid_spacetime(d.M, d.S, d.Q) ||
            !valid_camera(d.r0, d.theta0, d.fov_deg, d.res_x, d.res_y))
            return GT_ERR_INVALID_ARG;
        fill_desc(h[i], d.M, d.S, d.Q, d.r0, d.theta0, d.fov_deg, d.res_x, d.res_y, off);
        off += (int64_t)d.res_x * d.res_y;
        if (d.Q != 0.0)
            any_mn = true;
        else
            any_kerr = true;
    }
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    const gt_options e = effective(c->opts);
    cudaError_t err = cudaSuccess;
    if (c->batch_cap < n_cams) {
        cudaFree(c->d_batch);
        c->d_batch = nullptr;
        c->batch_cap = 0;
        err = cudaMalloc(&c->d_batch, sizeof(CamDesc) * n_cams);
        if (err != cudaSuccess) return cuda_code(err);
        c->batch_cap = n_cams;
    }
    err = cudaMemcpyAsync(c->d_batch, h.data(), sizeof(CamDesc) * n_cams, cudaMemcpyHostToDevice,
                          c->stream);
    if (err == cudaSuccess)
        err = gt::launch_camera_setup(c->d_batch, n_cams, e.flags, e.r_switch, c->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(h.data(), c->d_batch, sizeof(CamDesc) * n_cams,
                              cudaMemcpyDeviceToHost, c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    for (int i = 0; i < n_cams; i++)
        if (!h[i].valid) return GT_ERR_INVALID_ARG;
    const int kind = any_mn && any_kerr ? 2 : (any_mn ? gt::KIND_MN : gt::KIND_KERR);
    return run_trace(c, c->d_batch, n_cams, kind, 0, off, n_steps, sp, mode, t, r, th, ph, status,
                     nsteps);
}

int gt_sync(gt_ctx *c)
{
    if (!c) return GT_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    return cuda_code(cudaStreamSynchronize(c->stream));
}

int gt_device_sm_count(gt_ctx *c, int *out)
{
    if (!c || !out) return GT_ERR_INVALID_ARG;
    *out = c->sm_count;
    return GT_OK;
}

} // extern "C"
