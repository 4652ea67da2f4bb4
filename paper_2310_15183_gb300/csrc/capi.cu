// capi.cu -- the C ABI declared in include/geotrace.h: context, validation, launch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/geotrace.h"
#include "internal.cuh"
#include "surrogate.cuh"

using gt::CamDesc;
using gt::fill_desc;
using gt::valid_camera;
using gt::valid_spacetime;

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
    // FP32-mixed park lists (two, capacity park_cap items each)
    gt::ParkItem *d_park = nullptr;
    unsigned long long park_cap = 0;
    // CUDA graph of the last GT_FLAG_GRAPH launch (capture stream, key, executable)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    gt::TraceArgs graph_key = {};
    int graph_kmode = -1, graph_kind = -1, graph_block = 0, graph_grid = 0;
    gt::ParkItem *graph_park = nullptr;
    // per-ray parameter block (gt_trace_rays) and surrogate fallback list
    gt::RayParams *d_rays = nullptr;
    // spacetime descriptor of gt_trace_states (no camera)
    CamDesc *d_state_cam = nullptr;
    // gated surrogate inference: probe records; the network's answers (float4 per pixel)
    // followed by an integrator pixel list
    void *d_probe = nullptr;
    int64_t probe_cap = 0;
    void *d_infer = nullptr;
    int64_t infer_cap = 0;
};

cudaStream_t gt_internal_stream(gt_ctx *c) { return c->stream; }

namespace gt {
namespace sg {
int net_pass(gt_surrogate *s, const CamDesc *d_cam, int64_t n_pix, float4 *net, cudaStream_t st);
int select_first(const CamDesc *d_cam, int64_t n_pix, const float4 *net, const ProbeGrid &pg,
                 float tau, double band, double axis, float dir_tol, int64_t *list,
                 unsigned long long *count, cudaStream_t st);
int probe_records(const CamDesc *d_cam, const ProbeGrid &pg, const float4 *net,
                  const uint8_t *status, const double *th, const double *ph, ProbeRec *rec,
                  cudaStream_t st);
int gate_rest(const CamDesc *d_cam, int64_t n_pix, const float4 *net, const ProbeGrid &pg,
              float tau, double band, double axis, float dir_tol, double *t, double *r, double *th,
              double *ph, uint8_t *status, uint32_t *nsteps, int64_t *list,
              unsigned long long *count, cudaStream_t st);
} // namespace sg
} // namespace gt

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
    if (e == cudaErrorMemoryAllocation) {
        // a failed allocation is not sticky, but it stays the thread's "last error":
        // clear it so that the next launch check does not report it again
        (void)cudaGetLastError();
        return GT_ERR_OOM;
    }
    return GT_ERR_CUDA;
}

gt_options effective(const gt_options &o)
{
    gt_options e = o;
    if (e.block_size == 0) e.block_size = 128;
    if (e.blocks_per_sm == 0) e.blocks_per_sm = 4;
    if (e.reproject_every == 0) e.reproject_every = 4096;
    if (e.rays_per_thread == 0) e.rays_per_thread = 1;
    return e;
}

// FP32 rounds launches: two rays per thread when asked for and the launch allows it.
bool use_two(const gt_options &e, const gt::TraceArgs &a, int kind_hint, bool one_shot)
{
    return e.rays_per_thread == 2 && !one_shot &&
           gt::two_rays_supported(a, gt::KMODE_MIXED_FP32, kind_hint);
}

cudaError_t launch_fp32(const gt_options &e, const gt::TraceArgs &a, int kind_hint, int grid,
                        bool one_shot, cudaStream_t s)
{
    if (use_two(e, a, kind_hint, one_shot)) return gt::launch_trace_two(a, kind_hint, e.block_size, grid, s);
    return gt::launch_trace(a, gt::KMODE_MIXED_FP32, kind_hint, e.block_size, grid, one_shot, s);
}

// The listing passes the spacetime parameters to its kernels as float32.
void round_params_f32(CamDesc &d)
{
    d.M = (double)(float)d.M;
    d.S = (double)(float)d.S;
    d.Q = (double)(float)d.Q;
}

constexpr int PAPER_FLAGS = GT_FLAG_FD_DERIVS | GT_FLAG_F32_IO | GT_FLAG_EULER;

// Kind hint of a launch: per camera with forward differences when asked for.
int kind_for(int flags, int kind)
{
    return (flags & GT_FLAG_FD_DERIVS) ? (int)gt::KIND_FD : kind;
}

// Ring, redshift output and state arrays of a launch (all optional).
struct Extra {
    gt::DiskArgs disk = {};
    double *z = nullptr;
    gt::StateArrays states = {};
};

// Upload + set up the single camera if it changed; synchronous (reads validity).
int prepare_camera(gt_ctx *c)
{
    const gt_options e = effective(c->opts);
    if (!c->cam_dirty && c->cam_flags == e.flags && c->cam_rsw == e.r_switch) return GT_OK;
    CamDesc d;
    fill_desc(d, c->M, c->S, c->Q, c->r0, c->th0, c->fov, c->res_x, c->res_y, 0);
    if (e.flags & GT_FLAG_F32_IO) round_params_f32(d);
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

int grid_for(gt_ctx *c, const gt_options &e, int kmode, int kind_hint, int64_t n_work, bool one_shot,
             int *grid)
{
    if (one_shot) {
        const int64_t g = (n_work + e.block_size - 1) / e.block_size;
        if (g > 0x7fffffff) return GT_ERR_INVALID_ARG;
        *grid = g > 0 ? (int)g : 1;
    } else {
        // persistent grid: never more blocks than can be resident at once
        const int fit = (kmode == gt::KMODE_MIXED_FP32 && e.rays_per_thread == 2 &&
                         (kind_hint == gt::KIND_KERR || kind_hint == gt::KIND_MN))
                            ? gt::max_blocks_per_sm_two(kind_hint, e.block_size)
                            : gt::max_blocks_per_sm(kmode, kind_hint, e.block_size);
        *grid = (e.blocks_per_sm < fit ? e.blocks_per_sm : fit) * c->sm_count;
    }
    return GT_OK;
}

int ensure_park(gt_ctx *c, unsigned long long need)
{
    if (c->park_cap >= need) return GT_OK;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_park);
    c->d_park = nullptr;
    c->park_cap = 0;
    cudaError_t err = cudaMalloc(&c->d_park, 2 * need * sizeof(gt::ParkItem));
    if (err != cudaSuccess) return cuda_code(err);
    c->park_cap = need;
    return GT_OK;
}

// The same rounds as one CUDA graph: FP32 launch over the fresh rays, then a WHILE node
// whose body runs the FP64-zone launch and the FP32 continuation and sets the loop
// condition on the device from the park count.  No host round trip.
int build_mixed_graph(gt_ctx *c, const gt::TraceArgs &base, int kind_hint, const gt_options &e,
                      cudaGraphExec_t *exec_out)
{
    int rc = ensure_park(c, (unsigned long long)base.n_rays);
    if (rc != GT_OK) return rc;
    gt::ParkItem *listA = c->d_park, *listB = c->d_park + c->park_cap;
    unsigned long long *w = c->d_scratch;
    int grid32 = 0, grid64 = 0;
    rc = grid_for(c, e, gt::KMODE_MIXED_FP32, kind_hint, base.n_rays, false, &grid32);
    if (rc == GT_OK) rc = grid_for(c, e, gt::KMODE_ZONE_FP64, kind_hint, base.n_rays, false, &grid64);
    if (rc != GT_OK) return rc;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h;
    cudaError_t err = cudaGraphCreate(&g, 0);
    if (err == cudaSuccess) err = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_code(err);
    }
    const size_t W8 = sizeof(unsigned long long);
    cudaStream_t cs = c->cap_stream;
    // prologue: first FP32 round and the initial condition, then the WHILE node
    err = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    cudaGraph_t body = nullptr;
    if (err == cudaSuccess) {
        cudaError_t e1 = cudaMemsetAsync(w, 0, gt::SCR_WORDS * W8, cs);
        gt::TraceArgs a = base;
        a.in_items = listB;
        a.in_count = w + gt::SCR_TO32;
        a.in_cap = c->park_cap;
        a.out_items = listA;
        a.out_count = w + gt::SCR_TO64;
        a.out_cap = c->park_cap;
        if (e1 == cudaSuccess) e1 = launch_fp32(e, a, kind_hint, grid32, false, cs);
        if (e1 == cudaSuccess) e1 = gt::launch_set_condition(h, w + gt::SCR_TO64, cs);
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        cudaGraph_t gg = nullptr;
        if (e1 == cudaSuccess) e1 = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &gg, &deps, nullptr, &nd);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cn = nullptr;
        if (e1 == cudaSuccess) e1 = cudaGraphAddNode(&cn, gg, deps, nullptr, nd, &cp);
        if (e1 == cudaSuccess) {
            body = cp.conditional.phGraph_out[0];
            e1 = cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1,
                                                     cudaStreamSetCaptureDependencies);
        }
        cudaGraph_t done = nullptr;
        err = cudaStreamEndCapture(cs, &done);
        if (err == cudaSuccess) err = e1;
    }
    // body: FP64 zone round A -> B, FP32 round B -> A, condition from A's count
    if (err == cudaSuccess && body)
        err = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess && body) {
        gt::TraceArgs a = base;
        a.n_fresh = 0;
        a.in_cap = a.out_cap = c->park_cap;
        cudaError_t e1 = cudaMemsetAsync(w + gt::SCR_NEXT_RAY, 0, W8, cs);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(w + gt::SCR_TO32, 0, W8, cs);
        a.in_items = listA;
        a.in_count = w + gt::SCR_TO64;
        a.out_items = listB;
        a.out_count = w + gt::SCR_TO32;
        if (e1 == cudaSuccess)
            e1 = gt::launch_trace(a, gt::KMODE_ZONE_FP64, kind_hint, e.block_size, grid64, false, cs);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(w + gt::SCR_NEXT_RAY, 0, W8, cs);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(w + gt::SCR_TO64, 0, W8, cs);
        a.in_items = listB;
        a.in_count = w + gt::SCR_TO32;
        a.out_items = listA;
        a.out_count = w + gt::SCR_TO64;
        if (e1 == cudaSuccess) e1 = launch_fp32(e, a, kind_hint, grid32, false, cs);
        if (e1 == cudaSuccess) e1 = gt::launch_set_condition(h, w + gt::SCR_TO64, cs);
        cudaGraph_t done = nullptr;
        err = cudaStreamEndCapture(cs, &done);
        if (err == cudaSuccess) err = e1;
    } else if (err == cudaSuccess) {
        err = cudaErrorUnknown;
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(exec_out, g, 0);
    cudaGraphDestroy(g);
    return cuda_code(err);
}

// FP32-mixed runs in rounds on the context's stream: an FP32 launch over the fresh rays
// parks every ray that enters the FP64 zone; an FP64 launch integrates the parked rays
// until they leave the zone (parked again) or stop; an FP32 launch continues the
// returned rays; and so on until no ray is parked.  The host reads the park count
// between rounds, so this mode returns after the work has completed.
int run_mixed_rounds(gt_ctx *c, gt::TraceArgs &a, int kind_hint, const gt_options &e, bool one_shot)
{
    int prc = ensure_park(c, (unsigned long long)a.n_rays);
    if (prc != GT_OK) return prc;
    gt::ParkItem *listA = c->d_park, *listB = c->d_park + c->park_cap;
    unsigned long long *w = c->d_scratch;
    a.out_cap = c->park_cap;
    a.in_cap = c->park_cap;
    int grid;
    // round 0: FP32 over the fresh rays, zone entries parked on A
    a.in_items = listB;
    a.in_count = w + gt::SCR_TO32; // zero
    a.out_items = listA;
    a.out_count = w + gt::SCR_TO64;
    int rc = grid_for(c, e, gt::KMODE_MIXED_FP32, kind_hint, a.n_fresh, one_shot, &grid);
    if (rc != GT_OK) return rc;
    cudaError_t err = launch_fp32(e, a, kind_hint, grid, one_shot, c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    for (int round = 0; round < 100000; ++round) {
        unsigned long long parked = 0;
        err = cudaMemcpyAsync(&parked, w + gt::SCR_TO64, sizeof parked, cudaMemcpyDeviceToHost,
                              c->stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
        if (err != cudaSuccess) return cuda_code(err);
        if (parked == 0) return GT_OK;
        // FP64 zone: A -> (B, finished)
        a.n_fresh = 0;
        a.in_items = listA;
        a.in_count = w + gt::SCR_TO64;
        a.out_items = listB;
        a.out_count = w + gt::SCR_TO32;
        err = cudaMemsetAsync(w + gt::SCR_NEXT_RAY, 0, sizeof(unsigned long long), c->stream);
        if (err == cudaSuccess)
            err = cudaMemsetAsync(w + gt::SCR_TO32, 0, sizeof(unsigned long long), c->stream);
        if (err != cudaSuccess) return cuda_code(err);
        rc = grid_for(c, e, gt::KMODE_ZONE_FP64, kind_hint, (int64_t)parked, one_shot, &grid);
        if (rc != GT_OK) return rc;
        err = gt::launch_trace(a, gt::KMODE_ZONE_FP64, kind_hint, e.block_size, grid, one_shot,
                               c->stream);
        if (err != cudaSuccess) return cuda_code(err);
        // FP32 continuation: B -> (A, finished)
        a.in_items = listB;
        a.in_count = w + gt::SCR_TO32;
        a.out_items = listA;
        a.out_count = w + gt::SCR_TO64;
        err = cudaMemsetAsync(w + gt::SCR_NEXT_RAY, 0, sizeof(unsigned long long), c->stream);
        if (err == cudaSuccess)
            err = cudaMemsetAsync(w + gt::SCR_TO64, 0, sizeof(unsigned long long), c->stream);
        if (err != cudaSuccess) return cuda_code(err);
        rc = grid_for(c, e, gt::KMODE_MIXED_FP32, kind_hint, (int64_t)parked, one_shot, &grid);
        if (rc != GT_OK) return rc;
        err = launch_fp32(e, a, kind_hint, grid, one_shot, c->stream);
        if (err != cudaSuccess) return cuda_code(err);
    }
    return GT_ERR_CUDA;
}

int run_trace(gt_ctx *c, const CamDesc *d_cams, int n_cams, int kind_hint, int64_t first,
              int64_t n_rays, int64_t n_steps, double sp, int mode, double *t, double *r,
              double *th, double *ph, uint8_t *status, uint32_t *nsteps,
              const int64_t *fresh_ids = nullptr, const gt::RayParams *d_rays = nullptr,
              bool compact_out = false, const Extra &x = Extra())
{
    const gt_options e = effective(c->opts);
    if ((e.flags & PAPER_FLAGS) && mode != GT_MODE_FP64) return GT_ERR_INVALID_ARG;
    if (n_rays == 0) return GT_OK;
    kind_hint = kind_for(e.flags, kind_hint);
    gt::TraceArgs a;
    memset(&a, 0, sizeof a);
    a.cams = d_cams;
    a.n_cams = n_cams;
    a.n_rays = n_rays;
    a.n_fresh = n_rays;
    a.first = first;
    a.fresh_ids = fresh_ids;
    a.compact_out = compact_out ? 1 : 0;
    a.rays = d_rays;
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
    a.euler = (e.flags & GT_FLAG_EULER) ? 1 : 0;
    a.f32_io = (e.flags & GT_FLAG_F32_IO) ? 1 : 0;
    a.zone_df = (e.flags & GT_FLAG_ZONE_FP64) ? 0 : 1;
    a.disk = x.disk;
    a.z = x.z;
    a.states = x.states;
    cudaError_t err =
        cudaMemsetAsync(c->d_scratch, 0, gt::SCR_WORDS * sizeof(unsigned long long), c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    const bool one_shot = (e.flags & GT_FLAG_ONE_SHOT) != 0;
    int rc;
    if (e.flags & GT_FLAG_GRAPH) {
        // the launch replayed from a CUDA graph, captured once per distinct launch and
        // cached: FP64 is one persistent launch; FP32-mixed is its rounds under a WHILE
        // node whose condition the device sets from the park count
        const int kmode = mode == GT_MODE_FP64 ? gt::KMODE_FP64 : gt::KMODE_MIXED_FP32;
        if (one_shot) return GT_ERR_INVALID_ARG; // graphs replay the persistent launch
        int grid;
        rc = grid_for(c, e, kmode, kind_hint, n_rays, one_shot, &grid);
        if (rc != GT_OK) return rc;
        const bool same = c->graph_exec && memcmp(&c->graph_key, &a, sizeof a) == 0 &&
                          c->graph_kmode == kmode && c->graph_kind == kind_hint &&
                          c->graph_block == e.block_size && c->graph_grid == grid &&
                          c->graph_park == c->d_park && c->park_cap >= (unsigned long long)n_rays;
        if (!same) {
            if (!c->cap_stream) {
                err = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
                if (err != cudaSuccess) return cuda_code(err);
            }
            if (c->graph_exec) {
                cudaGraphExecDestroy(c->graph_exec);
                c->graph_exec = nullptr;
            }
            if (kmode == gt::KMODE_FP64) {
                cudaGraph_t graph = nullptr;
                err = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
                if (err != cudaSuccess) return cuda_code(err);
                cudaError_t e1 = cudaMemsetAsync(c->d_scratch, 0,
                                                 gt::SCR_WORDS * sizeof(unsigned long long),
                                                 c->cap_stream);
                cudaError_t e2 = gt::launch_trace(a, kmode, kind_hint, e.block_size, grid,
                                                  one_shot, c->cap_stream);
                err = cudaStreamEndCapture(c->cap_stream, &graph);
                if (e1 != cudaSuccess || e2 != cudaSuccess || err != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    return GT_ERR_CUDA;
                }
                err = cudaGraphInstantiate(&c->graph_exec, graph, 0);
                cudaGraphDestroy(graph);
                if (err != cudaSuccess) {
                    c->graph_exec = nullptr;
                    return cuda_code(err);
                }
            } else {
                rc = build_mixed_graph(c, a, kind_hint, e, &c->graph_exec);
                if (rc != GT_OK) {
                    c->graph_exec = nullptr;
                    return rc;
                }
            }
            c->graph_park = c->d_park;
            c->graph_key = a;
            c->graph_kmode = kmode;
            c->graph_kind = kind_hint;
            c->graph_block = e.block_size;
            c->graph_grid = grid;
        }
        rc = cuda_code(cudaGraphLaunch(c->graph_exec, c->stream));
    } else if (mode == GT_MODE_FP64) {
        int grid;
        rc = grid_for(c, e, gt::KMODE_FP64, kind_hint, n_rays, one_shot, &grid);
        if (rc != GT_OK) return rc;
        err = gt::launch_trace(a, gt::KMODE_FP64, kind_hint, e.block_size, grid, one_shot,
                               c->stream);
        rc = cuda_code(err);
    } else {
        rc = run_mixed_rounds(c, a, kind_hint, e, one_shot);
    }
    if (rc != GT_OK) return rc;
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
    cudaFree(c->d_park);
    cudaFree(c->d_rays);
    cudaFree(c->d_infer);
    cudaFree(c->d_state_cam);
    cudaFree(c->d_probe);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
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
    if (v.rays_per_thread < 0 || v.rays_per_thread > 2) return GT_ERR_INVALID_ARG;
    if (!isfinite(v.r_switch) || !(v.timeout_seconds >= 0.0) || !isfinite(v.timeout_seconds))
        return GT_ERR_INVALID_ARG;
    if (v.flags & ~(GT_FLAG_COMPAT_WEIGHTS | GT_FLAG_COMPAT_CAMERA | GT_FLAG_ONE_SHOT |
                    GT_FLAG_GRAPH | GT_FLAG_PRECISE_MN | GT_FLAG_ZONE_FP64 | PAPER_FLAGS))
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

int gt_trace_pixels(gt_ctx *c, const int64_t *pixels, int64_t n, int64_t n_steps, double sp,
                    int mode, double *t, double *r, double *th, double *ph, uint8_t *status,
                    uint32_t *nsteps)
{
    int rc = check_common(c, n_steps, sp, mode);
    if (rc != GT_OK) return rc;
    if (!c->st_set || !c->cam_set) return GT_ERR_NOT_CONFIGURED;
    if (n < 0 || (n > 0 && !pixels)) return GT_ERR_INVALID_ARG;
    if (!aligned8(t) || !aligned8(r) || !aligned8(th) || !aligned8(ph) || ((uintptr_t)nsteps & 3u))
        return GT_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    rc = prepare_camera(c);
    if (rc != GT_OK) return rc;
    if (!c->cam_valid) return GT_ERR_INVALID_ARG;
    const int kind = (c->Q != 0.0) ? gt::KIND_MN : gt::KIND_KERR;
    return run_trace(c, c->d_cam, 1, kind, 0, n, n_steps, sp, mode, t, r, th, ph, status, nsteps,
                     pixels, nullptr, true);
}

int gt_trace_disk(gt_ctx *c, double r_in, double r_out, double half_thickness, int64_t n_steps,
                  double sp, int mode, double *t, double *r, double *th, double *ph,
                  uint8_t *status, uint32_t *nsteps, double *z)
{
    int rc = check_common(c, n_steps, sp, mode);
    if (rc != GT_OK) return rc;
    if (!(r_in > 0.0) || !(r_out > r_in) || !isfinite(r_out) || !(half_thickness > 0.0) ||
        !isfinite(half_thickness) || !z || !aligned8(z))
        return GT_ERR_INVALID_ARG;
    if (!c->st_set || !c->cam_set) return GT_ERR_NOT_CONFIGURED;
    if (!aligned8(t) || !aligned8(r) || !aligned8(th) || !aligned8(ph) || ((uintptr_t)nsteps & 3u))
        return GT_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    rc = prepare_camera(c);
    if (rc != GT_OK) return rc;
    if (!c->cam_valid) return GT_ERR_INVALID_ARG;
    Extra x;
    x.disk.on = 1;
    x.disk.r_in = r_in;
    x.disk.r_out = r_out;
    x.disk.half_thickness = half_thickness;
    x.z = z;
    const int kind = (c->Q != 0.0) ? gt::KIND_MN : gt::KIND_KERR;
    return run_trace(c, c->d_cam, 1, kind, 0, (int64_t)c->res_x * c->res_y, n_steps, sp, mode, t,
                     r, th, ph, status, nsteps, nullptr, nullptr, false, x);
}

int gt_trace_states(gt_ctx *c, int64_t n, double *t, double *r, double *th, double *ph,
                    double *pt, double *pr, double *pth, double *pph, double r_escape,
                    int64_t n_steps, double sp, int mode, uint8_t *status, uint32_t *nsteps)
{
    int rc = check_common(c, n_steps, sp, mode);
    if (rc != GT_OK) return rc;
    if (n < 0 || !(r_escape > 0.0) || !isfinite(r_escape)) return GT_ERR_INVALID_ARG;
    double *arr[8] = {t, r, th, ph, pt, pr, pth, pph};
    for (double *p : arr)
        if (!p || !aligned8(p)) return GT_ERR_INVALID_ARG;
    if ((uintptr_t)nsteps & 3u) return GT_ERR_INVALID_ARG;
    if (!c->st_set) return GT_ERR_NOT_CONFIGURED;
    if (n == 0) return GT_OK;
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    const gt_options e = effective(c->opts);
    cudaError_t err = cudaSuccess;
    if (!c->d_state_cam) {
        err = cudaMalloc(&c->d_state_cam, sizeof(CamDesc));
        if (err != cudaSuccess) return cuda_code(err);
    }
    // the spacetime constants come from the camera set-up; the escape radius is
    // 1.5 r0 there, so r0 = r_escape / 1.5 (the camera's own fields are not used)
    CamDesc d;
    fill_desc(d, c->M, c->S, c->Q, r_escape / 1.5, 0.5 * M_PI, 90.0, 1, 1, 0);
    if (e.flags & GT_FLAG_F32_IO) round_params_f32(d);
    err = cudaMemcpyAsync(c->d_state_cam, &d, sizeof d, cudaMemcpyHostToDevice, c->stream);
    if (err == cudaSuccess)
        err = gt::launch_camera_setup(c->d_state_cam, 1, e.flags, e.r_switch, c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    Extra x;
    x.states = {t, r, th, ph, pt, pr, pth, pph};
    const int kind = (c->Q != 0.0) ? gt::KIND_MN : gt::KIND_KERR;
    // the end states reach the arrays through x.states (positions included)
    return run_trace(c, c->d_state_cam, 1, kind, 0, n, n_steps, sp, mode, nullptr, nullptr,
                     nullptr, nullptr, status, nsteps, nullptr, nullptr, false, x);
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
        if (c->opts.flags & GT_FLAG_F32_IO) round_params_f32(h[i]);
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

int gt_trace_rays(gt_ctx *c, int64_t n, const double *alpha, const double *beta,
                  const double *spin, const double *q, const double *theta0, double M, double r0,
                  int64_t n_steps, double sp, int mode, double *t, double *r, double *th,
                  double *ph, uint8_t *status, uint32_t *nsteps)
{
    int rc = check_common(c, n_steps, sp, mode);
    if (rc != GT_OK) return rc;
    if (n < 0 || !alpha || !beta || !spin || !q || !theta0) return GT_ERR_INVALID_ARG;
    if (!(M > 0.0) || !(r0 > 0.0) || !isfinite(M) || !isfinite(r0)) return GT_ERR_INVALID_ARG;
    if (!aligned8(t) || !aligned8(r) || !aligned8(th) || !aligned8(ph) || ((uintptr_t)nsteps & 3u))
        return GT_ERR_INVALID_ARG;
    if (n == 0) return GT_OK;
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    if (!c->d_rays) {
        cudaError_t e = cudaMalloc(&c->d_rays, sizeof(gt::RayParams));
        if (e != cudaSuccess) return cuda_code(e);
    }
    const gt_options e = effective(c->opts);
    gt::RayParams h;
    h.alpha = alpha;
    h.beta = beta;
    h.spin = spin;
    h.q = q;
    h.theta0 = theta0;
    h.M = M;
    h.r0 = r0;
    h.r_switch = e.r_switch;
    cudaError_t err = cudaMemcpyAsync(c->d_rays, &h, sizeof h, cudaMemcpyHostToDevice, c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    // the kernel reads descriptor 0 before the per-ray set-up replaces it
    return run_trace(c, c->d_cam, 1, 2, 0, n, n_steps, sp, mode, t, r, th, ph, status, nsteps,
                     nullptr, c->d_rays);
}

int gt_surrogate_infer(gt_ctx *c, gt_surrogate *s, const gt_gate_cfg *gate, int64_t n_steps,
                       double sp, int mode, double *t, double *r, double *th, double *ph,
                       uint8_t *status, uint32_t *nsteps, int64_t *n_fallback, int64_t *n_probes)
{
    int rc = check_common(c, n_steps, sp, mode);
    if (rc != GT_OK) return rc;
    if (!s || !gate || !t || !r || !th || !ph || !status || !nsteps) return GT_ERR_INVALID_ARG;
    const float tau = gate->tau, dir_tol = gate->dir_tol, probe_tol = gate->probe_tol;
    const double band = gate->band, axis = gate->axis;
    const int probe_stride = gate->probe_stride;
    if (!(tau >= 0.0f) || !(band >= 0.0) || !(axis >= 0.0 && axis < 1.0) || !(dir_tol >= 0.0f) ||
        probe_stride < 0 || !(probe_tol >= 0.0f))
        return GT_ERR_INVALID_ARG;
    if (!c->st_set || !c->cam_set) return GT_ERR_NOT_CONFIGURED;
    if (!aligned8(t) || !aligned8(r) || !aligned8(th) || !aligned8(ph) || ((uintptr_t)nsteps & 3u))
        return GT_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    rc = prepare_camera(c);
    if (rc != GT_OK) return rc;
    if (!c->cam_valid) return GT_ERR_INVALID_ARG;
    const int64_t n_pix = (int64_t)c->res_x * c->res_y;
    if (c->infer_cap < n_pix) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->d_infer);
        c->d_infer = nullptr;
        c->infer_cap = 0;
        cudaError_t e = cudaMalloc(&c->d_infer, n_pix * (sizeof(float4) + sizeof(int64_t)));
        if (e != cudaSuccess) return cuda_code(e);
        c->infer_cap = n_pix;
    }
    float4 *net = (float4 *)c->d_infer;
    int64_t *list = (int64_t *)(net + n_pix);
    const int kind = (c->Q != 0.0) ? gt::KIND_MN : gt::KIND_KERR;
    // integrator probes on a grid of the given stride (images of at least 2 x 2 pixels)
    gt::sg::ProbeGrid pg = {};
    int64_t np = 0;
    if (probe_stride > 0 && c->res_x >= 2 && c->res_y >= 2) {
        pg.stride = probe_stride;
        pg.nx = (c->res_x - 2) / probe_stride + 2;
        pg.ny = (c->res_y - 2) / probe_stride + 2;
        pg.tol = probe_tol;
        np = (int64_t)pg.nx * pg.ny;
        if (c->probe_cap < np) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->d_probe);
            c->d_probe = nullptr;
            c->probe_cap = 0;
            cudaError_t e = cudaMalloc(&c->d_probe, np * sizeof(gt::sg::ProbeRec));
            if (e != cudaSuccess) return cuda_code(e);
            c->probe_cap = np;
        }
    }
    // count of a list; the word is free until the integrator runs, and is read back first
    unsigned long long *d_count = c->d_scratch + gt::SCR_TO32;
    auto list_count = [&](int64_t *out) -> int {
        unsigned long long h = 0;
        cudaError_t e = cudaMemcpyAsync(&h, d_count, sizeof h, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_code(e);
        *out = (int64_t)h;
        return GT_OK;
    };
    // 1. the network on every pixel
    rc = gt::sg::net_pass(s, c->d_cam, n_pix, net, c->stream);
    if (rc != GT_OK) return rc;
    // 2. the probes and every pixel the network's answers alone send to the integrator
    cudaError_t err = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    rc = gt::sg::select_first(c->d_cam, n_pix, net, pg, tau, band, axis, dir_tol, list, d_count,
                              c->stream);
    int64_t n1 = 0, n2 = 0;
    if (rc == GT_OK) rc = list_count(&n1);
    if (rc == GT_OK && n1 > 0)
        rc = run_trace(c, c->d_cam, 1, kind, 0, n1, n_steps, sp, mode, t, r, th, ph, status,
                       nsteps, list, nullptr);
    if (rc != GT_OK) return rc;
    // 3. probe records from the traced probes
    if (pg.stride > 0) {
        gt::sg::ProbeRec *rec = (gt::sg::ProbeRec *)c->d_probe;
        rc = gt::sg::probe_records(c->d_cam, pg, net, status, th, ph, rec, c->stream);
        if (rc != GT_OK) return rc;
        pg.rec = rec;
    }
    // 4. the rest from the network where the probe cells hold, else to a second list
    err = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), c->stream);
    if (err != cudaSuccess) return cuda_code(err);
    rc = gt::sg::gate_rest(c->d_cam, n_pix, net, pg, tau, band, axis, dir_tol, t, r, th, ph,
                           status, nsteps, list, d_count, c->stream);
    if (rc == GT_OK) rc = list_count(&n2);
    if (rc == GT_OK && n2 > 0)
        rc = run_trace(c, c->d_cam, 1, kind, 0, n2, n_steps, sp, mode, t, r, th, ph, status,
                       nsteps, list, nullptr);
    if (rc != GT_OK) return rc;
    if (n_fallback) *n_fallback = n1 - np + n2;
    if (n_probes) *n_probes = np;
    return GT_OK;
}

int gt_autotune(gt_ctx *c, int mode, int64_t trial_rays, int64_t trial_steps, double sp,
                const char *cache_path, int *best_block, int *best_blocks_per_sm,
                int *best_rays_per_thread, double *best_steps_per_s)
{
    if (!c || trial_rays < 1 || trial_steps < 1 || !(sp > 0.0)) return GT_ERR_INVALID_ARG;
    if (mode != GT_MODE_FP64 && mode != GT_MODE_FP32_MIXED) return GT_ERR_INVALID_ARG;
    if (!c->st_set || !c->cam_set) return GT_ERR_NOT_CONFIGURED;
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    const int kind = (c->Q != 0.0) ? gt::KIND_MN : gt::KIND_KERR;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return GT_ERR_CUDA;
    char key[256];
    snprintf(key, sizeof key, "mode=%d kind=%d sms=%d dev=%s", mode, kind, c->sm_count, prop.name);
    auto report = [&](int b, int k, int rpt, double v) {
        c->opts.block_size = b;
        c->opts.blocks_per_sm = k;
        c->opts.rays_per_thread = rpt;
        if (best_block) *best_block = b;
        if (best_blocks_per_sm) *best_blocks_per_sm = k;
        if (best_rays_per_thread) *best_rays_per_thread = rpt;
        if (best_steps_per_s) *best_steps_per_s = v;
    };
    // cached result?
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[512];
            while (fgets(line, sizeof line, f)) {
                int b = 0, k = 0, rpt = 1;
                double v = 0;
                char *bar = strchr(line, '|');
                if (!bar) continue;
                *bar = 0;
                if (strcmp(line, key) == 0 && sscanf(bar + 1, "%d %d %d %lf", &b, &k, &rpt, &v) == 4 &&
                    b >= 32 && b <= 256 && b % 32 == 0 && k >= 1 && k <= 64 && (rpt == 1 || rpt == 2)) {
                    fclose(f);
                    report(b, k, rpt, v);
                    return GT_OK;
                }
            }
            fclose(f);
        }
    }
    const int64_t n_pix = (int64_t)c->res_x * c->res_y;
    const int64_t count = trial_rays < n_pix ? trial_rays : n_pix;
    const int64_t first = (n_pix - count) / 2;
    double *buf = nullptr;
    uint32_t *ns = nullptr;
    cudaError_t err = cudaMalloc(&buf, count * 4 * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&ns, count * sizeof(uint32_t));
    if (err != cudaSuccess) {
        cudaFree(buf);
        return cuda_code(err);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const gt_options saved = c->opts;
    const int blocks[] = {64, 128, 192, 256};
    const int per_sm[] = {1, 2, 3, 4, 6, 8};
    const int n_rpt = mode == GT_MODE_FP32_MIXED ? 2 : 1;
    int bb = 128, bk = 4, br = 1;
    double bv = -1.0;
    int rc = GT_OK;
    for (int rpt = 1; rpt <= n_rpt && rc == GT_OK; rpt++) {
        for (int bi = 0; bi < 4 && rc == GT_OK; bi++) {
            const int kmode = mode == GT_MODE_FP64 ? gt::KMODE_FP64 : gt::KMODE_MIXED_FP32;
            const int fit = rpt == 2 ? gt::max_blocks_per_sm_two(kind, blocks[bi])
                                     : gt::max_blocks_per_sm(kmode, kind, blocks[bi]);
            for (int ki = 0; ki < 6 && rc == GT_OK; ki++) {
                if (per_sm[ki] > fit) continue;
                c->opts = saved;
                c->opts.block_size = blocks[bi];
                c->opts.blocks_per_sm = per_sm[ki];
                c->opts.rays_per_thread = rpt;
                c->opts.timeout_seconds = 0.0;
                double best_ms = 1e300;
                for (int rep = 0; rep < 2 && rc == GT_OK; rep++) {
                    cudaEventRecord(e0, c->stream);
                    rc = gt_trace_range(c, first, count, trial_steps, sp, mode, buf, buf + count,
                                        buf + 2 * count, buf + 3 * count, nullptr, ns);
                    cudaEventRecord(e1, c->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess) rc = GT_ERR_CUDA;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0 && ms < best_ms) best_ms = ms; // first run warms up
                }
                if (rc != GT_OK) break;
                const double v = (double)count * (double)trial_steps / (best_ms * 1e-3);
                if (v > bv) {
                    bv = v;
                    bb = blocks[bi];
                    bk = per_sm[ki];
                    br = rpt;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(ns);
    c->opts = saved;
    if (rc != GT_OK) return rc;
    report(bb, bk, br, bv);
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s|%d %d %d %.6g\n", key, bb, bk, br, bv);
            fclose(f);
        }
    }
    return GT_OK;
}

int gt_sync(gt_ctx *c)
{
    if (!c) return GT_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    return cuda_code(cudaStreamSynchronize(c->stream));
}

int gt_get_stats(gt_ctx *c, int64_t *zone_steps, int64_t *zone_f64_evals)
{
    if (!c || !zone_steps) return GT_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    if (!g.ok) return GT_ERR_CUDA;
    unsigned long long v[2] = {0, 0}; // SCR_ZONE_STEPS, SCR_ZONE_F64 (adjacent words)
    static_assert(gt::SCR_ZONE_F64 == gt::SCR_ZONE_STEPS + 1, "zone words are adjacent");
    cudaError_t e = cudaMemcpyAsync(v, c->d_scratch + gt::SCR_ZONE_STEPS, sizeof v,
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_code(e);
    *zone_steps = (int64_t)v[0];
    if (zone_f64_evals) *zone_f64_evals = (int64_t)v[1];
    return GT_OK;
}

int gt_device_sm_count(gt_ctx *c, int *out)
{
    if (!c || !out) return GT_ERR_INVALID_ARG;
    *out = c->sm_count;
    return GT_OK;
}

} // extern "C"
