// internal.cuh -- structures shared by the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spacetime.cuh"

namespace gt {

// Raw camera parameters as uploaded by the host, plus everything the setup kernel
// derives from them on the device.
struct CamDesc {
    // inputs
    double M, S, Q;
    double r0, th0, fov_deg;
    int32_t res_x, res_y;
    int64_t offset; // first flat ray id of this camera
    // derived on the device (camera_setup_kernel)
    SpacetimeC st;
    double V, H;            // half ranges of v^theta and v^phi (before 1/sin theta0)
    double inv_sin_th0;     // 1/sin(theta0), or 1 with GT_FLAG_COMPAT_CAMERA
    double gl_tt, gl_tph, gl_phph, gl_rr, gl_thth; // lower metric at the camera
    double r_escape;        // 1.5 r0
    double r_switch;        // FP32-mixed: FP64 zone radius
    int32_t valid;          // 1 when the camera sits where g_tt < 0
    int32_t pad_;
};

// Scratch words of one launch (device memory owned by the context).
enum : int {
    SCR_NEXT_RAY = 0,   // persistent queue: next unclaimed ray id
    SCR_TIMEOUT = 1,    // set to 1 by the watchdog
    SCR_WORDS = 4
};

// Per-ray initial data (surrogate training labels): ray k starts at (0, r0, theta0[k], 0)
// of the spacetime (M, spin[k] M, q[k]) with direction (alpha[k], beta[k]) in the
// camera's (v^phi sin theta0, v^theta) plane, v^r = -1.
struct RayParams {
    const double *alpha, *beta, *spin, *q, *theta0; // device arrays, spin as a/M... see gt_trace_rays
    double M, r0, r_switch;
};

struct TraceArgs {
    const RayParams *rays; // device pointer; when non-null the camera descriptors are unused
    const CamDesc *cams; // device
    int n_cams;
    int64_t n_rays;   // rays in this launch; output index k is ray first + k
    int64_t first;    // first flat ray id (single-camera range traces)
    int64_t n_steps;
    double sp;        // step_precision
    double w6;        // RK4 weight (1/6, or 0.1667 in compat mode)
    int flags;
    int reproject_every;
    uint64_t timeout_ns; // 0 = no watchdog
    double *t, *r, *th, *ph;
    uint8_t *status;
    uint32_t *nsteps;
    unsigned long long *scratch; // SCR_WORDS words
};

// Launchers (trace.cu).  Return a cudaError_t from the launch.
cudaError_t launch_camera_setup(CamDesc *d_cams, int n_cams, int flags, double r_switch,
                                cudaStream_t s);
// Resident blocks per SM of the trace kernel for this block size (>= 1).
int max_blocks_per_sm(int mode, int kind_hint, int block);
cudaError_t launch_trace(const TraceArgs &a, int mode, int kind_hint, int block, int grid,
                         bool one_shot, cudaStream_t s);

} // namespace gt
