// internal.cuh -- structures shared by the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/geotrace.h"
#include "df.cuh"
#include "spacetime.cuh"

// The context's stream (capi.cu).
cudaStream_t gt_internal_stream(gt_ctx *c);

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
    double r_switch;        // FP32-mixed: zone radius
    SpacetimeT<DF> st_df;   // the spacetime constants in double-float (the zone's field)
    int32_t valid;          // 1 when the camera sits where g_tt < 0
    int32_t pad_;
};

// Scratch words of one launch (device memory owned by the context).
enum : int {
    SCR_NEXT_RAY = 0,   // persistent queue: next unclaimed work item
    SCR_TIMEOUT = 1,    // set to 1 by the watchdog
    SCR_TO64 = 2,       // FP32-mixed: rays parked for the FP64 zone kernel
    SCR_TO32 = 3,       // FP32-mixed: rays handed back to the FP32 kernel
    SCR_ZONE_STEPS = 4, // FP32-mixed: RK4 steps taken in the zone (gt_get_stats)
    SCR_ZONE_F64 = 5,   // FP32-mixed: zone field evaluations done in FP64 (gt_get_stats)
    SCR_WORDS = 6
};

// Kernel modes (public GT_MODE_FP32_MIXED runs MIXED_FP32 and ZONE_FP64 in rounds).
enum : int { KMODE_FP64 = 0, KMODE_MIXED_INLINE = 1, KMODE_MIXED_FP32 = 2, KMODE_ZONE_FP64 = 3 };

// Kind of a launch: one spacetime kind for every camera (KIND_KERR, KIND_MN), per camera
// (KIND_ANY), or per camera with the listing's forward-difference metric derivatives
// (KIND_FD, FP64 only).
enum : int { KIND_ANY = 2, KIND_FD = 3 };

// A ray handed between the FP32 and FP64-zone kernels (full state in FP64).
struct ParkItem {
    int64_t id;
    uint32_t n;
    int32_t cam;
    double t, r, th, ph, pr, pth, pt, pph;
};

// Per-ray initial data (surrogate training labels): ray k starts at (0, r0, theta0[k], 0)
// of the spacetime (M, spin[k] M, q[k]) with direction (alpha[k], beta[k]) in the
// camera's (v^phi sin theta0, v^theta) plane, v^r = -1.
struct RayParams {
    const double *alpha, *beta, *spin, *q, *theta0; // device arrays; spin is a/M (S = spin M^2)
    double M, r0, r_switch;
};

// The ring of the paper's renders as an exit (Sec. 3.3.3): r_in <= r <= r_out and
// |r cos theta| <= half_thickness; on = 0 disables it.
struct DiskArgs {
    int on;
    double r_in, r_out, half_thickness;
};

// Ray states as inputs and outputs (gt_trace_states): SoA device arrays, updated in place.
struct StateArrays {
    double *t, *r, *th, *ph, *pt, *pr, *pth, *pph;
};

struct TraceArgs {
    const RayParams *rays; // device pointer; when non-null the camera descriptors are unused
    const CamDesc *cams; // device
    int n_cams;
    int64_t n_rays;   // rays of the whole trace
    int64_t n_fresh;  // fresh rays started by this launch, ids [0, n_fresh); output index
                      // k belongs to flat ray first + k
    int64_t first;    // first flat ray id (single-camera range traces)
    const int64_t *fresh_ids; // when set, fresh work item w is ray fresh_ids[w]; otherwise ray w
    int compact_out;          // with fresh_ids: output index w instead of fresh_ids[w]
    const ParkItem *in_items;                // input list (modes 2, 3) or null
    const unsigned long long *in_count;      // its length (device word) or null
    unsigned long long in_cap;               // capacity of the input list
    ParkItem *out_items;                     // output list (modes 2, 3)
    unsigned long long *out_count;           // its length (device word)
    unsigned long long out_cap;
    int64_t n_steps;
    double sp;        // step_precision
    double w6;        // RK4 weight (1/6, or 0.1667 in compat mode)
    // float copies for the FP32 kernel, filled by launch_trace (kernel parameters the
    // loop reads directly, so no per-step conversions are rematerialised)
    float sp_f, w6_f, h_thr_f;
    DF sp_df, w6_df; // double-float copies for the zone
    int flags;
    int reproject_every;
    uint64_t timeout_ns; // 0 = no watchdog
    double *t, *r, *th, *ph;
    uint8_t *status;
    uint32_t *nsteps;
    unsigned long long *scratch; // SCR_WORDS words
    // paper-numerics and objects (FP64 kernels unless noted)
    int euler;        // explicit Euler instead of RK4 (Sec. 3.1.1)
    int f32_io;       // initial state and outputs rounded to float32 (listing)
    DiskArgs disk;    // the ring exit (also in the FP32-mixed kernels)
    double *z;        // redshift factor per ray (ring hits; NaN otherwise) or null
    StateArrays states; // with states.t != null fresh rays start from these arrays and the
                        // end states (all 8 components) are written back to them
    int zone_df;        // FP32-mixed: the zone's Manko-Novikov field in double-float
};

// Host-side validation shared by every entry point that takes a spacetime or a camera
// (Sec. 2.2.2: |S| < M^2 for a black hole; Sec. 2.2.3: alpha divides by S/M, so q != 0
// needs S != 0; Sec. 3.3.1: a pinhole camera at 0 < theta0 < pi with 0 < FOV < 180 deg).
inline bool valid_spacetime(double M, double S, double Q)
{
    if (!(M > 0.0) || !isfinite(M) || !isfinite(S) || !isfinite(Q)) return false;
    if (!(fabs(S) < M * M)) return false;
    if (Q != 0.0 && S == 0.0) return false;
    return true;
}

inline bool valid_camera(double r0, double th0, double fov, int rx, int ry)
{
    if (!(r0 > 0.0) || !isfinite(r0)) return false;
    if (!(th0 > 0.0 && th0 < M_PI)) return false;
    if (!(fov > 0.0 && fov < 180.0)) return false;
    if (rx < 1 || ry < 1) return false;
    return true;
}

// Raw descriptor of one camera (the derived fields are filled in on the device).
inline void fill_desc(CamDesc &d, double M, double S, double Q, double r0, double th0, double fov,
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

// Launchers (trace.cu).  Return a cudaError_t from the launch.
cudaError_t launch_camera_setup(CamDesc *d_cams, int n_cams, int flags, double r_switch,
                                cudaStream_t s);
// One-thread kernel setting a graph WHILE node's condition to (*count != 0).
cudaError_t launch_set_condition(cudaGraphConditionalHandle h, const unsigned long long *count,
                                 cudaStream_t s);
// Resident blocks per SM of the trace kernel for this block size (>= 1).
int max_blocks_per_sm(int kmode, int kind_hint, int block);
cudaError_t launch_trace(const TraceArgs &a, int kmode, int kind_hint, int block, int grid,
                         bool one_shot, cudaStream_t s);
// The FP32 rounds kernel with two rays per thread (persistent launch only), when the
// launch allows it (one camera of one spacetime kind; no watchdog, per-ray parameters,
// state arrays or ring).
bool two_rays_supported(const TraceArgs &a, int kmode, int kind_hint);
cudaError_t launch_trace_two(const TraceArgs &a, int kind_hint, int block, int grid,
                             cudaStream_t s);
int max_blocks_per_sm_two(int kind_hint, int block);

} // namespace gt
