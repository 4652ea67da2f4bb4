/*
 * geotrace.h -- C ABI of the GB300 (sm_103a) null-geodesic ray tracer.
 *
 * The library integrates one light ray per image pixel backwards from a pinhole
 * camera through a rotating black-hole spacetime with parameters (M, S, Q):
 * Kerr in Boyer-Lindquist coordinates (Sec. 2.2.2 of "Graphical Processing of
 * Geodesic Propagation in Python") when Q = 0, Manko-Novikov with quadrupole
 * deviation q = Q (Sec. 2.2.3) otherwise.  Each ray follows the Hamiltonian
 * equations of Eq. hamGeodesic,
 *     dq^mu/dtau = g^{mu nu} p_nu,     dp_mu/dtau = -1/2 d_mu g^{nu sigma} p_nu p_sigma,
 * under classical RK4 (Sec. 3.1.2) with the step h = step_precision/|dq^t/dtau|
 * taken from the first stage, and stops (appendix listing, propagation kernel)
 *     ESCAPED   when r > 1.5 r0 after a step,
 *     HORIZON   when the step just taken had h < step_precision * 3e-5,
 *     MAXSTEPS  after n_steps steps,
 *     NONFINITE when a step produces a non-finite value (the last finite state is kept).
 * Initial data (Sec. 3.3.1 and the listing's camera block): pixel (i, j), i along phi
 * in [0, res_x), j along theta in [0, res_y), direction v = (v^t, -1, beta_j,
 * alpha_i/sin theta0) with alpha_i, beta_j the inclusive linspaces over [-H, H],
 * [-V, V], V = tan(FOV/2)/r0, H = atan(tan(V) res_x/res_y); v^t from the null
 * condition, v rescaled so that v^t = -1, p_mu = g_{mu nu} v^nu at (0, r0, theta0, 0).
 *
 * Conventions
 *   - Every function returns GT_OK (0) or a negative GT_ERR_* code; nothing throws.
 *   - Output arrays of gt_trace / gt_trace_batch are DEVICE memory owned by the
 *     caller, one element per ray, flat index j*res_x + i (rows along theta).
 *     t, r, theta, phi are float64 (also in the FP32-mixed mode); status is uint8
 *     (GT_RAY_*), nsteps is uint32 and counts the terminal step.
 *   - Calls are asynchronous on the context's stream (a borrowed cudaStream_t,
 *     0 = legacy default stream); gt_sync waits for it.  Output pointers must stay
 *     valid until the work completes.
 *   - A context is bound to one device, is not thread-safe, and owns only small
 *     scratch memory (queue counters, camera descriptors), freed by gt_destroy.
 */
#ifndef GEOTRACE_H
#define GEOTRACE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define GT_OK 0
#define GT_ERR_INVALID_ARG (-1)    /* bad parameter, null or misaligned pointer */
#define GT_ERR_NOT_CONFIGURED (-2) /* spacetime or camera not set */
#define GT_ERR_CUDA (-3)           /* a CUDA runtime call failed */
#define GT_ERR_OOM (-4)            /* device allocation failed */
#define GT_ERR_TIMEOUT (-5)        /* the device watchdog stopped the launch */
#define GT_ERR_UNSUPPORTED (-6)    /* no sm_103 device / feature not built */

/* per-ray status */
#define GT_RAY_ESCAPED 0
#define GT_RAY_HORIZON 1
#define GT_RAY_MAXSTEPS 2
#define GT_RAY_NONFINITE 3
#define GT_RAY_TIMEOUT 4
#define GT_RAY_DISK 5 /* entered the ring volume (gt_trace_disk) */

/* arithmetic modes */
#define GT_MODE_FP64 0       /* FP64 end to end */
#define GT_MODE_FP32_MIXED 1 /* FP32 RK4 with compensated state; a zone r < r_switch stepped with
                              * an FP64 state (its field and stage arithmetic in double-float
                              * where the evaluation's range allows, else FP64) and H = 0
                              * re-projection.
                              * Runs in rounds (FP32 launch, zone launch, ...) and returns
                              * once the work has completed. */

/* option flags */
#define GT_FLAG_COMPAT_WEIGHTS 1 /* RK4 weights 0.1667 as printed in the listing (default 1/6) */
#define GT_FLAG_COMPAT_CAMERA 2  /* v^phi = alpha_i as in the listing (default alpha_i/sin theta0) */
#define GT_FLAG_ONE_SHOT 4       /* one ray per thread instead of the persistent ray queue */
#define GT_FLAG_GRAPH 8          /* replay the trace from a CUDA graph captured once per distinct
                                  * launch and cached in the context: FP64 is one persistent
                                  * launch; FP32-mixed runs its rounds under a conditional WHILE
                                  * node whose condition the device sets, so the call stays
                                  * asynchronous.  Not with GT_FLAG_ONE_SHOT. */
#define GT_FLAG_ZONE_FP64 256    /* FP32-mixed: step the zone in FP64 throughout instead of
                                  * double-float (two floats, ~48 bits, on the FP32 pipes) */
#define GT_FLAG_PRECISE_MN 16    /* FP32-mixed, Manko-Novikov: evaluate the metric's multipole
                                  * sums as closed-form series tails, free of the cancellation
                                  * that costs the plain FP32 form ~2 beta ulp(1) in its
                                  * exponents (about 100x closer to FP64; ~20 % slower) */
/* The paper's own numerics (appendix listing, propagation kernel), GT_MODE_FP64 only;
 * with GT_FLAG_COMPAT_WEIGHTS and GT_FLAG_COMPAT_CAMERA they reproduce the listing. */
#define GT_FLAG_FD_DERIVS 32     /* forward-difference metric derivatives with the listing's
                                  * derPrecision 1e-8: three evaluations of g^{mu nu} per RK4
                                  * stage instead of the exact derivatives */
#define GT_FLAG_F32_IO 64        /* float32 kernel arguments and results as in the listing:
                                  * M, S, Q, the camera's initial state and the end position
                                  * t, r, theta, phi rounded to float32 (arithmetic in FP64) */
#define GT_FLAG_EULER 128        /* explicit Euler (Sec. 3.1.1) instead of RK4, same step rule */

typedef struct gt_ctx gt_ctx;

/* Launch and precision options; zero fields take the defaults noted. */
typedef struct gt_options {
    int block_size;          /* threads per block, multiple of 32 in [32, 256]; 0 = 128 */
    int blocks_per_sm;       /* persistent grid = min(blocks_per_sm, resident limit) * SMs; 0 = 4 */
    int flags;               /* GT_FLAG_* */
    int reproject_every;     /* FP32-mixed: steps between H = 0 re-projections; 0 = 4096 */
    double r_switch;         /* FP32-mixed: zone r < r_switch; < 0 = none; 0 = automatic:
                                none for Kerr, 4M for Manko-Novikov */
    double timeout_seconds;  /* device watchdog (wall clock per launch); 0 = none */
    int rays_per_thread;     /* FP32-mixed: rays each thread integrates at once, 1 or 2 (two
                                independent RK4 chains interleaved); 0 = 1.  Two apply to
                                persistent single-camera traces without the watchdog, ring,
                                state arrays or per-ray parameters; others use one. */
} gt_options;

/* One camera of a batch (gt_trace_batch); same meaning as gt_set_spacetime and
 * gt_set_camera.  Rays of camera c occupy flat ids [offset_c, offset_c + res_x*res_y)
 * with offset_c the sum of the preceding cameras' pixel counts. */
typedef struct gt_camera_desc {
    double M, S, Q;
    double r0, theta0, fov_deg;
    int32_t res_x, res_y;
} gt_camera_desc;

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t owned by the caller, e.g. torch's current stream; NULL = the
 * legacy default stream).  Allocates the context's scratch memory.
 * Errors: GT_ERR_INVALID_ARG (out == NULL), GT_ERR_UNSUPPORTED (device is not
 * compute capability 10.3), GT_ERR_CUDA, GT_ERR_OOM. */
int gt_create(gt_ctx **out, int device, void *cuda_stream);

/* Synchronise the context's stream and free everything the context owns. */
int gt_destroy(gt_ctx *ctx);

/* Replace the stream later calls are issued on (the old stream is not synchronised). */
int gt_set_stream(gt_ctx *ctx, void *cuda_stream);

/* Spacetime (Sec. 2.2): mass M > 0, spin S with |S| < M^2 (Sec. 2.2.2), Q the
 * Manko-Novikov quadrupole deviation q (Sec. 2.2.3); Q != 0 requires S != 0
 * because alpha divides by S/M.  Errors: GT_ERR_INVALID_ARG. */
int gt_set_spacetime(gt_ctx *ctx, double M, double S, double Q);

/* Pinhole camera (Sec. 3.3.1): position (0, r0, theta0, 0) with r0 > 0,
 * 0 < theta0 < pi (radians), full vertical field of view 0 < fov_deg < 180
 * (degrees), res_x, res_y >= 1.  The camera must sit where g_tt < 0 (outside
 * the ergoregion); gt_trace reports GT_ERR_INVALID_ARG otherwise. */
int gt_set_camera(gt_ctx *ctx, double r0, double theta0, double fov_deg, int res_x, int res_y);

/* Options for later calls; opts == NULL restores the defaults. */
int gt_set_options(gt_ctx *ctx, const gt_options *opts);

/* Trace every pixel of the configured camera (n_steps >= 0 RK4 steps at most,
 * step_precision > 0, mode GT_MODE_*).  Outputs: device arrays of res_x*res_y
 * elements, 8-byte aligned for the float64 ones; any of t, r, theta, phi, status,
 * nsteps may be NULL to skip it.  Asynchronous; on a watchdog stop the call
 * returns GT_ERR_TIMEOUT after synchronising, and unfinished rays carry
 * GT_RAY_TIMEOUT.  Errors: GT_ERR_NOT_CONFIGURED, GT_ERR_INVALID_ARG, GT_ERR_CUDA,
 * GT_ERR_TIMEOUT. */
int gt_trace(gt_ctx *ctx, int64_t n_steps, double step_precision, int mode, double *t, double *r,
             double *theta, double *phi, uint8_t *status, uint32_t *nsteps);

/* As gt_trace, restricted to the contiguous flat pixel range [first, first + count)
 * of the configured camera; output element k belongs to pixel first + k.  Used to
 * shard one image across devices or processes and to sample long runs.
 * Errors as gt_trace, plus GT_ERR_INVALID_ARG when the range leaves the image. */
int gt_trace_range(gt_ctx *ctx, int64_t first, int64_t count, int64_t n_steps,
                   double step_precision, int mode, double *t, double *r, double *theta,
                   double *phi, uint8_t *status, uint32_t *nsteps);

/* As gt_trace for the `n` flat pixel indices in `pixels` (a DEVICE int64 array, each in
 * [0, res_x*res_y); the caller keeps them in range -- they are not checked on the host);
 * output element k belongs to pixels[k].  Used to subsample large images.
 * Errors as gt_trace. */
int gt_trace_pixels(gt_ctx *ctx, const int64_t *pixels, int64_t n, int64_t n_steps,
                    double step_precision, int mode, double *t, double *r, double *theta,
                    double *phi, uint8_t *status, uint32_t *nsteps);

/* As gt_trace, but the outputs are HOST arrays: the library copies the results
 * back (through its own device staging buffers) and returns after they arrived. */
int gt_trace_host(gt_ctx *ctx, int64_t n_steps, double step_precision, int mode, double *t,
                  double *r, double *theta, double *phi, uint8_t *status, uint32_t *nsteps);

/* Trace n_cams cameras (host array of descriptors) in one persistent launch.  Outputs
 * are device arrays over the flattened id space (sum of res_x*res_y).  Errors as gt_trace. */
int gt_trace_batch(gt_ctx *ctx, const gt_camera_desc *cams, int n_cams, int64_t n_steps,
                   double step_precision, int mode, double *t, double *r, double *theta,
                   double *phi, uint8_t *status, uint32_t *nsteps);

/* Trace n rays whose spacetime and camera differ per ray (the surrogate's training
 * data): ray k starts at (0, r0, theta0[k], 0) of the spacetime (M, S = spin[k] M^2,
 * Q = q[k]) -- spin[k] is the dimensionless a/M -- with direction v = (v^t, -1,
 * beta[k], alpha[k]/sin theta0[k]) completed as in the camera (Sec. 3.3.1).  All
 * per-ray inputs are float64 DEVICE arrays of n elements; outputs as gt_trace over n
 * rays.  A ray whose camera position is inside the ergoregion gets GT_RAY_NONFINITE.
 * Errors as gt_trace. */
int gt_trace_rays(gt_ctx *ctx, int64_t n, const double *alpha, const double *beta,
                  const double *spin, const double *q, const double *theta0, double M, double r0,
                  int64_t n_steps, double step_precision, int mode, double *t, double *r,
                  double *theta, double *phi, uint8_t *status, uint32_t *nsteps);

/* The paper's ring (Sec. 3.3.3 "Redshift"; the ring renders of Sec. 5): as gt_trace, with
 * the region r_in <= r <= r_out, |r cos theta| <= half_thickness (a solid ring around the
 * equator; 0 < r_in < r_out, half_thickness > 0) as an extra exit, tested after every step
 * after the escape test and before the horizon test.  Rays that enter it end with status
 * GT_RAY_DISK and get the redshift factor z = lambda_O / lambda_S =
 * (p . u_S) / (p . u_O): u_S the 4-velocity of a ring element on the circular orbit through
 * the hit point (p_r = p_theta = 0, dp_r/dtau = 0, p_t = -1, the prograde root, normalised
 * to g^{mu nu} p_mu p_nu = -1), u_O the static observer at the camera.  z (a DEVICE float64
 * array of res_x*res_y elements, 8-byte aligned) is NaN for the other rays and where no
 * timelike circular orbit exists.  Other outputs and errors as gt_trace, plus
 * GT_ERR_INVALID_ARG for a bad ring or z == NULL. */
int gt_trace_disk(gt_ctx *ctx, double r_in, double r_out, double half_thickness, int64_t n_steps,
                  double step_precision, int mode, double *t, double *r, double *theta,
                  double *phi, uint8_t *status, uint32_t *nsteps, double *z);

/* Integrate n rays (or massive particles) of the configured spacetime from arbitrary
 * states: SoA DEVICE float64 arrays t, r, theta, phi, p_t, p_r, p_theta, p_phi of n
 * elements hold the initial state and receive the end state (in place).  Null rays
 * have g^{mu nu} p_mu p_nu = 0, timelike orbits -1 (Sec. 3.2.1 "Orbits": H = -1/2); the
 * step rule and exit tests are gt_trace's with the escape radius r_escape (> 0).  A ray
 * that stopped at MAXSTEPS continues from its returned state on the next call: the
 * state is the whole integrator state, so n1 steps followed by n2 steps give the same
 * bits as n1 + n2 steps in one call (GT_MODE_FP64) -- a checkpoint.  status and nsteps
 * (steps of this call) as gt_trace, optional.  No camera is needed.  Errors:
 * GT_ERR_NOT_CONFIGURED (no spacetime), GT_ERR_INVALID_ARG, GT_ERR_CUDA. */
int gt_trace_states(gt_ctx *ctx, int64_t n, double *t, double *r, double *theta, double *phi,
                    double *p_t, double *p_r, double *p_theta, double *p_phi, double r_escape,
                    int64_t n_steps, double step_precision, int mode, uint8_t *status,
                    uint32_t *nsteps);

/* ---------------------------------------------------------------------------------
 * Surrogate: an MLP (alpha, beta, spin a/M, q, theta0) -> (escape logit, unit end
 * direction) with layers 16(10 used) -> 256 -> 256 -> 256 -> 256 -> 16(4 used), SiLU,
 * on tcgen05 tensor cores with FP32 accumulation: FP16 weights and activations in the
 * forward products, BF16 in the backward products, FP32 master weights and AdamW.  Trained on rays traced by the integrator; the integrator
 * is its fallback.  Not part of the paper's method. */
typedef struct gt_surrogate gt_surrogate;

/* Input ranges the features are normalised over: camera distance r0 and field of view
 * (pixel directions), spin a/M in [0, spin_max], |q| <= q_max, theta0 range (rad). */
typedef struct gt_surrogate_norm {
    double r0, fov_deg, spin_max, q_max, theta0_min, theta0_max;
} gt_surrogate_norm;

typedef struct gt_train_cfg {
    int epochs;          /* passes over the training rays */
    int batch;           /* rows per step, multiple of 128, <= 2^20 */
    double lr;           /* peak AdamW learning rate (cosine decay to 0) */
    double weight_decay; /* decoupled weight decay (weights only) */
    double dir_weight;   /* weight of the squared end-direction error of escaped rays */
} gt_train_cfg;

/* Number of float32 parameters (weights row-major [out][in], then bias, per layer). */
int gt_surrogate_num_params(int64_t *out);

/* Create a network on `device` with seeded LeCun-normal weights and zero biases. */
int gt_surrogate_create(int device, const gt_surrogate_norm *norm, uint64_t seed,
                        gt_surrogate **out);
int gt_surrogate_destroy(gt_surrogate *s);

/* Copy the float32 parameters to / from a host array of gt_surrogate_num_params. */
int gt_surrogate_get_params(gt_surrogate *s, float *host, int64_t n);
int gt_surrogate_set_params(gt_surrogate *s, const float *host, int64_t n);

/* Network outputs for n samples (device float64 inputs) into `out` (device float32,
 * n x 4: logit, direction x, y, z).  Runs on the context's stream. */
int gt_surrogate_eval(gt_ctx *ctx, gt_surrogate *s, int64_t n, const double *alpha,
                      const double *beta, const double *spin, const double *q,
                      const double *theta0, float *out);

/* One forward and backward pass over n <= 2^20 samples (one batch) with labels from
 * traced rays (status, end theta, end phi): loss = mean(BCE(logit, escaped) +
 * dir_weight * escaped * |d_pred - d_end|^2).  Gradients to a host array of
 * gt_surrogate_num_params floats; loss to *loss_host.  For checking the gradients. */
int gt_surrogate_grad(gt_ctx *ctx, gt_surrogate *s, int64_t n, const double *alpha,
                      const double *beta, const double *spin, const double *q,
                      const double *theta0, const uint8_t *status, const double *th_end,
                      const double *ph_end, float dir_weight, float *grads_host,
                      float *loss_host);

/* Train on n samples (device arrays; inputs and the traced labels) for cfg->epochs
 * passes of n / cfg->batch full batches.  Mean loss per epoch to loss_per_epoch (host,
 * cfg->epochs floats) when not NULL.  Synchronous. */
int gt_surrogate_train(gt_ctx *ctx, gt_surrogate *s, const gt_train_cfg *cfg, int64_t n,
                       const double *alpha, const double *beta, const double *spin,
                       const double *q, const double *theta0, const uint8_t *status,
                       const double *th_end, const double *ph_end, float *loss_per_epoch);

/* Gates of gt_surrogate_infer (zero fields disable a gate). */
typedef struct gt_gate_cfg {
    float tau;         /* network pixels need |logit| >= tau */
    double band;       /* Kerr photon-ring band: |min_r R(r)/(E^2 r^4)| < band falls back
                          (97 geometric radii from 1.0001 r_+ to r0, from the pixel's
                          constants of motion) */
    double axis;       /* rays that can reach |sin theta| < axis fall back (Kerr turning
                          point of the theta motion from the pixel's constants of motion;
                          the Kerr values of M and S estimate it for Manko-Novikov); in [0, 1) */
    float dir_tol;     /* escaping predictions whose direction vector's length is off 1 by
                          more than dir_tol fall back */
    int probe_stride;  /* integrator probes every probe_stride pixels (0 = none) */
    float probe_tol;   /* largest accepted spread of the probe errors over a cell */
} gt_gate_cfg;

/* Image of the configured camera through the surrogate, with the integrator as judge and
 * fallback.  The network runs on every pixel first.  With gate->probe_stride > 0 the pixels
 * (i, j) with i, j multiples of probe_stride or the last column/row (images of at least
 * 2 x 2 pixels) are probes: the integrator traces them, their exact results go to the image,
 * and each probe records the network's error vector (exact unit end direction minus the
 * predicted one).  A pixel inside a probe cell is then taken from the network only when the
 * cell's four corners are classified alike by the integrator and the network -- all escaped,
 * or all not escaping with one common integrator status (HORIZON, or MAXSTEPS for rays still
 * bound at the step cap), which the pixel takes -- the pixel's own prediction agrees with
 * theirs, and, when escaping, the corners' error vectors differ by less than probe_tol
 * (|e00 - e11| and |e01 - e10|); its end direction is the network's plus the bilinear
 * interpolation of the corner errors.  In every case a network pixel also passes the gates
 * of gt_gate_cfg.  Network pixels get status ESCAPED with end theta, phi from the
 * (corrected) direction, or HORIZON (MAXSTEPS inside an all-MAXSTEPS probe cell) with NaN
 * angles; t and r are NaN and nsteps 0 for them.  All other pixels are traced by the
 * integrator (mode, n_steps, step_precision as gt_trace) and written in place: in one
 * launch with the probes, the pixels that the network's answers alone send there (a gate,
 * or a prediction differing from a corner's), in a second one those that the probes'
 * results send there.  Outputs as gt_trace (device, res_x*res_y each, none may be NULL);
 * *n_fallback receives the number of integrated pixels besides the probes, *n_probes the
 * number of probes (either may be NULL).  Errors: GT_ERR_INVALID_ARG (gate NULL or out of
 * range, NULL outputs) and those of gt_trace.  Synchronous. */
int gt_surrogate_infer(gt_ctx *ctx, gt_surrogate *s, const gt_gate_cfg *gate, int64_t n_steps,
                       double step_precision, int mode, double *t, double *r, double *theta,
                       double *phi, uint8_t *status, uint32_t *nsteps, int64_t *n_fallback,
                       int64_t *n_probes);

/* Copy the float32 gradient of the last training step (or of gt_surrogate_grad) to a host
 * array of gt_surrogate_num_params floats. */
int gt_surrogate_get_grads(gt_surrogate *s, float *host, int64_t n);

/* Largest batch gt_trace_batch_noalloc accepts. */
#define GT_NOALLOC_MAX_CAMS 64

/* gt_trace_batch for callers that cannot allocate device memory -- for example code
 * inside a host framework that owns the whole device-memory budget through its own
 * pool, or latency-critical loops where cudaMalloc's implicit device synchronisation
 * is not acceptable.  The paper has no counterpart.
 *
 * No context is needed and nothing is allocated: the queue counter and the camera
 * descriptors live in one static device array of the library (about 22 KB for
 * GT_NOALLOC_MAX_CAMS cameras), which every device that loads the library holds until
 * the process exits.  The caller still owns and passes the device output arrays
 * (layout as gt_trace_batch; default launch options, no watchdog).  In FP32-mixed
 * mode the zone steps run inline in the FP32 kernel (H = 0 re-projection every
 * 4096 steps, the context's default), because the park lists gt_trace_batch uses would
 * need allocated memory; FP64 results are identical to gt_trace_batch's.  Each call
 * looks up that array's device address on `device` once per process (with the device
 * current) and keeps it, so the entry point must not be used on a device across a
 * cudaDeviceReset of that device.  The call uploads the descriptors and synchronises
 * `cuda_stream` to check them, so it cannot be issued while that stream is being
 * captured; it then clears the queue counter and launches asynchronously.
 * All calls share the array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must not be issued.
 * Errors: GT_ERR_INVALID_ARG (including n_cams > GT_NOALLOC_MAX_CAMS, or a camera
 * inside the ergoregion), GT_ERR_UNSUPPORTED (not compute capability 10.3), GT_ERR_CUDA. */
int gt_trace_batch_noalloc(int device, void *cuda_stream, const gt_camera_desc *cams, int n_cams,
                           int64_t n_steps, double step_precision, int mode, double *t, double *r,
                           double *theta, double *phi, uint8_t *status, uint32_t *nsteps);

/* Autotuner: time gt_trace_range over `trial_rays` central pixels of the configured
 * camera for `trial_steps` steps with every candidate launch shape (block size in
 * {64, 128, 192, 256} x resident blocks per SM in {1, 2, 3, 4, 6, 8}, within the
 * kernel's occupancy limit, x rays per thread in {1, 2} for GT_MODE_FP32_MIXED), keep the
 * fastest in the context's options, and report it (best_rays_per_thread may be NULL).
 * With cache_path != NULL the result is looked up first and appended after tuning,
 * keyed by mode, spacetime kind, SM count and device name (plain text lines).
 * Synchronous.  Errors: GT_ERR_NOT_CONFIGURED, GT_ERR_INVALID_ARG, GT_ERR_CUDA. */
int gt_autotune(gt_ctx *ctx, int mode, int64_t trial_rays, int64_t trial_steps,
                double step_precision, const char *cache_path, int *best_block,
                int *best_blocks_per_sm, int *best_rays_per_thread, double *best_steps_per_s);

/* Wait for all work issued by the context. */
int gt_sync(gt_ctx *ctx);

/* RK4 steps the last trace of the context took in the zone of GT_MODE_FP32_MIXED (0 for
 * FP64 traces and for mixed traces that never entered it; compare with the sum of nsteps
 * for the zone's share of the work) and, in zone_f64_evals (may be NULL), the field
 * evaluations of those steps done in FP64 (all of them with GT_FLAG_ZONE_FP64; otherwise
 * those outside the double-float range).  Synchronises the context's stream. */
int gt_get_stats(gt_ctx *ctx, int64_t *zone_steps, int64_t *zone_f64_evals);

/* Number of streaming multiprocessors of the context's device (for grid sizing). */
int gt_device_sm_count(gt_ctx *ctx, int *out);

/* Measure the device's FMA throughput (FP64 when fp64 != 0, else FP32) with a
 * synthetic kernel of independent FMA chains: grid 8 x SMs x 256 threads, `iters`
 * x 128 FMAs per thread, timed with CUDA events on the legacy stream.  Writes
 * FLOP/s (2 per FMA).  Used as the ALU roofline denominator; not part of the
 * paper's method.  Errors: GT_ERR_INVALID_ARG, GT_ERR_CUDA. */
int gt_measure_fma_peak(int device, int fp64, int iters, double *flops_per_s);

/* BF16 tensor-core GEMM on `device` / `cuda_stream` (tcgen05, FP32 accumulation in
 * tensor memory), the building block of the surrogate network's training and
 * inference (which also runs it on FP16 operands internally):
 * C[m, n] (+)= act(sum_k A[m, k] B[n, k] + bias[n]) for m < M, n < N.
 * A (m, k) is read at A[m * a_sm + k * a_sk] and B (n, k) at B[n * b_sn + k * b_sk]
 * (bf16 device arrays, any strides, so transposed views need no copy); bias is an
 * optional float32[N]; act 0 = identity, 1 = SiLU; C is float32 row-major with
 * leading dimension ldc >= N.  accumulate != 0 adds into C atomically; splits > 1
 * splits K over that many CTAs (implies accumulate: C must be zeroed first).
 * bn (tile width) is one of 16, 32, 64, 128, 256.  Asynchronous on the stream.
 * Not part of the paper's method.  Errors: GT_ERR_INVALID_ARG, GT_ERR_CUDA. */
int gt_gemm_bf16(int device, void *cuda_stream, int M, int N, int K, const void *A, int64_t a_sm,
                 int64_t a_sk, const void *B, int64_t b_sn, int64_t b_sk, const float *bias,
                 int act, float *C, int64_t ldc, int accumulate, int splits, int bn);

/* Static description of an error code; never NULL. */
const char *gt_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GEOTRACE_H */
