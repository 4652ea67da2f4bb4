// trace.cu -- camera set-up and the persistent RK4 ray-queue kernels (sm_103a).
//
// One lane integrates one ray.  In the persistent form a grid of a few blocks per
// SM loops until the global ray queue is empty: whenever lanes of a warp finish,
// the warp counts them with __ballot_sync, one elected lane claims that many new
// ray ids with a single atomicAdd, and the lanes rebuild their initial data from
// the pixel index (camera initialisation is fused -- there are no input arrays).
// Rays that stop early (horizon) therefore do not leave their lanes idle.  Every
// ray runs the same instruction sequence whatever lane, warp or launch shape it
// lands in, so results are bitwise independent of the launch configuration.
//
// Method (Sec. 3.1.2 RK4; appendix listing's propagation kernel for the step rule
// and exit tests):
//   k1 = F(x);  h = |sp / k1.q^t|;  k2 = F(x + h/2 k1);  k3 = F(x + h/2 k2);
//   k4 = F(x + h k3);  x += h w (k1 + 2 k2 + 2 k3 + k4),  w = 1/6 (0.1667 compat);
//   then r > 1.5 r0 -> ESCAPED, else h < sp 3e-5 -> HORIZON, else n_steps -> MAXSTEPS;
//   a non-finite step -> NONFINITE keeping the last finite state.
// Only (r, theta, p_r, p_theta) enter F; t and phi are quadratures and p_t, p_phi
// are constants of motion, so the state is 6 evolving numbers plus 2 constants.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/geotrace.h"
#include "camera.cuh"
#include "compensated.cuh"
#include "internal.cuh"
#include "spacetime.cuh"
#include "zone_df.cuh"

namespace gt {

#define FULL_MASK 0xffffffffu

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------ camera set-up
// Spacetime constants (Sec. 2.2.2: a = S/M; Sec. 2.2.3: alpha, k, beta), the pixel
// ranges V = tan(FOV/2)/r0 and H = atan(tan(V) res_x/res_y) of the listing, and the
// lower metric at the camera (inverse of g^{mu nu}'s (t, phi) block and diagonal).
__device__ void setup_desc(CamDesc &d, int flags, double r_switch)
{
    SpacetimeC st = {};
    st.M = d.M;
    if (d.Q != 0.0) {
        st.kind = KIND_MN;
        const double sm = d.S / d.M;
        const double al = (-d.M + sqrt(d.M * d.M - sm * sm)) / sm;
        const double k = d.M * (1.0 - al * al) / (1.0 + al * al);
        st.alpha = al;
        st.k = k;
        st.ik = 1.0 / k;
        st.beta = d.Q * d.M * d.M * d.M / (k * k * k);
        st.two_beta = 2.0 * st.beta;
        st.three_beta2 = 3.0 * st.beta * st.beta;
        st.c_g = (1.0 - al * al) * (1.0 - al * al) / (k * k);
        st.w_inf = 4.0 * k * al / (1.0 - al * al);
        st.k2 = k * k;
        st.inv_k2 = 1.0 / (k * k);
        st.two_k = 2.0 * k;
        st.r_plus = d.M + k;
    } else {
        st.kind = KIND_KERR;
        st.a = d.S / d.M;
        st.a2 = st.a * st.a;
        st.r_plus = d.M + sqrt(d.M * d.M - st.a2);
    }
    d.st = st;
    d.st_df = to_df(st);
    d.V = tan(0.5 * d.fov_deg / 180.0 * M_PI) / d.r0;
    d.H = atan(tan(d.V) * (double)d.res_x / (double)d.res_y);
    d.inv_sin_th0 = (flags & GT_FLAG_COMPAT_CAMERA) ? 1.0 : 1.0 / sin(d.th0);
    double g[5];
    upper_metric(st, d.r0, d.th0, g);
    const double det = g[0] * g[2] - g[1] * g[1];
    d.gl_tt = g[2] / det;
    d.gl_tph = -g[1] / det;
    d.gl_phph = g[0] / det;
    d.gl_rr = 1.0 / g[3];
    d.gl_thth = 1.0 / g[4];
    d.r_escape = 1.5 * d.r0;
    if (r_switch > 0.0) {
        d.r_switch = r_switch;
    } else if (r_switch < 0.0) {
        d.r_switch = 0.0;
    } else if (st.kind == KIND_KERR) {
        // Kerr needs no FP64 zone: with the compensated FP32 state, escape/capture and the
        // end directions agree with the FP64 path from a = 0.5M to 0.99M and inclinations
        // 5-85 deg, while a zone covering the horizon approach costs 7-35x in time
        d.r_switch = 0.0;
    } else {
        // Manko-Novikov: the photon region and the horizon approach in FP64 (its metric
        // exponentials come close to the FP32 range there, and FP32 there misclassifies
        // about 0.2 % of the rays of the listing's spacetime)
        d.r_switch = 4.0 * d.M;
    }
    d.valid = (d.gl_tt < 0.0 && isfinite(d.gl_tt) && isfinite(d.gl_phph) && isfinite(d.gl_rr) &&
               isfinite(d.gl_thth) && d.gl_rr > 0.0 && d.gl_thth > 0.0)
                  ? 1
                  : 0;
}

__global__ void camera_setup_kernel(CamDesc *cams, int n, int flags, double r_switch)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    CamDesc d = cams[c];
    setup_desc(d, flags, r_switch);
    cams[c] = d;
}

cudaError_t launch_camera_setup(CamDesc *d_cams, int n_cams, int flags, double r_switch,
                                cudaStream_t s)
{
    const int block = 64;
    camera_setup_kernel<<<(n_cams + block - 1) / block, block, 0, s>>>(d_cams, n_cams, flags,
                                                                       r_switch);
    return cudaGetLastError();
}

template <int KIND>
__device__ __forceinline__ void rates_any(const SpacetimeC &st, double r, double s, double cs,
                                          double pr, double pth, double pt, double pph,
                                          Rates<double> &o)
{
    if (KIND == KIND_KERR || (KIND == KIND_ANY && st.kind == KIND_KERR))
        kerr_rates_sc<double>(st, r, s, cs, pr, pth, pt, pph, o);
    else
        mn_rates_sc<double>(st, r, s, cs, pr, pth, pt, pph, o);
}

// The listing's numerics (KIND_FD): the inverse metric at (r, theta) and the forward
// differences d_r g ~ (g(r + delta, theta) - g(r, theta))/delta, d_theta likewise, with
// delta = derPrecision = 1e-8 -- three metric evaluations -- contracted into
// dp = -1/2 d g^{nu sigma} p_nu p_sigma component by component.
constexpr double FD_DELTA = 1e-8;

__device__ __forceinline__ double fd_quad(const double d[5], double pr, double pth, double pt,
                                          double pph)
{
    return d[0] * pt * pt + 2.0 * d[1] * pt * pph + d[2] * pph * pph + d[3] * pr * pr +
           d[4] * pth * pth;
}

__device__ __forceinline__ void rates_fd(const SpacetimeC &st, double r, double th, double pr,
                                         double pth, double pt, double pph, Rates<double> &o)
{
    double g0[5], gr[5], gt[5], dr[5], dt[5];
    upper_metric(st, r, th, g0);
    upper_metric(st, r + FD_DELTA, th, gr);
    upper_metric(st, r, th + FD_DELTA, gt);
#pragma unroll
    for (int i = 0; i < 5; i++) {
        dr[i] = (gr[i] - g0[i]) / FD_DELTA;
        dt[i] = (gt[i] - g0[i]) / FD_DELTA;
    }
    o.dt = g0[0] * pt + g0[1] * pph;
    o.dph = g0[1] * pt + g0[2] * pph;
    o.dr = g0[3] * pr;
    o.dth = g0[4] * pth;
    o.dpr = -0.5 * fd_quad(dr, pr, pth, pt, pph);
    o.dpth = -0.5 * fd_quad(dt, pr, pth, pt, pph);
}

// One FP64 RK4 step; returns h and writes the candidate state to y.  sin and cos of
// theta are evaluated once per step and rotated to the later stages by their small
// angle offsets (Taylor series, FP64 accurate); the forward-difference kind evaluates
// its metric at each stage's theta as the listing does.
template <int KIND>
__device__ __forceinline__ double rk4_step64(const SpacetimeC &st, const Ray64 &x, double sp,
                                             double w6, Ray64 &y)
{
    Rates<double> k1, k2, k3, k4;
    double h, hh;
    if constexpr (KIND == KIND_FD) {
        rates_fd(st, x.r, x.th, x.pr, x.pth, x.pt, x.pph, k1);
        h = fabs(sp / k1.dt);
        hh = 0.5 * h;
        rates_fd(st, x.r + hh * k1.dr, x.th + hh * k1.dth, x.pr + hh * k1.dpr,
                 x.pth + hh * k1.dpth, x.pt, x.pph, k2);
        rates_fd(st, x.r + hh * k2.dr, x.th + hh * k2.dth, x.pr + hh * k2.dpr,
                 x.pth + hh * k2.dpth, x.pt, x.pph, k3);
        rates_fd(st, x.r + h * k3.dr, x.th + h * k3.dth, x.pr + h * k3.dpr,
                 x.pth + h * k3.dpth, x.pt, x.pph, k4);
    } else {
        double s1, c1, s, c;
        sincos(x.th, &s1, &c1);
        rates_any<KIND>(st, x.r, s1, c1, x.pr, x.pth, x.pt, x.pph, k1);
        h = fabs(sp / k1.dt);
        hh = 0.5 * h;
        rotate_sc(s1, c1, x.th, hh * k1.dth, &s, &c);
        rates_any<KIND>(st, x.r + hh * k1.dr, s, c, x.pr + hh * k1.dpr, x.pth + hh * k1.dpth,
                        x.pt, x.pph, k2);
        rotate_sc(s1, c1, x.th, hh * k2.dth, &s, &c);
        rates_any<KIND>(st, x.r + hh * k2.dr, s, c, x.pr + hh * k2.dpr, x.pth + hh * k2.dpth,
                        x.pt, x.pph, k3);
        rotate_sc(s1, c1, x.th, h * k3.dth, &s, &c);
        rates_any<KIND>(st, x.r + h * k3.dr, s, c, x.pr + h * k3.dpr, x.pth + h * k3.dpth, x.pt,
                        x.pph, k4);
    }
    const double hw = h * w6;
    y.t = x.t + hw * (k1.dt + 2.0 * k2.dt + 2.0 * k3.dt + k4.dt);
    y.r = x.r + hw * (k1.dr + 2.0 * k2.dr + 2.0 * k3.dr + k4.dr);
    y.th = x.th + hw * (k1.dth + 2.0 * k2.dth + 2.0 * k3.dth + k4.dth);
    y.ph = x.ph + hw * (k1.dph + 2.0 * k2.dph + 2.0 * k3.dph + k4.dph);
    y.pr = x.pr + hw * (k1.dpr + 2.0 * k2.dpr + 2.0 * k3.dpr + k4.dpr);
    y.pth = x.pth + hw * (k1.dpth + 2.0 * k2.dpth + 2.0 * k3.dpth + k4.dpth);
    y.pt = x.pt;
    y.pph = x.pph;
    return h;
}

// One explicit Euler step (Sec. 3.1.1): x += h F(x) with the same step rule.
template <int KIND>
__device__ __forceinline__ double euler_step64(const SpacetimeC &st, const Ray64 &x, double sp,
                                               Ray64 &y)
{
    Rates<double> k1;
    if constexpr (KIND == KIND_FD) {
        rates_fd(st, x.r, x.th, x.pr, x.pth, x.pt, x.pph, k1);
    } else {
        double s1, c1;
        sincos(x.th, &s1, &c1);
        rates_any<KIND>(st, x.r, s1, c1, x.pr, x.pth, x.pt, x.pph, k1);
    }
    const double h = fabs(sp / k1.dt);
    y.t = x.t + h * k1.dt;
    y.r = x.r + h * k1.dr;
    y.th = x.th + h * k1.dth;
    y.ph = x.ph + h * k1.dph;
    y.pr = x.pr + h * k1.dpr;
    y.pth = x.pth + h * k1.dpth;
    y.pt = x.pt;
    y.pph = x.pph;
    return h;
}

template <int KIND>
__device__ __forceinline__ double step64(const TraceArgs &A, const SpacetimeC &st, const Ray64 &x,
                                         Ray64 &y)
{
    if (A.euler) return euler_step64<KIND>(st, x, A.sp, y);
    return rk4_step64<KIND>(st, x, A.sp, A.w6, y);
}

// ------------------------------------------------------------------ the zone in double-float
// The FP32-mixed path's zone steps an FP64 state.  Within a step the stage arithmetic --
// the stage points, the sin/cos rotation, the field (Manko-Novikov, or Kerr when a zone
// is set for it), the stage sums and the step length -- runs in double-float
// (zone_df.cuh) on the FP32 pipes; the state is converted once into double-float at the
// start of the step, the increments once back, and added in FP64.  A field evaluation
// outside the double-float range (Manko-Novikov exponents out of bounds, or a rate that
// is not finite) takes FP64; n_f64 counts those evaluations.
template <int KIND>
__device__ __forceinline__ void zone_rates(const SpacetimeC &st, const SpacetimeT<DF> *sd, DF r,
                                           DF s, DF cs, DF pr, DF pth, DF pt, DF pph,
                                           Rates<DF> &o, uint32_t &n_f64)
{
    const bool mn = KIND == KIND_MN || (KIND == KIND_ANY && st.kind == KIND_MN);
    if (mn) {
        if (mn_rates_df(*sd, r, s, cs, pr, pth, pt, pph, o)) return;
    } else if (KIND != KIND_FD) {
        kerr_rates_sc<DF>(*sd, r, s, cs, pr, pth, pt, pph, o);
        if (isfinite(o.dt.hi) && isfinite(o.dr.hi) && isfinite(o.dth.hi) &&
            isfinite(o.dph.hi) && isfinite(o.dpr.hi) && isfinite(o.dpth.hi))
            return;
    }
    ++n_f64;
    Rates<double> o64;
    rates_any<KIND>(st, df_to(r), df_to(s), df_to(cs), df_to(pr), df_to(pth), df_to(pt),
                    df_to(pph), o64);
    o.dt = DF(o64.dt);
    o.dr = DF(o64.dr);
    o.dth = DF(o64.dth);
    o.dph = DF(o64.dph);
    o.dpr = DF(o64.dpr);
    o.dpth = DF(o64.dpth);
}

__device__ __forceinline__ DF df_twice(DF a) { return DF(2.0f * a.hi, 2.0f * a.lo); }

// One RK4 step of the zone: the stages of rk4_step64 (stage points x + h/2 k1, x + h/2 k2,
// x + h k3; weights 1, 2, 2, 1 times h w6; h = |sp / k1.dt|) in a rolled stage loop, so one
// copy of the double-float field is compiled.  sd: the spacetime constants in
// double-float; sp_df, w6_df: step precision and RK4 weight in double-float.
template <int KIND>
__device__ __forceinline__ double rk4_step_zone(const SpacetimeC &st, const SpacetimeT<DF> *sd,
                                                const Ray64 &x, DF sp_df, DF w6_df, Ray64 &y,
                                                uint32_t &n_f64)
{
    double s64, c64;
    sincos(x.th, &s64, &c64);
    const DF S1(s64), C1(c64), R0(x.r), PR0(x.pr), PTH0(x.pth), PT(x.pt), PPH(x.pph);
    Rates<DF> k, acc;
    DF h(0.0f, 0.0f), r = R0, pr = PR0, pth = PTH0, s = S1, c = C1;
#pragma unroll 1
    for (int stage = 0; stage < 4; stage++) {
        zone_rates<KIND>(st, sd, r, s, c, pr, pth, PT, PPH, k, n_f64);
        if (stage == 0) {
            h = sp_df * rcp_t(k.dt);
            if (h.hi < 0.0f) h = -h;
            acc = k;
        } else if (stage < 3) {
            acc.dt = acc.dt + df_twice(k.dt);
            acc.dr = acc.dr + df_twice(k.dr);
            acc.dth = acc.dth + df_twice(k.dth);
            acc.dph = acc.dph + df_twice(k.dph);
            acc.dpr = acc.dpr + df_twice(k.dpr);
            acc.dpth = acc.dpth + df_twice(k.dpth);
        } else {
            acc.dt = acc.dt + k.dt;
            acc.dr = acc.dr + k.dr;
            acc.dth = acc.dth + k.dth;
            acc.dph = acc.dph + k.dph;
            acc.dpr = acc.dpr + k.dpr;
            acc.dpth = acc.dpth + k.dpth;
        }
        if (stage < 3) {
            const DF d = stage < 2 ? DF(0.5f * h.hi, 0.5f * h.lo) : h;
            r = R0 + d * k.dr;
            pr = PR0 + d * k.dpr;
            pth = PTH0 + d * k.dpth;
            const DF dth = d * k.dth;
            if (!rotate_sc_df(S1, C1, dth, &s, &c)) {
                double s2, c2;
                sincos(x.th + df_to(dth), &s2, &c2);
                s = DF(s2);
                c = DF(c2);
            }
        }
    }
    if (!isfinite(h.hi)) return nan("");
    const DF hw = h * w6_df;
    y.t = x.t + df_to(hw * acc.dt);
    y.r = x.r + df_to(hw * acc.dr);
    y.th = x.th + df_to(hw * acc.dth);
    y.ph = x.ph + df_to(hw * acc.dph);
    y.pr = x.pr + df_to(hw * acc.dpr);
    y.pth = x.pth + df_to(hw * acc.dpth);
    y.pt = x.pt;
    y.pph = x.pph;
    return df_to(h);
}

// ------------------------------------------------------------------ ring and redshift
__device__ __forceinline__ bool in_disk(const DiskArgs &dk, double r, double th)
{
    return r >= dk.r_in && r <= dk.r_out && fabs(r * cos(th)) <= dk.half_thickness;
}

// Redshift factor of the ray x at the ring (Sec. 3.3.3): the emitter moves on the
// circular orbit through (r, theta) -- p_r = p_theta = 0, dp_r/dtau = 0 and p_t = -1,
// i.e. A p_phi^2 - 2 B p_phi + C = 0 with (A, B, C) = d_r (g^{phi phi}, g^{t phi}, g^{tt}),
// the root with positive angular velocity, rescaled to g^{mu nu} p_mu p_nu = -1 -- and
// z = (p . u_S) / (p . u_O), u_O the static observer at the camera, p . u_O =
// p_t / sqrt(-g_tt(camera)).  Exact r derivatives by dual numbers (forward differences
// with KIND_FD).  NaN where no timelike circular orbit exists.
template <int KIND>
__device__ double redshift64(const SpacetimeC &st, double gl_tt_cam, const Ray64 &x)
{
    double g[3], A, B, C;
    if (KIND == KIND_FD) {
        double g0[5], gr[5];
        upper_metric(st, x.r, x.th, g0);
        upper_metric(st, x.r + FD_DELTA, x.th, gr);
        A = (gr[2] - g0[2]) / FD_DELTA;
        B = (gr[1] - g0[1]) / FD_DELTA;
        C = (gr[0] - g0[0]) / FD_DELTA;
        g[0] = g0[0];
        g[1] = g0[1];
        g[2] = g0[2];
    } else {
        D3<double> gd[3];
        if (st.kind == KIND_KERR)
            kerr_upper_tphi<double, D3<double>>(st, x.r, x.th, gd);
        else
            mn_upper_tphi<double, D3<double>>(st, x.r, x.th, gd);
        C = gd[0].r;
        B = gd[1].r;
        A = gd[2].r;
        g[0] = gd[0].v;
        g[1] = gd[1].v;
        g[2] = gd[2].v;
    }
    const double disc = B * B - A * C;
    if (!(disc >= 0.0) || A == 0.0) return nan("");
    const double sq = sqrt(disc);
    const double roots[2] = {(B + sq) / A, (B - sq) / A};
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const double pph = roots[k];
        const double ut = -g[0] + g[1] * pph;
        const double uph = -g[1] + g[2] * pph;
        const double norm = g[0] - 2.0 * g[1] * pph + g[2] * pph * pph;
        if (ut > 0.0 && uph / ut > 0.0 && norm < 0.0) {
            const double lam = 1.0 / sqrt(-norm);
            const double num = (x.pt * ut + x.pph * uph) * lam;
            return num / (x.pt / sqrt(-gl_tt_cam));
        }
    }
    return nan("");
}

__device__ __forceinline__ bool finite6(const Ray64 &y)
{
    return isfinite(y.t) && isfinite(y.r) && isfinite(y.th) && isfinite(y.ph) && isfinite(y.pr) &&
           isfinite(y.pth);
}

__device__ __forceinline__ double round_f32(double v) { return (double)(float)v; }

// End position of a ray that did not run (watchdog drain): position outputs only.
__device__ __forceinline__ void store_ray(const TraceArgs &A, int64_t id, double t, double r,
                                          double th, double ph, int status, uint32_t n)
{
    if (A.f32_io) {
        t = round_f32(t);
        r = round_f32(r);
        th = round_f32(th);
        ph = round_f32(ph);
    }
    if (A.t) A.t[id] = t;
    if (A.r) A.r[id] = r;
    if (A.th) A.th[id] = th;
    if (A.ph) A.ph[id] = ph;
    if (A.status) A.status[id] = (uint8_t)status;
    if (A.nsteps) A.nsteps[id] = n;
    if (A.z) A.z[id] = nan("");
}

// End state of a ray: position outputs (float32-rounded with f32_io), the redshift
// factor, and with state arrays the whole state written back.
__device__ __forceinline__ void store_full(const TraceArgs &A, int64_t id, const Ray64 &x,
                                           int status, uint32_t n, double z)
{
    store_ray(A, id, x.t, x.r, x.th, x.ph, status, n);
    if (A.z) A.z[id] = z;
    if (A.states.t) {
        A.states.t[id] = x.t;
        A.states.r[id] = x.r;
        A.states.th[id] = x.th;
        A.states.ph[id] = x.ph;
        A.states.pt[id] = x.pt;
        A.states.pr[id] = x.pr;
        A.states.pth[id] = x.pth;
        A.states.pph[id] = x.pph;
    }
}

// Camera of flat ray id (binary search over the prefix offsets).
__device__ __forceinline__ int find_camera(const CamDesc *__restrict__ cams, int n_cams, int64_t id)
{
    int lo = 0, hi = n_cams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].offset <= id)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Status after a step (listing's order: escape first, then step collapse).
__device__ __forceinline__ int exit_status(double r, double h, double r_esc, double sp, uint32_t n,
                                           int64_t n_steps)
{
    if (r > r_esc) return GT_RAY_ESCAPED;
    if (h < sp * 0.00003) return GT_RAY_HORIZON;
    if ((int64_t)n >= n_steps) return GT_RAY_MAXSTEPS;
    return -1;
}

// ------------------------------------------------------------------ FP32-mixed pieces
struct RayMixed {
    F2 t, r, th, ph, pr, pth;
    double pt, pph; // constants of motion kept in FP64
    float ptf, pphf;
};

__device__ __forceinline__ void mixed_from64(const Ray64 &x, RayMixed &m)
{
    m.t = f2_from(x.t);
    m.r = f2_from(x.r);
    m.th = f2_from(x.th);
    m.ph = f2_from(x.ph);
    m.pr = f2_from(x.pr);
    m.pth = f2_from(x.pth);
    m.pt = x.pt;
    m.pph = x.pph;
    m.ptf = (float)x.pt;
    m.pphf = (float)x.pph;
}

__device__ __forceinline__ void mixed_to64(const RayMixed &m, Ray64 &x)
{
    x.t = f2_to(m.t);
    x.r = f2_to(m.r);
    x.th = f2_to(m.th);
    x.ph = f2_to(m.ph);
    x.pr = f2_to(m.pr);
    x.pth = f2_to(m.pth);
    x.pt = m.pt;
    x.pph = m.pph;
}

// The FP32 field is evaluated 4 times per step; GT_FIELD_NOINLINE keeps one out-of-line
// copy instead of four inlined ones (smaller code, fewer instruction-cache misses).
#ifdef GT_FIELD_NOINLINE
#define GT_FIELD_ATTR __noinline__
#else
#define GT_FIELD_ATTR __forceinline__
#endif

template <int KIND, bool PRECISE>
__device__ GT_FIELD_ATTR void rates_f32(const SpacetimeF &st, float r, float s, float cs,
                                          float pr, float pth, float pt, float pph,
                                          Rates<float> &o)
{
    if (KIND == KIND_KERR || (KIND == 2 && st.kind == KIND_KERR))
        kerr_rates_sc<float>(st, r, s, cs, pr, pth, pt, pph, o);
    else
        mn_rates_sc<float, PRECISE>(st, r, s, cs, pr, pth, pt, pph, o);
}

// One FP32 RK4 step on the compensated state; returns h (as float).
template <int KIND, bool PRECISE = false>
__device__ __forceinline__ float rk4_step32(const SpacetimeF &st, RayMixed &m, float sp, float w6)
{
    Rates<float> k1, k2, k3, k4;
    const float r = m.r.hi, th = m.th.hi, pr = m.pr.hi, pth = m.pth.hi;
    // sin/cos of theta once per step; the later stages rotate them by their small offsets
    float s1, c1, s, c;
    sincosf(th, &s1, &c1);
    rates_f32<KIND, PRECISE>(st, r, s1, c1, pr, pth, m.ptf, m.pphf, k1);
    const float h = fabsf(sp / k1.dt);
    const float hh = 0.5f * h;
    rotate_sc(s1, c1, th, hh * k1.dth, &s, &c);
    rates_f32<KIND, PRECISE>(st, fmaf(hh, k1.dr, r), s, c, fmaf(hh, k1.dpr, pr),
                             fmaf(hh, k1.dpth, pth), m.ptf, m.pphf, k2);
    rotate_sc(s1, c1, th, hh * k2.dth, &s, &c);
    rates_f32<KIND, PRECISE>(st, fmaf(hh, k2.dr, r), s, c, fmaf(hh, k2.dpr, pr),
                             fmaf(hh, k2.dpth, pth), m.ptf, m.pphf, k3);
    rotate_sc(s1, c1, th, h * k3.dth, &s, &c);
    rates_f32<KIND, PRECISE>(st, fmaf(h, k3.dr, r), s, c, fmaf(h, k3.dpr, pr),
                             fmaf(h, k3.dpth, pth), m.ptf, m.pphf, k4);
    const float hw = h * w6;
    f2_add(m.t, hw * (k1.dt + 2.0f * k2.dt + 2.0f * k3.dt + k4.dt));
    f2_add(m.r, hw * (k1.dr + 2.0f * k2.dr + 2.0f * k3.dr + k4.dr));
    f2_add(m.th, hw * (k1.dth + 2.0f * k2.dth + 2.0f * k3.dth + k4.dth));
    f2_add(m.ph, hw * (k1.dph + 2.0f * k2.dph + 2.0f * k3.dph + k4.dph));
    f2_add(m.pr, hw * (k1.dpr + 2.0f * k2.dpr + 2.0f * k3.dpr + k4.dpr));
    f2_add(m.pth, hw * (k1.dpth + 2.0f * k2.dpth + 2.0f * k3.dpth + k4.dpth));
    return h;
}

// H = 0 re-projection in FP64 (mixed mode): solve g^rr p_r^2 = -(rest) for |p_r|,
// keeping the sign of p_r.  Skipped near radial turning points, where the radial
// term is small against the rest and the square root is ill-conditioned.
__device__ __forceinline__ void reproject_pr(const SpacetimeC &st, Ray64 &x)
{
    double g[5];
    upper_metric(st, x.r, x.th, g);
    const double rest = g[0] * x.pt * x.pt + 2.0 * g[1] * x.pt * x.pph + g[2] * x.pph * x.pph +
                        g[4] * x.pth * x.pth;
    const double rad = g[3] * x.pr * x.pr;
    const double scale = fabs(g[0] * x.pt * x.pt) + fabs(g[2] * x.pph * x.pph) + rad +
                         g[4] * x.pth * x.pth;
    if (!(rad > 0.05 * scale)) return;
    const double pr2 = -rest / g[3];
    if (!(pr2 > 0.0) || !isfinite(pr2)) return;
    x.pr = copysign(sqrt(pr2), x.pr);
}

// ------------------------------------------------------------------ the kernel
// MODE 0: FP64 plain.
// MODE 1: FP32-mixed with the FP64 zone inline (used where no park lists exist).
// MODE 2: FP32-mixed, FP32 steps only; a ray entering the FP64 zone (r < r_switch) is
//         parked on the output list; input list items continue in FP32.
// MODE 3: FP64 zone steps for parked rays; a ray leaving the zone (r > 1.25 r_switch)
//         is parked on the output list for the next FP32 launch.
// KIND: 0 Kerr, 1 Manko-Novikov, 2 per-camera, 3 per-camera with forward-difference
// derivatives (MODE 0 only).
// Work of a launch: fresh rays [0, n_fresh) then input-list items [0, *in_count).

__device__ __forceinline__ void park(const TraceArgs &A, int64_t id, uint32_t n, int cam,
                                     const Ray64 &x, bool *ok)
{
    const unsigned long long slot = atomicAdd(A.out_count, 1ull);
    if (slot >= A.out_cap) { // cannot happen with capacity = rays of the launch
        *ok = false;
        return;
    }
    ParkItem &it = A.out_items[slot];
    it.id = id;
    it.n = n;
    it.cam = cam;
    it.t = x.t;
    it.r = x.r;
    it.th = x.th;
    it.ph = x.ph;
    it.pr = x.pr;
    it.pth = x.pth;
    it.pt = x.pt;
    it.pph = x.pph;
    *ok = true;
}

template <int MODE, int KIND, bool PRECISE>
__device__ __forceinline__ void trace_body(const TraceArgs &A, int one_shot)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long *next = A.scratch + SCR_NEXT_RAY;
    volatile unsigned long long *tflag = A.scratch + SCR_TIMEOUT;
    const uint64_t t_start = A.timeout_ns ? globaltimer_ns() : 0;
    const CamDesc *__restrict__ cams = A.cams;
    const int64_t n_in =
        A.in_count ? (int64_t)(*A.in_count < A.in_cap ? *A.in_count : A.in_cap) : 0;
    const int64_t n_work = A.n_fresh + n_in;

    int64_t id = -1;
    int cam = 0;
    bool active = false;
    bool drained = false;
    uint32_t n = 0;
    uint32_t n_entry = 0;           // step count when the ray entered this launch (zone steps)
    uint32_t n_f64 = 0;             // zone field evaluations of the ray in FP64 (this launch)
    SpacetimeT<DF> sd_ray;          // double-float constants of a per-ray spacetime
    uint32_t rp_next = 0xFFFFFFFFu; // next step count that is a multiple of reproject_every
    Ray64 x;
    RayMixed m;
    SpacetimeC st = cams[0].st;
    SpacetimeF stf = to_float(st);
    double r_esc = cams[0].r_escape;
    double r_sw = cams[0].r_switch;
    const float spf = A.sp_f, w6f = A.w6_f;
    const float h_thr_f = A.h_thr_f;
    F2 r_esc_f = f2_from(r_esc);
    float r_sw_f = (float)r_sw;

    auto load_camera = [&](int c) {
        cam = c;
        // the FP32-only kernel keeps just the float constants live; the FP64 ones are
        // reloaded for the occasional re-projection
        if (MODE != 2) st = cams[c].st;
        r_esc = cams[c].r_escape;
        r_sw = cams[c].r_switch;
        if (MODE == 1 || MODE == 2) stf = to_float(cams[c].st);
        if (MODE == 2) {
            r_esc_f = f2_from(r_esc);
            r_sw_f = (float)r_sw;
        }
    };
    auto load_rayparams = [&](int64_t rid, bool init) {
        CamDesc d;
        d.M = A.rays->M;
        d.S = A.rays->spin[rid] * A.rays->M * A.rays->M; // spin = a/M
        d.Q = A.rays->q[rid];
        d.r0 = A.rays->r0;
        d.th0 = A.rays->theta0[rid];
        d.fov_deg = 90.0;
        d.res_x = d.res_y = 1;
        d.offset = 0;
        setup_desc(d, A.flags, A.rays->r_switch);
        if (MODE != 2) st = d.st;
        if (MODE == 1 || MODE == 3) sd_ray = d.st_df;
        r_esc = d.r_escape;
        r_sw = d.r_switch;
        if (MODE == 1 || MODE == 2) stf = to_float(d.st);
        if (MODE == 2) {
            r_esc_f = f2_from(r_esc);
            r_sw_f = (float)r_sw;
        }
        if (init) camera_init_dir(d, A.rays->alpha[rid], A.rays->beta[rid], x);
        return d.valid != 0;
    };

    // Start work item `w`; returns false when the ray is already finished and stored.
    auto start = [&](int64_t w) -> bool {
        if (w < A.n_fresh) { // a fresh ray: initial data from the camera
            const int64_t pix = A.fresh_ids ? A.fresh_ids[w] : w;
            id = (A.fresh_ids && A.compact_out) ? w : pix;
            if (A.rays) {
                const bool valid = load_rayparams(pix, true);
                n = 0;
                if (!valid || A.n_steps <= 0) {
                    store_ray(A, id, x.t, x.r, x.th, x.ph, valid ? GT_RAY_MAXSTEPS : GT_RAY_NONFINITE, 0);
                    return false;
                }
            } else if (A.states.t) { // an arbitrary initial state (gt_trace_states)
                x.t = A.states.t[pix];
                x.r = A.states.r[pix];
                x.th = A.states.th[pix];
                x.ph = A.states.ph[pix];
                x.pt = A.states.pt[pix];
                x.pr = A.states.pr[pix];
                x.pth = A.states.pth[pix];
                x.pph = A.states.pph[pix];
                n = 0;
                if (A.n_steps <= 0) {
                    store_full(A, id, x, GT_RAY_MAXSTEPS, 0, nan(""));
                    return false;
                }
            } else {
                if (KIND >= KIND_ANY || A.n_cams > 1) load_camera(find_camera(cams, A.n_cams, pix));
                camera_init(cams[cam], A.first + pix - cams[cam].offset, x);
                if (A.f32_io) { // the listing's kernels take the initial state as float32
                    x.t = round_f32(x.t);
                    x.r = round_f32(x.r);
                    x.th = round_f32(x.th);
                    x.ph = round_f32(x.ph);
                    x.pt = round_f32(x.pt);
                    x.pr = round_f32(x.pr);
                    x.pth = round_f32(x.pth);
                    x.pph = round_f32(x.pph);
                }
                n = 0;
                if (A.n_steps <= 0) {
                    store_full(A, id, x, GT_RAY_MAXSTEPS, 0, nan(""));
                    return false;
                }
            }
        } else { // a parked ray from the input list
            const ParkItem &it = A.in_items[w - A.n_fresh];
            id = it.id;
            n = it.n;
            if (A.rays)
                load_rayparams(id, false);
            else if (KIND >= KIND_ANY || A.n_cams > 1)
                load_camera(it.cam);
            x.t = it.t;
            x.r = it.r;
            x.th = it.th;
            x.ph = it.ph;
            x.pr = it.pr;
            x.pth = it.pth;
            x.pt = it.pt;
            x.pph = it.pph;
        }
        n_entry = n;
        n_f64 = 0;
        if (MODE == 1 || MODE == 2) {
            mixed_from64(x, m);
            if (A.reproject_every > 0) {
                const uint64_t k = (uint64_t)A.reproject_every;
                const uint64_t nx = ((uint64_t)n / k + 1u) * k;
                rp_next = nx < 0xFFFFFFFFull ? (uint32_t)nx : 0xFFFFFFFFu;
            }
        }
        return true;
    };

    if (one_shot) {
        drained = true;
        const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (w < n_work) active = start(w);
    }

    for (uint32_t it = 0;; ++it) {
        // ---- refill finished lanes from the global queue
        if (!drained) {
            const unsigned need = __ballot_sync(FULL_MASK, !active);
            if (need) {
                const int cnt = __popc(need);
                const int leader = __ffs(need) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(next, (unsigned long long)cnt);
                base = __shfl_sync(FULL_MASK, base, leader);
                if (base + (unsigned long long)cnt >= (unsigned long long)n_work) drained = true;
                if (!active) {
                    const int64_t w = (int64_t)base + __popc(need & lt_mask);
                    if (w < n_work) active = start(w);
                }
            }
        }
        if (!__any_sync(FULL_MASK, active)) {
            if (drained) break;
            continue;
        }
        // ---- watchdog: stop every lane with status TIMEOUT
        if (A.timeout_ns && (it & 127u) == 0u) {
            int stop = 0;
            if (lane == 0) {
                if (*tflag) {
                    stop = 1;
                } else if (globaltimer_ns() - t_start > A.timeout_ns) {
                    atomicExch(A.scratch + SCR_TIMEOUT, 1ull);
                    stop = 1;
                }
            }
            stop = __shfl_sync(FULL_MASK, stop, 0);
            if (stop) {
                if (active) {
                    if (MODE == 1 || MODE == 2) mixed_to64(m, x);
                    store_full(A, id, x, GT_RAY_TIMEOUT, n, nan(""));
                }
                if (!one_shot) {
                    for (;;) { // drain the queue without integrating
                        unsigned long long base = 0;
                        if (lane == 0) base = atomicAdd(next, 32ull);
                        base = __shfl_sync(FULL_MASK, base, 0);
                        if (base >= (unsigned long long)n_work) break;
                        const int64_t w = (int64_t)base + lane;
                        if (w < n_work) {
                            if (w < A.n_fresh && A.states.t) {
                                if (A.status) A.status[w] = GT_RAY_TIMEOUT; // state untouched
                                if (A.nsteps) A.nsteps[w] = 0;
                            } else if (w < A.n_fresh) {
                                const int64_t pix = A.fresh_ids ? A.fresh_ids[w] : w;
                                const int c = A.n_cams > 1 ? find_camera(cams, A.n_cams, pix) : 0;
                                const double r0 = A.rays ? A.rays->r0 : cams[c].r0;
                                const double th0 = A.rays ? A.rays->theta0[pix] : cams[c].th0;
                                store_ray(A, (A.fresh_ids && A.compact_out) ? w : pix, 0.0, r0,
                                          th0, 0.0, GT_RAY_TIMEOUT, 0);
                            } else {
                                const ParkItem &p = A.in_items[w - A.n_fresh];
                                Ray64 y;
                                y.t = p.t;
                                y.r = p.r;
                                y.th = p.th;
                                y.ph = p.ph;
                                y.pt = p.pt;
                                y.pr = p.pr;
                                y.pth = p.pth;
                                y.pph = p.pph;
                                store_full(A, p.id, y, GT_RAY_TIMEOUT, p.n, nan(""));
                            }
                        }
                    }
                }
                return;
            }
        }
        if (!active) continue;

        // ---- one RK4 step
        int status = -1;
        if (MODE == 0 || MODE == 3) {
            Ray64 y;
            double h;
            if (MODE == 3 && A.zone_df) {
                h = rk4_step_zone<KIND>(st, A.rays ? &sd_ray : &cams[cam].st_df, x, A.sp_df,
                                        A.w6_df, y, n_f64);
            } else {
                h = step64<KIND>(A, st, x, y);
                if (MODE == 3) n_f64 += 4;
            }
            ++n;
            if (!isfinite(h) || !finite6(y)) {
                status = GT_RAY_NONFINITE;
            } else {
                x = y;
                status = exit_status(x.r, h, r_esc, A.sp, n, A.n_steps);
                // the ring is tested after the escape and before the horizon
                if (A.disk.on && status != GT_RAY_ESCAPED && in_disk(A.disk, x.r, x.th))
                    status = GT_RAY_DISK;
                if (MODE == 3 && status < 0 && x.r > 1.25 * r_sw) { // leave the FP64 zone
                    bool ok;
                    park(A, id, n, cam, x, &ok);
                    if (ok) {
                        active = false;
                        atomicAdd(A.scratch + SCR_ZONE_STEPS, (unsigned long long)(n - n_entry));
                        if (n_f64) atomicAdd(A.scratch + SCR_ZONE_F64, (unsigned long long)n_f64);
                    }
                }
            }
        } else if (MODE == 1) {
            double h;
            bool ok = true;
            if ((double)m.r.hi < r_sw) { // the zone inline
                Ray64 y;
                mixed_to64(m, x);
                if (A.zone_df) {
                    h = rk4_step_zone<KIND>(st, A.rays ? &sd_ray : &cams[cam].st_df, x,
                                            A.sp_df, A.w6_df, y, n_f64);
                } else {
                    h = step64<KIND>(A, st, x, y);
                    n_f64 += 4;
                }
                ok = isfinite(h) && finite6(y);
                if (ok) mixed_from64(y, m);
            } else {
                RayMixed keep = m;
                h = (double)rk4_step32<KIND>(stf, m, spf, w6f);
                ok = isfinite(h) && isfinite(m.t.hi) && isfinite(m.r.hi) && isfinite(m.th.hi) &&
                     isfinite(m.ph.hi) && isfinite(m.pr.hi) && isfinite(m.pth.hi);
                if (!ok) m = keep;
            }
            ++n;
            if (!ok) {
                status = GT_RAY_NONFINITE;
                mixed_to64(m, x);
            } else {
                const double r_now = f2_to(m.r);
                status = exit_status(r_now, h, r_esc, A.sp, n, A.n_steps);
                if (A.disk.on && status != GT_RAY_ESCAPED && in_disk(A.disk, r_now, f2_to(m.th)))
                    status = GT_RAY_DISK;
                if (status >= 0) {
                    mixed_to64(m, x);
                } else if (n == rp_next) {
                    rp_next = rp_next + (uint32_t)A.reproject_every < rp_next
                                  ? 0xFFFFFFFFu
                                  : rp_next + (uint32_t)A.reproject_every;
                    mixed_to64(m, x);
                    reproject_pr(st, x);
                    m.pr = f2_from(x.pr);
                }
            }
        } else { // MODE 2: FP32 steps only, exit tests in FP32
            RayMixed keep = m;
            const float h = rk4_step32<KIND, PRECISE>(stf, m, spf, w6f);
            ++n;
            const bool ok = isfinite(h) && isfinite(m.t.hi) && isfinite(m.r.hi) &&
                            isfinite(m.th.hi) && isfinite(m.ph.hi) && isfinite(m.pr.hi) &&
                            isfinite(m.pth.hi);
            if (!ok) {
                m = keep;
                status = GT_RAY_NONFINITE;
            } else if (m.r.hi > r_esc_f.hi || (m.r.hi == r_esc_f.hi && m.r.lo > r_esc_f.lo)) {
                status = GT_RAY_ESCAPED;
            } else if (A.disk.on && in_disk(A.disk, f2_to(m.r), f2_to(m.th))) {
                status = GT_RAY_DISK;
            } else if (h < h_thr_f) {
                status = GT_RAY_HORIZON;
            } else if ((int64_t)n >= A.n_steps) {
                status = GT_RAY_MAXSTEPS;
            } else if (m.r.hi < r_sw_f) { // enter the FP64 zone: hand the ray over
                mixed_to64(m, x);
                bool parked;
                park(A, id, n, cam, x, &parked);
                if (parked) active = false;
            } else if (n == rp_next) {
                rp_next = rp_next + (uint32_t)A.reproject_every < rp_next
                              ? 0xFFFFFFFFu
                              : rp_next + (uint32_t)A.reproject_every;
                mixed_to64(m, x);
                SpacetimeC st64;
                if (A.rays) {
                    CamDesc d;
                    d.M = A.rays->M;
                    d.S = A.rays->spin[id] * A.rays->M * A.rays->M;
                    d.Q = A.rays->q[id];
                    d.r0 = A.rays->r0;
                    d.th0 = A.rays->theta0[id];
                    d.fov_deg = 90.0;
                    d.res_x = d.res_y = 1;
                    d.offset = 0;
                    setup_desc(d, A.flags, A.rays->r_switch);
                    st64 = d.st;
                } else {
                    st64 = cams[cam].st;
                }
                reproject_pr(st64, x);
                m.pr = f2_from(x.pr);
            }
            if (status >= 0) mixed_to64(m, x);
        }
        if (status >= 0) {
            if (MODE == 3) {
                atomicAdd(A.scratch + SCR_ZONE_STEPS, (unsigned long long)(n - n_entry));
                if (n_f64) atomicAdd(A.scratch + SCR_ZONE_F64, (unsigned long long)n_f64);
            }
            double z = nan("");
            if (status == GT_RAY_DISK && A.z) z = redshift64<KIND>(cams[cam].st, cams[cam].gl_tt, x);
            store_full(A, id, x, status, n, z);
            active = false;
        }
    }
}

// The FP32 rounds kernel (MODE 2) is held to 128 registers: four resident blocks of 128
// threads per SM, also with PRECISE (GT_FLAG_PRECISE_MN), which needs a few more.
template <int MODE, int KIND, bool PRECISE = false>
__global__ void __launch_bounds__(256, MODE == 2 ? 2 : 1) trace_kernel(TraceArgs A, int one_shot)
{
    trace_body<MODE, KIND, PRECISE>(A, one_shot);
}

// ------------------------------------------------------------------ two rays per thread
// The FP32 rounds kernel (MODE 2) with two independent ray slots per thread: both slots'
// RK4 steps are issued back to back in one basic block, so the scheduler can interleave
// two dependency chains (instruction-level parallelism at half the resident threads).
// Same arithmetic per ray as trace_kernel<2, KIND>, so results are bitwise equal; for one
// camera of a fixed spacetime kind, without the watchdog, per-ray parameters, state
// arrays or the ring (the launcher falls back to one ray per thread otherwise).
struct Slot32 {
    bool active;
    int64_t id;
    uint32_t n, rp_next;
    RayMixed m;
};

template <int KIND, bool PRECISE>
__global__ void __launch_bounds__(256, 1) trace2_kernel(TraceArgs A)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long *next = A.scratch + SCR_NEXT_RAY;
    const CamDesc &cam = A.cams[0];
    const SpacetimeF stf = to_float(cam.st);
    const F2 r_esc_f = f2_from(cam.r_escape);
    const float r_sw_f = (float)cam.r_switch;
    const float spf = A.sp_f, w6f = A.w6_f, h_thr_f = A.h_thr_f;
    const int64_t n_in = A.in_count ? (int64_t)(*A.in_count < A.in_cap ? *A.in_count : A.in_cap) : 0;
    const int64_t n_work = A.n_fresh + n_in;
    Slot32 sl[2];
    sl[0].active = sl[1].active = false;
    bool drained = false;
    Ray64 x;

    auto start = [&](Slot32 &q, int64_t w) {
        if (w < A.n_fresh) {
            const int64_t pix = A.fresh_ids ? A.fresh_ids[w] : w;
            q.id = (A.fresh_ids && A.compact_out) ? w : pix;
            camera_init(cam, A.first + pix, x);
            q.n = 0;
            if (A.n_steps <= 0) {
                store_full(A, q.id, x, GT_RAY_MAXSTEPS, 0, nan(""));
                return false;
            }
        } else {
            const ParkItem &it = A.in_items[w - A.n_fresh];
            q.id = it.id;
            q.n = it.n;
            x.t = it.t;
            x.r = it.r;
            x.th = it.th;
            x.ph = it.ph;
            x.pr = it.pr;
            x.pth = it.pth;
            x.pt = it.pt;
            x.pph = it.pph;
        }
        mixed_from64(x, q.m);
        q.rp_next = 0xFFFFFFFFu;
        if (A.reproject_every > 0) {
            const uint64_t k = (uint64_t)A.reproject_every;
            const uint64_t nx = ((uint64_t)q.n / k + 1u) * k;
            q.rp_next = nx < 0xFFFFFFFFull ? (uint32_t)nx : 0xFFFFFFFFu;
        }
        return true;
    };

    // exit tests, zone hand-over and re-projection of one slot after its step
    auto finish = [&](Slot32 &q, float h, const RayMixed &keep) {
        ++q.n;
        int status = -1;
        const bool ok = isfinite(h) && isfinite(q.m.t.hi) && isfinite(q.m.r.hi) &&
                        isfinite(q.m.th.hi) && isfinite(q.m.ph.hi) && isfinite(q.m.pr.hi) &&
                        isfinite(q.m.pth.hi);
        if (!ok) {
            q.m = keep;
            status = GT_RAY_NONFINITE;
        } else if (q.m.r.hi > r_esc_f.hi || (q.m.r.hi == r_esc_f.hi && q.m.r.lo > r_esc_f.lo)) {
            status = GT_RAY_ESCAPED;
        } else if (h < h_thr_f) {
            status = GT_RAY_HORIZON;
        } else if ((int64_t)q.n >= A.n_steps) {
            status = GT_RAY_MAXSTEPS;
        } else if (q.m.r.hi < r_sw_f) { // enter the FP64 zone: hand the ray over
            mixed_to64(q.m, x);
            bool parked;
            park(A, q.id, q.n, 0, x, &parked);
            if (parked) q.active = false;
        } else if (q.n == q.rp_next) {
            q.rp_next = q.rp_next + (uint32_t)A.reproject_every < q.rp_next
                            ? 0xFFFFFFFFu
                            : q.rp_next + (uint32_t)A.reproject_every;
            mixed_to64(q.m, x);
            reproject_pr(cam.st, x);
            q.m.pr = f2_from(x.pr);
        }
        if (status >= 0) {
            mixed_to64(q.m, x);
            store_full(A, q.id, x, status, q.n, nan(""));
            q.active = false;
        }
    };

    for (;;) {
#pragma unroll
        for (int k = 0; k < 2; k++) { // refill each slot from the global queue
            if (drained) break;
            const unsigned need = __ballot_sync(FULL_MASK, !sl[k].active);
            if (need) {
                const int cnt = __popc(need);
                const int leader = __ffs(need) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(next, (unsigned long long)cnt);
                base = __shfl_sync(FULL_MASK, base, leader);
                if (base + (unsigned long long)cnt >= (unsigned long long)n_work) drained = true;
                if (!sl[k].active) {
                    const int64_t w = (int64_t)base + __popc(need & lt_mask);
                    if (w < n_work) sl[k].active = start(sl[k], w);
                }
            }
        }
        if (!__any_sync(FULL_MASK, sl[0].active || sl[1].active)) {
            if (drained) break;
            continue;
        }
        // both steps back to back (a lane's idle slot steps its last state and drops the
        // result); a slot idle in the whole warp -- the queue's tail, or more slots than
        // rays -- is skipped, a warp-uniform branch
        const bool any0 = __any_sync(FULL_MASK, sl[0].active);
        const bool any1 = __any_sync(FULL_MASK, sl[1].active);
        if (any0 && any1) {
            const RayMixed keep0 = sl[0].m, keep1 = sl[1].m;
            const float h0 = rk4_step32<KIND, PRECISE>(stf, sl[0].m, spf, w6f);
            const float h1 = rk4_step32<KIND, PRECISE>(stf, sl[1].m, spf, w6f);
            if (sl[0].active) finish(sl[0], h0, keep0);
            if (sl[1].active) finish(sl[1], h1, keep1);
        } else if (any0) { // static slot indices keep the slots in registers
            const RayMixed keep = sl[0].m;
            const float h = rk4_step32<KIND, PRECISE>(stf, sl[0].m, spf, w6f);
            if (sl[0].active) finish(sl[0], h, keep);
        } else {
            const RayMixed keep = sl[1].m;
            const float h = rk4_step32<KIND, PRECISE>(stf, sl[1].m, spf, w6f);
            if (sl[1].active) finish(sl[1], h, keep);
        }
    }
}

template <int KIND>
static cudaError_t launch_two(const TraceArgs &a, int block, int grid, cudaStream_t s)
{
    if constexpr (KIND == KIND_MN) {
        if (a.flags & GT_FLAG_PRECISE_MN) {
            trace2_kernel<KIND, true><<<grid, block, 0, s>>>(a);
            return cudaGetLastError();
        }
    }
    trace2_kernel<KIND, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

bool two_rays_supported(const TraceArgs &a, int kmode, int kind_hint)
{
    return kmode == KMODE_MIXED_FP32 && (kind_hint == KIND_KERR || kind_hint == KIND_MN) &&
           a.n_cams == 1 && !a.rays && !a.states.t && !a.disk.on && a.timeout_ns == 0;
}

cudaError_t launch_trace_two(const TraceArgs &args, int kind_hint, int block, int grid,
                             cudaStream_t s)
{
    TraceArgs a = args;
    a.sp_f = (float)a.sp;
    a.w6_f = (float)a.w6;
    a.h_thr_f = (float)(a.sp * 0.00003);
    a.sp_df = DF(a.sp);
    a.w6_df = DF(a.w6);
    return kind_hint == KIND_KERR ? launch_two<KIND_KERR>(a, block, grid, s)
                                  : launch_two<KIND_MN>(a, block, grid, s);
}

int max_blocks_per_sm_two(int kind_hint, int block)
{
    int n = 0;
    const cudaError_t e = kind_hint == KIND_KERR
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace2_kernel<KIND_KERR, false>, block, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace2_kernel<KIND_MN, false>, block, 0);
    return (e == cudaSuccess && n > 0) ? n : 1;
}

// Loop condition of the graph-resident FP32-mixed rounds: continue while rays are parked.
__global__ void set_loop_condition_kernel(cudaGraphConditionalHandle h,
                                          const unsigned long long *count)
{
    cudaGraphSetConditional(h, *count != 0ull ? 1u : 0u);
}

cudaError_t launch_set_condition(cudaGraphConditionalHandle h, const unsigned long long *count,
                                 cudaStream_t s)
{
    set_loop_condition_kernel<<<1, 1, 0, s>>>(h, count);
    return cudaGetLastError();
}

template <int MODE, int KIND>
static cudaError_t launch_one(const TraceArgs &a, int block, int grid, bool one_shot, cudaStream_t s)
{
    if constexpr (MODE == 2 && KIND != KIND_KERR) {
        if (a.flags & GT_FLAG_PRECISE_MN) {
            trace_kernel<MODE, KIND, true><<<grid, block, 0, s>>>(a, one_shot ? 1 : 0);
            return cudaGetLastError();
        }
    }
    trace_kernel<MODE, KIND><<<grid, block, 0, s>>>(a, one_shot ? 1 : 0);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_mode(const TraceArgs &a, int kind_hint, int block, int grid,
                               bool one_shot, cudaStream_t s)
{
    if (kind_hint == KIND_KERR) return launch_one<MODE, KIND_KERR>(a, block, grid, one_shot, s);
    if (kind_hint == KIND_MN) return launch_one<MODE, KIND_MN>(a, block, grid, one_shot, s);
    if (kind_hint == KIND_FD) {
        if constexpr (MODE == 0) return launch_one<0, KIND_FD>(a, block, grid, one_shot, s);
        return cudaErrorInvalidValue; // the listing's numerics run in FP64 only
    }
    return launch_one<MODE, KIND_ANY>(a, block, grid, one_shot, s);
}

cudaError_t launch_trace(const TraceArgs &args, int kmode, int kind_hint, int block, int grid,
                         bool one_shot, cudaStream_t s)
{
    TraceArgs a = args;
    a.sp_f = (float)a.sp;
    a.w6_f = (float)a.w6;
    a.h_thr_f = (float)(a.sp * 0.00003);
    a.sp_df = DF(a.sp);
    a.w6_df = DF(a.w6);
    switch (kmode) {
    case KMODE_FP64: return launch_mode<0>(a, kind_hint, block, grid, one_shot, s);
    case KMODE_MIXED_INLINE: return launch_mode<1>(a, kind_hint, block, grid, one_shot, s);
    case KMODE_MIXED_FP32: return launch_mode<2>(a, kind_hint, block, grid, one_shot, s);
    case KMODE_ZONE_FP64: return launch_mode<3>(a, kind_hint, block, grid, one_shot, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODE, int KIND>
static int occupancy_one(int block)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, trace_kernel<MODE, KIND>, block, 0) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <int MODE>
static int occupancy_mode(int kind_hint, int block)
{
    if (kind_hint == KIND_KERR) return occupancy_one<MODE, KIND_KERR>(block);
    if (kind_hint == KIND_MN) return occupancy_one<MODE, KIND_MN>(block);
    if (kind_hint == KIND_FD) {
        if constexpr (MODE == 0) return occupancy_one<0, KIND_FD>(block);
        return 1;
    }
    return occupancy_one<MODE, KIND_ANY>(block);
}

int max_blocks_per_sm(int kmode, int kind_hint, int block)
{
    switch (kmode) {
    case KMODE_FP64: return occupancy_mode<0>(kind_hint, block);
    case KMODE_MIXED_INLINE: return occupancy_mode<1>(kind_hint, block);
    case KMODE_MIXED_FP32: return occupancy_mode<2>(kind_hint, block);
    case KMODE_ZONE_FP64: return occupancy_mode<3>(kind_hint, block);
    default: return 1;
    }
}

} // namespace gt
