// camera.cuh -- per-ray state and the fused camera initialisation (device, inline).
#pragma once

#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace gt {

struct Ray64 {
    double t, r, th, ph, pr, pth; // evolving
    double pt, pph;               // constants of motion
};

// Initial data of pixel `local` of camera `c` (Sec. 3.3.1, listing's camera block):
// v = (T, -1, beta_j, alpha_i / sin theta0), T the root (-B + sqrt(B^2 - 4AC))/(2A)
// of g(v, v) = 0, v /= |T|, p = g v at (0, r0, theta0, 0).
__device__ __forceinline__ void camera_init_dir(const CamDesc &c, double al, double bt, Ray64 &x)
{
    double vr = -1.0, vth = bt, vph = al * c.inv_sin_th0;
    const double A = c.gl_tt;
    const double B = 2.0 * c.gl_tph * vph;
    const double C = c.gl_rr * vr * vr + c.gl_thth * vth * vth + c.gl_phph * vph * vph;
    const double T = (-B + sqrt(B * B - 4.0 * A * C)) / (2.0 * A);
    const double sc = 1.0 / fabs(T);
    const double vt = T * sc;
    vr *= sc;
    vth *= sc;
    vph *= sc;
    x.t = 0.0;
    x.r = c.r0;
    x.th = c.th0;
    x.ph = 0.0;
    x.pt = c.gl_tt * vt + c.gl_tph * vph;
    x.pr = c.gl_rr * vr;
    x.pth = c.gl_thth * vth;
    x.pph = c.gl_tph * vt + c.gl_phph * vph;
}

__device__ __forceinline__ void camera_init(const CamDesc &c, int64_t local, Ray64 &x)
{
    const int i = (int)(local % c.res_x);
    const int j = (int)(local / c.res_x);
    const double al = c.res_x > 1 ? c.H * (double)(2 * i - (c.res_x - 1)) / (double)(c.res_x - 1) : 0.0;
    const double bt = c.res_y > 1 ? c.V * (double)(2 * j - (c.res_y - 1)) / (double)(c.res_y - 1) : 0.0;
    camera_init_dir(c, al, bt, x);
}


} // namespace gt
