// compensated.cuh -- the (hi, lo) float pair of the FP32-mixed ray state and the
// rotation of sin/cos across the RK4 stages (host and device, so host tests can check
// their error bounds).
#pragma once

#include <math.h>

#ifndef GT_HD
#define GT_HD __host__ __device__ __forceinline__
#endif

namespace gt {

// x = hi + lo with |lo| <= ulp(hi)/2 after every update.
struct F2 {
    float hi, lo;
};

GT_HD F2 f2_from(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

GT_HD double f2_to(F2 a) { return (double)a.hi + (double)a.lo; }

// a += d.  The increment is first added to the low part, t = fl(lo + d), and the pair is
// renormalised with Fast2Sum (Dekker 1971): s = fl(hi + t), e = fl(t - fl(s - hi)), which
// is error-free when the exponent of hi is at least that of t -- the normal case, since
// an RK4 increment is small against the coordinate it moves.  Four operations instead of
// the six of TwoSum plus a renormalisation.  The rounding of t adds at most ulp(t)/2, the
// order of the rounding error the FP32 increment d already carries; where hi is the
// smaller term (a momentum crossing zero) Fast2Sum may drop up to ulp(t)/2 more.  Either
// way the error per update stays within u |d| + u^2 |hi| (u = 2^-24), which the host
// test of this function checks against exact sums, sign changes and zero crossings
// included.
GT_HD void f2_add(F2 &a, float d)
{
    const float t = a.lo + d;
    const float s = a.hi + t;
    a.lo = t - (s - a.hi);
    a.hi = s;
}

// sin and cos of theta + d from those of theta, for the small angle d an RK4 stage adds.
// FP32: Taylor series of sin d through d^7 and cos d through d^6 (truncation below 4e-10
// for |d| <= 1/4); FP64: through d^9 and d^8 (truncation below 3e-19 for |d| <= 1/16).
// Larger d -- not met in practice -- evaluates sin/cos afresh.
#ifdef __CUDACC__
__device__ __forceinline__ void rotate_sc(float s, float c, float th, float d, float *s2, float *c2)
{
    if (fabsf(d) <= 0.25f) {
        const float d2 = d * d;
        const float sd = fmaf(d * d2, fmaf(d2, fmaf(d2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), d);
        const float cd = fmaf(d2, fmaf(d2, fmaf(d2, -1.0f / 720.0f, 1.0f / 24.0f), -0.5f), 1.0f);
        *s2 = fmaf(s, cd, c * sd);
        *c2 = fmaf(c, cd, -(s * sd));
    } else {
        sincosf(th + d, s2, c2);
    }
}

__device__ __forceinline__ void rotate_sc(double s, double c, double th, double d, double *s2,
                                          double *c2)
{
    if (fabs(d) <= 0.0625) {
        const double d2 = d * d;
        // sin d - d = d^3 (-1/3! + d^2/5! - d^4/7! + d^6/9!)
        double ps = fma(d2, 1.0 / 362880.0, -1.0 / 5040.0);
        ps = fma(d2, ps, 1.0 / 120.0);
        ps = fma(d2, ps, -1.0 / 6.0);
        const double sd = fma(d * d2, ps, d);
        // cos d - 1 = d^2 (-1/2! + d^2/4! - d^4/6! + d^6/8!)
        double pc = fma(d2, 1.0 / 40320.0, -1.0 / 720.0);
        pc = fma(d2, pc, 1.0 / 24.0);
        pc = fma(d2, pc, -0.5);
        const double cdm1 = d2 * pc;
        // rotate: sin(th + d) = s + (s (cos d - 1) + c sin d), likewise cos
        *s2 = s + fma(s, cdm1, c * sd);
        *c2 = c + fma(c, cdm1, -(s * sd));
    } else {
        sincos(th + d, s2, c2);
    }
}
#endif

} // namespace gt
