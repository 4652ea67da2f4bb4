// zone_df.cuh -- the Manko-Novikov rates of the FP32-mixed path's zone in double-float
// (df.cuh): the FP64 state goes in, FP64 rates come out, and the evaluation between runs
// on the FP32 pipes.  Where the evaluation would leave the range in which double-float
// keeps its precision, mn_rates_df returns false and the caller evaluates in FP64.
#pragma once

#include "df.cuh"

#ifndef GT_HD
#define GT_HD __host__ __device__ __forceinline__
#endif

namespace gt {

// Largest |exponent| of the evaluation taken in double-float: |2 beta Ea|, |2 beta Eb|
// <= 24 and |2 psi|, |2 psi - 2 gamma''| <= 48.  Inside these bounds a product of the
// metric functions can still overflow the float range; an infinite high part turns the
// low part into NaN in the error-free transformations (inf - inf), the rates come out
// non-finite and the caller takes FP64.  What the bounds guard against is the silent
// case, low parts falling below the normal floats.  The host test of this header finds
// the accepted double-float rates within ~30x the FP64 rounding error over the zone of
// eight spacetimes; binned by the largest exponent, the points between 1x and 1.5x of
// the bounds first used (16, 32) keep p99 9e-12 and max 4e-10 of the largest rate
// (FP64: 3e-13, 3e-11), while beyond 1.5x some overflow.  The trapped rays of the
// listing's spacetime (near r = 1.83M) stay within |2 beta Ea| < 8,
// |2 psi - 2 gamma''| < 19; deeper orbits (r < 1.8M) reach the bounds.
constexpr float ZONE_DF_MAX_EF = 24.0f;
constexpr float ZONE_DF_MAX_EPSI = 48.0f;

GT_HD SpacetimeT<DF> to_df(const SpacetimeC &c)
{
    SpacetimeT<DF> d;
    d.kind = c.kind;
    d.M = DF(c.M);
    d.a = DF(c.a);
    d.a2 = DF(c.a2);
    d.r_plus = DF(c.r_plus);
    d.k = DF(c.k);
    d.ik = DF(c.ik);
    d.alpha = DF(c.alpha);
    d.beta = DF(c.beta);
    d.two_beta = DF(c.two_beta);
    d.three_beta2 = DF(c.three_beta2);
    d.c_g = DF(c.c_g);
    d.w_inf = DF(c.w_inf);
    d.k2 = DF(c.k2);
    d.inv_k2 = DF(c.inv_k2);
    d.two_k = DF(c.two_k);
    return d;
}

// Rates of Manko-Novikov at a phase-space point given in double-float (theta through
// s = sin, cs = cos) by the reverse sweep in double-float; false (o unspecified) where an
// exponent is out of range or a rate is not finite.
GT_HD bool mn_rates_df(const SpacetimeT<DF> &c, DF r, DF s, DF cs, DF pr, DF pth, DF pt,
                       DF pph, Rates<DF> &o)
{
    DF ex[4];
    mn_rates_sc<DF>(c, r, s, cs, pr, pth, pt, pph, o, ex);
    if (!(fabsf(ex[0].hi) <= ZONE_DF_MAX_EF && fabsf(ex[1].hi) <= ZONE_DF_MAX_EF &&
          fabsf(ex[2].hi) <= ZONE_DF_MAX_EPSI && fabsf(ex[3].hi) <= ZONE_DF_MAX_EPSI))
        return false;
    return isfinite(o.dt.hi) && isfinite(o.dr.hi) && isfinite(o.dth.hi) &&
           isfinite(o.dph.hi) && isfinite(o.dpr.hi) && isfinite(o.dpth.hi);
}

// The same, returned in FP64.
GT_HD bool mn_rates_df(const SpacetimeT<DF> &c, DF r, DF s, DF cs, DF pr, DF pth, DF pt,
                       DF pph, Rates<double> &o)
{
    Rates<DF> od;
    if (!mn_rates_df(c, r, s, cs, pr, pth, pt, pph, od)) return false;
    o.dt = df_to(od.dt);
    o.dr = df_to(od.dr);
    o.dth = df_to(od.dth);
    o.dph = df_to(od.dph);
    o.dpr = df_to(od.dpr);
    o.dpth = df_to(od.dpth);
    return true;
}

// sin and cos of theta + d from s = sin theta, c = cos theta for the small angle d of an
// RK4 stage, in double-float: sin d = d + d^3 q(d^2), cos d - 1 = d^2 p(d^2) with the
// Taylor polynomials q = -1/6 + d^2/120 - d^4/5040 + d^6/362880 and
// p = -1/2 + d^2/24 - d^4/720 + d^6/40320.  For |d| <= 1/16 (truncation below 2^-60) the
// terms of q after -1/6 and of p after d^2/24 are summed in float: their float rounding
// stays below 2^-50 once multiplied by d^3 or d^2; -1/6 and d^2/24 take double-float.
// Then s' = s + (s (cos d - 1) + c sin d), c' = c + (c (cos d - 1) - s sin d).  false for
// |d| > 1/16 (the caller evaluates sin and cos afresh).
GT_HD bool rotate_sc_df(DF s, DF c, DF d, DF *s2, DF *c2)
{
    if (!(fabsf(d.hi) <= 0.0625f)) return false;
    const DF d2 = d * d;
    const float t = d2.hi;
    const float qf = t * fmaf(t, fmaf(t, 1.0f / 362880.0f, -1.0f / 5040.0f), 1.0f / 120.0f);
    const float pf = t * t * fmaf(t, 1.0f / 40320.0f, -1.0f / 720.0f);
    const DF q = DF(-1.0 / 6.0) + DF(qf, 0.0f);
    const DF p = (DF(-0.5f, 0.0f) + d2 * DF(1.0 / 24.0)) + DF(pf, 0.0f);
    const DF sd = d + (d2 * d) * q; // sin d
    const DF cdm1 = d2 * p;         // cos d - 1
    *s2 = s + (s * cdm1 + c * sd);
    *c2 = c + (c * cdm1 - s * sd);
    return true;
}

} // namespace gt
