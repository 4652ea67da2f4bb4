// df.cuh -- double-float arithmetic: a value held as the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits carried by the FP32 pipes
// (host and device, so host tests can check it against FP64 and extended precision).
//
// On GB300 the FP32 pipes issue 64 times the FP64 rate, so a field evaluation in
// double-float costs a few FP64-equivalents of what the same evaluation costs in FP64.
// The range is FP32's: magnitudes must stay within about [2e-31, 3e38] for lo to stay a
// normal float; callers check the inputs that decide this and use FP64 outside.
//
// Building blocks (error-free transformations of two floats):
//   TwoSum (Knuth):      s = fl(a + b), e = (a - (s - b')) + (b - b'), b' = fl(s - a);
//   Fast2Sum (Dekker):   s = fl(a + b), e = b - fl(s - a) when exponent(a) >= exponent(b);
//   product error:       p = fl(a b), e = fma(a, b, -p).
// The sum of two double-floats is the accurate one (both pairs summed with TwoSum, then
// two renormalisations; relative error below 3 u^2, u = 2^-24, cancellation included);
// the product drops lo*lo (relative error below 5 u^2); reciprocal and inverse square
// root take one Newton correction of the FP32 estimate with the residual evaluated in
// double-float and the correction series carried to second order; exp reduces the
// argument by n ln 2 and by 2^-4, sums the Taylor series through the 7th power and
// squares back four times.
#pragma once

#include <math.h>

#ifndef GT_HD
#define GT_HD __host__ __device__ __forceinline__
#endif

namespace gt {

// Round-to-nearest float add and multiply that the compiler may not fuse into an FMA:
// the error-free transformations depend on each operation rounding on its own.
#ifdef __CUDA_ARCH__
#define GT_DF_ADD(a, b) __fadd_rn((a), (b))
#define GT_DF_MUL(a, b) __fmul_rn((a), (b))
#else
#define GT_DF_ADD(a, b) ((a) + (b)) // host builds of this header use -ffp-contract=off
#define GT_DF_MUL(a, b) ((a) * (b))
#endif

struct DF {
    float hi, lo;
    DF() = default;
    GT_HD constexpr DF(float h, float l) : hi(h), lo(l) {}
    GT_HD explicit DF(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    GT_HD explicit constexpr DF(int v) : hi((float)v), lo(0.0f) {}
};

GT_HD double df_to(DF a) { return (double)a.hi + (double)a.lo; }

GT_HD DF df_two_sum(float a, float b)
{
    const float s = GT_DF_ADD(a, b);
    const float bb = GT_DF_ADD(s, -a);
    const float e = GT_DF_ADD(GT_DF_ADD(a, -GT_DF_ADD(s, -bb)), GT_DF_ADD(b, -bb));
    return DF(s, e);
}

// requires exponent(a) >= exponent(b) (or a == 0)
GT_HD DF df_fast_two_sum(float a, float b)
{
    const float s = GT_DF_ADD(a, b);
    const float e = GT_DF_ADD(b, -GT_DF_ADD(s, -a));
    return DF(s, e);
}

GT_HD DF df_two_prod(float a, float b)
{
    const float p = GT_DF_MUL(a, b);
    return DF(p, fmaf(a, b, -p));
}

GT_HD DF operator-(DF a) { return DF(-a.hi, -a.lo); }

GT_HD DF operator+(DF a, DF b)
{
    DF s = df_two_sum(a.hi, b.hi);
    const DF t = df_two_sum(a.lo, b.lo);
    s = df_fast_two_sum(s.hi, GT_DF_ADD(s.lo, t.hi));
    return df_fast_two_sum(s.hi, GT_DF_ADD(s.lo, t.lo));
}

GT_HD DF operator-(DF a, DF b) { return a + (-b); }

GT_HD DF operator*(DF a, DF b)
{
    const float p = GT_DF_MUL(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.lo, b.hi, fmaf(a.hi, b.lo, e));
    return df_fast_two_sum(p, e);
}

// exact scaling by a power of two (no overflow or underflow assumed)
GT_HD DF df_ldexp(DF a, int n) { return DF(ldexpf(a.hi, n), ldexpf(a.lo, n)); }

GT_HD DF fma_t(DF a, DF b, DF c) { return a * b + c; }

// 1/a: y = RN(1/hi) has the exactly representable residual 1 - hi y (one FMA);
// r = 1 - a y to float precision, and 1/a = y / (1 - r) = y (1 + r + r^2 + ...).
GT_HD DF rcp_t(DF a)
{
#ifdef __CUDA_ARCH__
    const float y = __frcp_rn(a.hi);
#else
    const float y = 1.0f / a.hi;
#endif
    float r = fmaf(-a.hi, y, 1.0f);
    r = fmaf(-a.lo, y, r);
    return df_fast_two_sum(y, GT_DF_MUL(y, fmaf(r, r, r)));
}

// 1/sqrt(a): y an FP32 estimate; a y^2 = 1 - r with y^2 exact (product error) and the
// product by a in double-float, so r holds to float precision; then
// 1/sqrt(a) = y (1 - r)^(-1/2) = y (1 + r/2 + 3 r^2/8 + ...).
GT_HD DF rsqrt_t(DF a)
{
#ifdef __CUDA_ARCH__
    const float y = rsqrtf(a.hi);
#else
    const float y = 1.0f / sqrtf(a.hi);
#endif
    const DF ay2 = a * df_two_prod(y, y);
    const float r = GT_DF_ADD(GT_DF_ADD(1.0f, -ay2.hi), -ay2.lo); // 1 - hi exact (Sterbenz)
    return df_fast_two_sum(y, GT_DF_MUL(y, GT_DF_MUL(r, fmaf(0.375f, r, 0.5f))));
}

// exp(a) = 2^n exp(r), r = a - n ln2 with |r| <= ln2/2 (ln 2 split into three floats
// L0 + L1 + L2; n L0 and n L1 exact as product pairs, n L2 rounded -- below 2^-70 of
// ln 2 for the |n| <= 127 met here), s = r/16, exp(s) - 1 by its Taylor series (terms of
// order 5-7 in float: they stay below 2^-24 of the sum), then e <- 2e + e^2 four times,
// result (1 + e) 2^n.  Valid for |a| up to about 87.
GT_HD DF exp_t(DF a)
{
    const float L0 = 0.693147182464599609375f;      // float nearest ln 2
    const float L1 = -1.9046542121259336e-09f;      // float nearest ln 2 - L0
    const float L2 = -8.78318373858934e-17f;        // float nearest ln 2 - L0 - L1
    const float n = rintf(GT_DF_MUL(a.hi, 1.44269502162933349609375f));
    const DF p1 = df_two_prod(n, L0);
    DF p2 = df_two_prod(n, L1);
    p2.lo = fmaf(n, L2, p2.lo);
    const DF r = (a - p1) - p2;
    const DF s(GT_DF_MUL(r.hi, 0.0625f), GT_DF_MUL(r.lo, 0.0625f));
    // q = 1/120 + s/720 + s^2/5040 in float
    const float q = fmaf(s.hi, fmaf(s.hi, 1.0f / 5040.0f, 1.0f / 720.0f), 1.0f / 120.0f);
    DF t = s * DF(q, 0.0f) + DF(1.0 / 24.0);
    t = s * t + DF(1.0 / 6.0);
    t = s * t + DF(0.5f, 0.0f);
    DF e = s * (s * t) + s; // exp(s) - 1
#pragma unroll
    for (int k = 0; k < 4; k++) e = e * e + DF(GT_DF_MUL(e.hi, 2.0f), GT_DF_MUL(e.lo, 2.0f));
    return df_ldexp(DF(1.0f, 0.0f) + e, (int)n);
}

#undef GT_DF_ADD
#undef GT_DF_MUL

} // namespace gt
