// compensated_sum.cpp -- host check of the FP32-mixed state update f2_add
// (csrc/compensated.cuh): a (hi, lo) float pair accumulating float increments, against
// the exact running sum (double, whose own rounding is ~1e-9 of the bound checked).
// Sequences: a coordinate moved by small increments of both signs, a coordinate
// starting at zero (t, phi), and a momentum driven through zero and back (where hi is
// the smaller term of its updates).  Prints, per sequence, the largest ratio of the
// pair's error to the bound sum_k (u |d_k| + u^2 |hi_k|), u = 2^-24, and the largest
// |lo| / ulp(hi) seen.
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#define GT_HD inline
#include "../paper_2310_15183_gb300/csrc/compensated.cuh"

static uint64_t g_state = 0x5eed2310ull;
static double uni(double lo, double hi)
{
    g_state = g_state * 6364136223846793005ull + 1442695040888963407ull;
    return lo + (hi - lo) * (double)(g_state >> 11) * (1.0 / 9007199254740992.0);
}

struct Result {
    double worst_ratio, worst_lo;
};

// kind 0: start 15, d ~ U[-1e-4, 1e-4]; 1: start 0, d ~ U[0, 2e-4];
// 2: start 0.3, drift -1e-5 per step for 6e4 steps then +1e-5 (two zero crossings)
static Result run(int kind, int steps)
{
    const double u = ldexp(1.0, -24);
    gt::F2 a = gt::f2_from(kind == 0 ? 15.0 : (kind == 1 ? 0.0 : 0.3));
    double exact = gt::f2_to(a), bound = 0.0;
    Result res = {0.0, 0.0};
    for (int k = 0; k < steps; k++) {
        float d;
        if (kind == 0)
            d = (float)uni(-1e-4, 1e-4);
        else if (kind == 1)
            d = (float)uni(0.0, 2e-4);
        else
            d = (float)((k < steps / 2 ? -1e-5 : 1e-5) * uni(0.5, 1.5));
        bound += u * fabs((double)d) + u * u * fabs((double)a.hi);
        gt::f2_add(a, d);
        exact += (double)d;
        const double err = fabs(gt::f2_to(a) - exact);
        const double ratio = err / (bound + 1e-300);
        if (ratio > res.worst_ratio) res.worst_ratio = ratio;
        if (a.hi != 0.0f) {
            int e;
            frexpf(a.hi, &e);
            const double ulp = ldexp(1.0, e - 24);
            const double l = fabs((double)a.lo) / ulp;
            if (l > res.worst_lo) res.worst_lo = l;
        }
    }
    return res;
}

int main()
{
    const Result r0 = run(0, 400000), r1 = run(1, 400000), r2 = run(2, 120000);
    printf("{\"coordinate\": [%.6g, %.6g], \"from_zero\": [%.6g, %.6g], "
           "\"zero_crossing\": [%.6g, %.6g]}\n",
           r0.worst_ratio, r0.worst_lo, r1.worst_ratio, r1.worst_lo, r2.worst_ratio, r2.worst_lo);
    return 0;
}
