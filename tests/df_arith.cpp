// df_arith.cpp -- host check of the double-float arithmetic of the FP32-mixed zone
// (csrc/df.cuh, csrc/zone_df.cuh) against extended precision: sum, difference
// (cancellation included), product, reciprocal, inverse square root, exp and the stage
// rotation of sin/cos on seeded random operands; the reverse-sweep Manko-Novikov rates
// evaluated in double-float and in double against the same rates in long double, at
// seeded random phase-space points of the zone (r_+ < r < 5M, all inclinations) of
// several spacetimes -- the zone's range check (every exponent of the evaluation within
// its bound) decides which points the double-float evaluation takes, the rest go to
// FP64 in the kernels; and the Kerr rates likewise for four spins, half the points
// within 10 % of r_+.
// Prints one JSON line of worst relative errors (units of the operation's result, or of
// the largest rate component).
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#define GT_HD inline
static inline void sincos_t(double x, double *s, double *c) { *s = sin(x); *c = cos(x); }
static inline void sincos_t(float x, float *s, float *c) { *s = sinf(x); *c = cosf(x); }
static inline double exp_t(double x) { return exp(x); }
static inline float exp_t(float x) { return expf(x); }
static inline double rcp_t(double x) { return 1.0 / x; }
static inline float rcp_t(float x) { return 1.0f / x; }
static inline double rsqrt_t(double x) { return 1.0 / sqrt(x); }
static inline float rsqrt_t(float x) { return 1.0f / sqrtf(x); }
static inline double fma_t(double a, double b, double c) { return fma(a, b, c); }
static inline float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
typedef long double LD;
static inline void sincos_t(LD x, LD *s, LD *c) { *s = sinl(x); *c = cosl(x); }
static inline LD exp_t(LD x) { return expl(x); }
static inline LD rcp_t(LD x) { return 1.0L / x; }
static inline LD rsqrt_t(LD x) { return 1.0L / sqrtl(x); }
static inline LD fma_t(LD a, LD b, LD c) { return fmal(a, b, c); }
// the kernels' headers declare the double-float overloads in namespace gt, where they
// would hide these
namespace gt {
using ::exp_t;
using ::fma_t;
using ::rcp_t;
using ::rsqrt_t;
using ::sincos_t;
} // namespace gt

#include "../paper_2310_15183_gb300/csrc/df.cuh"
#include "../paper_2310_15183_gb300/csrc/spacetime.cuh"
#include "../paper_2310_15183_gb300/csrc/zone_df.cuh"

using gt::DF;

static uint64_t g_state = 0x2310151883ull;
static double uni(double lo, double hi)
{ // splitmix64
    uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return lo + (hi - lo) * (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

static LD ld(DF a) { return (LD)a.hi + (LD)a.lo; }
// a double-float whose value is exactly representable in long double, with a random
// exponent in [2^lo_e, 2^hi_e] and a random sign
static DF rnd_df(int lo_e, int hi_e)
{
    const double m = uni(1.0, 2.0) * ldexp(1.0, (int)floor(uni(lo_e, hi_e)));
    return DF(uni(0, 1) < 0.5 ? -m : m);
}
static double relerr(LD got, LD want) { return (double)(fabsl(got - want) / fabsl(want)); }

template <class T>
static gt::SpacetimeT<T> mn_constants(LD M, LD S, LD Q)
{
    const LD sm = S / M;
    const LD al = (-M + sqrtl(M * M - sm * sm)) / sm;
    const LD k = M * (1 - al * al) / (1 + al * al);
    const LD beta = Q * M * M * M / (k * k * k);
    gt::SpacetimeT<T> c = {};
    c.kind = gt::KIND_MN;
    c.M = T((double)M);
    c.alpha = T((double)al);
    c.k = T((double)k);
    c.ik = T((double)(1 / k));
    c.beta = T((double)beta);
    c.two_beta = T((double)(2 * beta));
    c.three_beta2 = T((double)(3 * beta * beta));
    c.c_g = T((double)((1 - al * al) * (1 - al * al) / (k * k)));
    c.w_inf = T((double)(4 * k * al / (1 - al * al)));
    c.k2 = T((double)(k * k));
    c.inv_k2 = T((double)(1 / (k * k)));
    c.two_k = T((double)(2 * k));
    c.r_plus = T((double)(M + k));
    return c;
}

// the long double constants from the same double values the other two start from
static gt::SpacetimeT<LD> widen(const gt::SpacetimeC &c)
{
    gt::SpacetimeT<LD> w = {};
    w.kind = c.kind;
    w.M = c.M;
    w.alpha = c.alpha;
    w.k = c.k;
    w.ik = c.ik;
    w.beta = c.beta;
    w.two_beta = c.two_beta;
    w.three_beta2 = c.three_beta2;
    w.c_g = c.c_g;
    w.w_inf = c.w_inf;
    w.k2 = c.k2;
    w.inv_k2 = c.inv_k2;
    w.two_k = c.two_k;
    w.r_plus = c.r_plus;
    return w;
}

int main()
{
    // ---- arithmetic
    double w_add = 0, w_cancel = 0, w_mul = 0, w_rcp = 0, w_rsqrt = 0, w_exp = 0, w_rot = 0;
    long n_rot_refused = 0;
    for (int i = 0; i < 200000; ++i) {
        const DF a = rnd_df(-40, 40), b = rnd_df(-40, 40);
        const LD sa = ld(a), sb = ld(b);
        if (sa + sb != 0) w_add = fmax(w_add, relerr(ld(a + b), sa + sb));
        // near-cancellation: b = -a (1 + eps), eps down to 2^-40
        const DF c = DF(-(double)sa * (1.0 + ldexp(uni(-1, 1), -(int)uni(1, 40))));
        if (sa + ld(c) != 0) w_cancel = fmax(w_cancel, relerr(ld(a + c), sa + ld(c)));
        w_mul = fmax(w_mul, relerr(ld(a * b), sa * sb));
        w_rcp = fmax(w_rcp, relerr(ld(gt::rcp_t(a)), 1 / sa));
        const DF p = DF(fabs((double)sa));
        w_rsqrt = fmax(w_rsqrt, relerr(ld(gt::rsqrt_t(p)), 1 / sqrtl(ld(p))));
        const DF x = DF(uni(-69.0, 87.0)) + DF(uni(-1, 1) * 1e-9); // lo normal: e^-69 > 2^-99
        w_exp = fmax(w_exp, relerr(ld(gt::exp_t(x)), expl(ld(x))));
        // the stage rotation of sin/cos by d (|d| <= 1/16; beyond it the caller refuses)
        const double th = uni(0.0, M_PI), d = uni(-1, 1) * ldexp(1.0, -(int)uni(4, 30));
        const DF S(sin(th)), C(cos(th)), D(d);
        DF s2, c2;
        if (!gt::rotate_sc_df(S, C, D, &s2, &c2)) {
            ++n_rot_refused;
            continue;
        }
        const LD ang = atan2l(ld(S), ld(C)) + ld(D); // the angle of (S, C), rotated by D
        w_rot = fmax(w_rot, (double)fmaxl(fabsl(ld(s2) - sinl(ang)), fabsl(ld(c2) - cosl(ang))));
    }

    // ---- Manko-Novikov rates in the zone
    const double spacetimes[][3] = {{0.5, 0.24, 2.0},      {0.5, 0.24, -2.0},
                                    {0.5, 0.025, 2.0},     {0.5, 0.245, 2.0},
                                    {0.5, 0.245, -2.0},    {1.0, 0.5, 1.0},
                                    {1.0, 0.9, 5.0},       {1.0, 0.3, -0.5}};
    std::vector<double> e_df, e_f64; // per accepted point: largest error / largest rate
    long n_pts = 0, n_df = 0, n_shell = 0, n_shell_df = 0;
    for (const auto &sp : spacetimes) {
        const double M = sp[0], S = sp[1], Q = sp[2];
        const gt::SpacetimeC c = mn_constants<double>(M, S, Q);
        const gt::SpacetimeT<LD> cl = widen(c);
        const gt::SpacetimeT<DF> cd = gt::to_df(c);
        const bool listing = (M == 0.5 && S == 0.24 && Q == 2.0);
        for (int i = 0; i < 20000; ++i) {
            // the listing's spacetime: the shell its trapped rays live in (1.6M - 2.4M);
            // all spacetimes: the whole zone from just outside r_+ to 5M
            const double r = (listing && i % 2) ? uni(0.8, 1.2)
                                                : c.r_plus + uni(1e-4, 5.0 * M - c.r_plus);
            const double th = uni(1e-3, M_PI - 1e-3);
            const double pr = uni(-2, 2), pth = uni(-3, 3), pt = -1.0, pph = uni(-4, 4);
            const double s = sin(th), cs = cos(th);
            gt::Rates<LD> oL;
            gt::mn_rates_sc<LD>(cl, (LD)r, (LD)s, (LD)cs, (LD)pr, (LD)pth, (LD)pt, (LD)pph, oL);
            const LD vL[6] = {oL.dt, oL.dr, oL.dth, oL.dph, oL.dpr, oL.dpth};
            LD scale = 0;
            bool fin = true;
            for (int j = 0; j < 6; ++j) {
                scale = fmaxl(scale, fabsl(vL[j]));
                fin = fin && isfinite(vL[j]);
            }
            if (!fin || !(scale > 0)) continue;
            ++n_pts;
            const bool shell = listing && i % 2;
            n_shell += shell;
            gt::Rates<double> o64, odf;
            gt::mn_rates_sc<double>(c, r, s, cs, pr, pth, pt, pph, o64);
            if (!gt::mn_rates_df(cd, DF(r), DF(s), DF(cs), DF(pr), DF(pth), DF(pt), DF(pph), odf))
                continue;
            ++n_df;
            n_shell_df += shell;
            const double v64[6] = {o64.dt, o64.dr, o64.dth, o64.dph, o64.dpr, o64.dpth};
            const double vd[6] = {odf.dt, odf.dr, odf.dth, odf.dph, odf.dpr, odf.dpth};
            double ed = 0, e6 = 0;
            for (int j = 0; j < 6; ++j) {
                ed = fmax(ed, (double)(fabsl(vd[j] - vL[j]) / scale));
                e6 = fmax(e6, (double)(fabsl(v64[j] - vL[j]) / scale));
            }
            e_df.push_back(ed);
            e_f64.push_back(e6);
        }
    }
    // ---- Kerr rates from just outside r_+ to 5M (the zone an explicit r_switch sets)
    std::vector<double> k_df, k_f64;
    for (const double a : {0.3, 0.6, 0.9, 0.99}) {
        const double M = 1.0;
        gt::SpacetimeC c = {};
        c.kind = gt::KIND_KERR;
        c.M = M;
        c.a = a * M;
        c.a2 = c.a * c.a;
        c.r_plus = M + sqrt(M * M - c.a2);
        gt::SpacetimeT<LD> cl = {};
        cl.kind = gt::KIND_KERR;
        cl.M = c.M;
        cl.a = c.a;
        cl.a2 = c.a2;
        const gt::SpacetimeT<DF> cd = gt::to_df(c);
        for (int i = 0; i < 20000; ++i) {
            const double r = c.r_plus * (1.0 + uni(1e-4, 0.1)) + (i % 2 ? uni(0.0, 5.0 * M) : 0.0);
            const double th = uni(1e-3, M_PI - 1e-3);
            const double pr = uni(-2, 2), pth = uni(-3, 3), pt = -1.0, pph = uni(-4, 4);
            const double s = sin(th), cs = cos(th);
            gt::Rates<LD> oL;
            gt::kerr_rates_sc<LD>(cl, (LD)r, (LD)s, (LD)cs, (LD)pr, (LD)pth, (LD)pt, (LD)pph, oL);
            const LD vL[6] = {oL.dt, oL.dr, oL.dth, oL.dph, oL.dpr, oL.dpth};
            LD scale = 0;
            for (int j = 0; j < 6; ++j) scale = fmaxl(scale, fabsl(vL[j]));
            if (!(scale > 0) || !isfinite(scale)) continue;
            gt::Rates<double> o64;
            gt::kerr_rates_sc<double>(c, r, s, cs, pr, pth, pt, pph, o64);
            gt::Rates<DF> od;
            gt::kerr_rates_sc<DF>(cd, DF(r), DF(s), DF(cs), DF(pr), DF(pth), DF(pt), DF(pph), od);
            const double v64[6] = {o64.dt, o64.dr, o64.dth, o64.dph, o64.dpr, o64.dpth};
            const DF vd[6] = {od.dt, od.dr, od.dth, od.dph, od.dpr, od.dpth};
            double ed = 0, e6 = 0;
            for (int j = 0; j < 6; ++j) {
                ed = fmax(ed, (double)(fabsl(ld(vd[j]) - vL[j]) / scale));
                e6 = fmax(e6, (double)(fabsl(v64[j] - vL[j]) / scale));
            }
            k_df.push_back(ed);
            k_f64.push_back(e6);
        }
    }
    auto pct = [](std::vector<double> v, double q) {
        std::sort(v.begin(), v.end());
        return v.empty() ? NAN : v[(size_t)(q * (double)(v.size() - 1))];
    };
    printf("{\"add\": %.3e, \"add_cancel\": %.3e, \"mul\": %.3e, \"rcp\": %.3e, \"rsqrt\": %.3e, "
           "\"exp\": %.3e, \"rotate_abs\": %.3e, \"rotate_refused\": %ld, \"zone_points\": %ld, \"zone_points_df\": %ld, "
           "\"shell_points\": %ld, \"shell_points_df\": %ld, \"rates_df_median\": %.3e, "
           "\"rates_df_p99\": %.3e, \"rates_df_max\": %.3e, \"rates_f64_median\": %.3e, "
           "\"rates_f64_p99\": %.3e, \"rates_f64_max\": %.3e, \"kerr_points\": %zu, "
           "\"kerr_df_median\": %.3e, \"kerr_df_p99\": %.3e, \"kerr_df_max\": %.3e, "
           "\"kerr_f64_median\": %.3e, \"kerr_f64_p99\": %.3e, \"kerr_f64_max\": %.3e}\n",
           w_add, w_cancel, w_mul, w_rcp, w_rsqrt, w_exp, w_rot, n_rot_refused, n_pts, n_df, n_shell, n_shell_df,
           pct(e_df, 0.5), pct(e_df, 0.99), pct(e_df, 1.0), pct(e_f64, 0.5), pct(e_f64, 0.99),
           pct(e_f64, 1.0), k_df.size(), pct(k_df, 0.5), pct(k_df, 0.99), pct(k_df, 1.0),
           pct(k_f64, 0.5), pct(k_f64, 0.99), pct(k_f64, 1.0));
    return 0;
}
