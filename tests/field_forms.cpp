// field_forms.cpp -- host check of the device field templates: the reverse-sweep
// Manko-Novikov rates (direct multipole sums, as the FP64 kernels run them, and the
// closed-form series tails of the FP32 kernels) against the forward dual-number rates,
// in double and in float, at seeded random phase-space points of several (alpha, k,
// beta) spacetimes.
// Prints the largest relative differences (against the largest rate component) of
// reverse vs forward in double, and of float reverse vs double reverse at the points
// where the float forward form is finite (both float forms overflow together where the
// Manko-Novikov exponentials leave the float range), plus the count of points where one
// float form is finite and the other is not.
#include <math.h>
#include <stdint.h>
#include <stdio.h>

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

#include "../paper_2310_15183_gb300/csrc/spacetime.cuh"

static uint64_t g_state = 0x2310151830ull;
static double uni(double lo, double hi)
{ // splitmix64
    uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return lo + (hi - lo) * (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

static double rel(double a, double b, double scale) { return fabs(a - b) / scale; }

int main()
{
    double worst_fwd = 0.0, worst_tail = 0.0, worst_f32 = 0.0, worst_f32_fwd = 0.0;
    long n = 0, n_f32 = 0, finite_mismatch = 0;
    const double Ms[] = {0.5, 1.0};
    for (double M : Ms)
        for (int sp = 0; sp < 4; ++sp) {
            const double a = M * (0.05 + 0.3 * sp); // spin S / M
            const double Q = (sp % 2 ? -1.0 : 1.0) * (0.5 + sp);
            const double al = (-M + sqrt(M * M - a * a)) / a;
            const double k = M * (1.0 - al * al) / (1.0 + al * al);
            gt::SpacetimeT<double> c = {};
            c.kind = gt::KIND_MN;
            c.M = M;
            c.alpha = al;
            c.k = k;
            c.ik = 1.0 / k;
            c.beta = Q * M * M * M / (k * k * k);
            c.two_beta = 2.0 * c.beta;
            c.three_beta2 = 3.0 * c.beta * c.beta;
            c.c_g = (1.0 - al * al) * (1.0 - al * al) / (k * k);
            c.w_inf = 4.0 * k * al / (1.0 - al * al);
            c.k2 = k * k;
            c.inv_k2 = 1.0 / (k * k);
            c.two_k = 2.0 * k;
            c.r_plus = M + k;
            const gt::SpacetimeT<float> cf = gt::to_float(c);
            for (int i = 0; i < 400; ++i) {
                const double r = c.r_plus + uni(0.3, 40.0) * M, th = uni(0.05, M_PI - 0.05);
                const double pr = uni(-2, 2), pth = uni(-3, 3), pt = -1.0, pph = uni(-4, 4);
                gt::Rates<double> o1, o2, o3;
                gt::mn_rates<double>(c, r, th, pr, pth, pt, pph, o1);
                gt::mn_rates_fwd<double>(c, r, th, pr, pth, pt, pph, o2);
                gt::mn_rates<double, true>(c, r, th, pr, pth, pt, pph, o3); // the FP32 form
                const double v1[6] = {o1.dt, o1.dr, o1.dth, o1.dph, o1.dpr, o1.dpth};
                const double v2[6] = {o2.dt, o2.dr, o2.dth, o2.dph, o2.dpr, o2.dpth};
                const double v3[6] = {o3.dt, o3.dr, o3.dth, o3.dph, o3.dpr, o3.dpth};
                double scale = 0.0;
                for (int j = 0; j < 6; ++j) scale = fmax(scale, fabs(v2[j]));
                if (!(scale > 0.0) || !isfinite(scale)) continue;
                gt::Rates<float> of, og;
                gt::mn_rates<float>(cf, (float)r, (float)th, (float)pr, (float)pth, (float)pt,
                                    (float)pph, of);
                gt::mn_rates_fwd<float>(cf, (float)r, (float)th, (float)pr, (float)pth, (float)pt,
                                        (float)pph, og);
                const double vf[6] = {of.dt, of.dr, of.dth, of.dph, of.dpr, of.dpth};
                const double vg[6] = {og.dt, og.dr, og.dth, og.dph, og.dpr, og.dpth};
                bool fin_f = true, fin_g = true;
                for (int j = 0; j < 6; ++j) {
                    worst_fwd = fmax(worst_fwd, rel(v1[j], v2[j], scale));
                    worst_tail = fmax(worst_tail, rel(v3[j], v2[j], scale));
                    fin_f = fin_f && isfinite(vf[j]);
                    fin_g = fin_g && isfinite(vg[j]);
                }
                if (fin_f != fin_g) ++finite_mismatch;
                if (fin_g) {
                    for (int j = 0; j < 6; ++j) {
                        worst_f32 = fmax(worst_f32, fin_f ? rel(vf[j], v1[j], scale) : INFINITY);
                        worst_f32_fwd = fmax(worst_f32_fwd, rel(vg[j], v1[j], scale));
                    }
                    ++n_f32;
                }
                ++n;
            }
        }
    printf("{\"points\": %ld, \"reverse_vs_forward_f64\": %.3e, \"tail_form_vs_forward_f64\": %.3e, "
           "\"points_f32\": %ld, "
           "\"f32_vs_f64\": %.3e, \"f32_forward_vs_f64\": %.3e, \"finite_mismatch\": %ld}\n",
           n, worst_fwd, worst_tail, n_f32, worst_f32, worst_f32_fwd, finite_mismatch);
    return 0;
}
