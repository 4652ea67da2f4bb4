/*
 * geodesic_oracle.c -- plain, slow FP64 CPU oracle of the null-geodesic
 * ray tracer described in "Graphical Processing of Geodesic Propagation in
 * Python" (F. Imbens).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference legs load this library.  The product
 * path (the CUDA library and its Python binding) never calls it, and the two
 * share no source: nothing here is included by, or includes, the CUDA code.
 *
 * What it computes, function by function (each cites its passage):
 *   - the spacetimes of Sec. 2.2: Schwarzschild (Eq. schwMetric) as Kerr with
 *     a = 0, Kerr in Boyer-Lindquist coordinates (Sec. 2.2.2) and
 *     Manko-Novikov (Sec. 2.2.3), as the lower metric g_{mu nu}, the inverse
 *     g^{mu nu} and the coordinate derivatives d_mu g^{nu sigma};
 *   - the Hamiltonian equations of motion, Eq. hamGeodesic (Sec. 2.1 and
 *     Appendix A, "The Legendre Transform"):
 *         dq^mu/dtau = g^{mu nu} p_nu,   dp_mu/dtau = -1/2 d_mu g^{nu sigma} p_nu p_sigma;
 *   - the pinhole camera of the appendix listing "Code for propagation of
 *     rays" together with Sec. 3.3.1 (light-like v^t by the quadratic, rescale
 *     to v^t = -1, p_mu = g_{mu nu} v^nu);
 *   - RK4 (Sec. 3.1.2) with the step normalised by dq^t/dtau from the first
 *     stage, and the exit tests of the listing's propagation kernel: escape
 *     when r > 1.5 r_start, horizon when the step falls below
 *     step_precision * 3e-5, otherwise stop after n_steps.
 *
 *   - the optional paper-numerics variants: forward-difference metric
 *     derivatives with the listing's derPrecision 1e-8 (three metric
 *     evaluations per stage), float32 kernel arguments and outputs, and the
 *     explicit Euler integrator of Sec. 3.1.1;
 *   - the equatorial ring of Sec. 5's renders as an exit condition and the
 *     redshift of Sec. 3.3.3 (circular-orbit emitter, static observer).
 *
 * Derivatives are exact, not finite differences: Kerr uses hand-derived
 * closed forms of d_r, d_theta g^{mu nu}; Manko-Novikov uses complex-step
 * differentiation Im g(x + i h)/h with h = 1e-30 (exact to rounding because
 * every operation in the metric is analytic).
 *
 * Readings of the paper that this file takes (where the text is garbled or
 * silent) are marked READING and listed in the design notes:
 *   Kerr g_{t phi} sign and g_tt denominator (Carroll convention), the
 *   Manko-Novikov line element, B as a sum of squares, gamma' with the
 *   (-1)^(2-l) factor and "-2 + sum", the 1/2 in dp/dtau, exact 1/6 RK4
 *   weights (0.1667 with OR_FLAG_COMPAT_WEIGHTS), v^phi = alpha/sin(theta0)
 *   (alpha with OR_FLAG_COMPAT_CAMERA), v^t normalised to -1, strict exit
 *   comparisons, and the NONFINITE status.
 *
 * Parity pins: every function here is pinned by tests that do not re-type
 * its formula (closed forms, invariants, special cases, convergence order).
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_ESCAPED 0
#define OR_HORIZON 1
#define OR_MAXSTEPS 2
#define OR_NONFINITE 3
#define OR_DISK 5 /* the ray entered the ring volume */

#define OR_OK 0
#define OR_ERR_INVALID_ARG (-1)

#define OR_FLAG_COMPAT_WEIGHTS 1 /* RK4 weights 0.1667 as in the listing */
#define OR_FLAG_COMPAT_CAMERA 2  /* v^phi = alpha (no 1/sin(theta0)) */
#define OR_FLAG_FD_DERIVS 4      /* forward-difference metric derivatives, derPrecision 1e-8 */
#define OR_FLAG_F32_IO 8         /* float32 spacetime parameters, initial state and outputs */
#define OR_FLAG_EULER 16         /* explicit Euler instead of RK4 (Sec. 3.1.1) */

#define OR_FD_DELTA 1e-8 /* the listing's derPrecision */

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Spacetime parameters                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double M, S, Q; /* mass, spin S, Manko-Novikov quadrupole deviation q */
    int is_mn;      /* Q != 0 -> Manko-Novikov, else Kerr */
    double a;       /* Kerr a = S/M (Sec. 2.2.2) */
    /* Manko-Novikov constants (Sec. 2.2.3) */
    double alpha, k, beta;
} spacetime;

/* Sec. 2.2.2: a black hole for -M^2 < S < M^2.  Sec. 2.2.3: alpha has S/M in
 * its denominator, so Q != 0 needs S != 0 (the paper substitutes S = 0.1 M^2
 * when it wants a "non-rotating" Manko-Novikov hole, Sec. 5). */
static int spacetime_init(spacetime *st, double M, double S, double Q)
{
    if (!(M > 0.0) || !isfinite(M) || !isfinite(S) || !isfinite(Q)) return OR_ERR_INVALID_ARG;
    if (!(fabs(S) < M * M)) return OR_ERR_INVALID_ARG;
    if (Q != 0.0 && S == 0.0) return OR_ERR_INVALID_ARG;
    st->M = M;
    st->S = S;
    st->Q = Q;
    st->is_mn = (Q != 0.0);
    st->a = S / M;
    if (st->is_mn) {
        double sm = S / M;
        st->alpha = (-M + sqrt(M * M - sm * sm)) / sm;
        st->k = M * (1.0 - st->alpha * st->alpha) / (1.0 + st->alpha * st->alpha);
        st->beta = Q * M * M * M / (st->k * st->k * st->k);
    } else {
        st->alpha = st->k = st->beta = 0.0;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Kerr, Boyer-Lindquist coordinates (Sec. 2.2.2)                            */
/* ------------------------------------------------------------------------ */

/* Lower metric g_{mu nu}, index order (t, r, theta, phi).
 * READING: the printed g_tt has rho where rho^2 is meant and the printed
 * g_{t phi} has a plus sign; Carroll's convention (which the paper says it
 * follows) is g_tt = -(1 - 2Mr/rho^2) and g_{t phi} = -2 M a r sin^2/rho^2. */
static void kerr_lower(const spacetime *st, double r, double th, double g[4][4])
{
    const double M = st->M, a = st->a;
    const double s = sin(th), c = cos(th), s2 = s * s;
    const double rho2 = r * r + a * a * c * c;
    const double Delta = r * r - 2.0 * M * r + a * a;
    memset(g, 0, 16 * sizeof(double));
    g[0][0] = -(1.0 - 2.0 * M * r / rho2);
    g[0][3] = g[3][0] = -2.0 * M * a * r * s2 / rho2;
    g[1][1] = rho2 / Delta;
    g[2][2] = rho2;
    g[3][3] = s2 / rho2 * ((r * r + a * a) * (r * r + a * a) - a * a * Delta * s2);
}

/* Inverse metric g^{mu nu} in closed form (inverse of kerr_lower). */
static void kerr_upper(const spacetime *st, double r, double th, double g[4][4])
{
    const double M = st->M, a = st->a;
    const double s = sin(th), c = cos(th), s2 = s * s;
    const double rho2 = r * r + a * a * c * c;
    const double Delta = r * r - 2.0 * M * r + a * a;
    const double AK = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s2;
    const double D = rho2 * Delta;
    memset(g, 0, 16 * sizeof(double));
    g[0][0] = -AK / D;
    g[0][3] = g[3][0] = -2.0 * M * a * r / D;
    g[1][1] = Delta / rho2;
    g[2][2] = 1.0 / rho2;
    g[3][3] = (Delta - a * a * s2) / (D * s2);
}

/* The same inverse metric in complex arithmetic; used only to check the
 * hand-derived derivatives against complex-step differentiation. */
static void kerr_upper_c(const spacetime *st, cplx r, cplx th, cplx g[4][4])
{
    const double M = st->M, a = st->a;
    const cplx s = csin(th), c = ccos(th), s2 = s * s;
    const cplx rho2 = r * r + a * a * c * c;
    const cplx Delta = r * r - 2.0 * M * r + a * a;
    const cplx AK = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s2;
    const cplx D = rho2 * Delta;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) g[i][j] = 0.0;
    g[0][0] = -AK / D;
    g[0][3] = g[3][0] = -2.0 * M * a * r / D;
    g[1][1] = Delta / rho2;
    g[2][2] = 1.0 / rho2;
    g[3][3] = (Delta - a * a * s2) / (D * s2);
}

/* Hand-derived d_r and d_theta of kerr_upper; dg[mu][nu][sigma] = d_mu g^{nu sigma}
 * (mu = 0 and mu = 3 vanish: the metric depends on r and theta only). */
static void kerr_dupper(const spacetime *st, double r, double th, double dg[4][4][4])
{
    const double M = st->M, a = st->a;
    const double s = sin(th), c = cos(th), s2 = s * s;
    const double rho2 = r * r + a * a * c * c;
    const double Delta = r * r - 2.0 * M * r + a * a;
    const double AK = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s2;
    const double D = rho2 * Delta;
    const double Nphi = Delta - a * a * s2; /* numerator of g^{phi phi} */
    memset(dg, 0, 64 * sizeof(double));

    /* d/dr */
    const double rho2_r = 2.0 * r;
    const double Delta_r = 2.0 * r - 2.0 * M;
    const double AK_r = 4.0 * r * (r * r + a * a) - a * a * s2 * Delta_r;
    const double D_r = rho2_r * Delta + rho2 * Delta_r;
    dg[1][0][0] = -(AK_r * D - AK * D_r) / (D * D);
    dg[1][0][3] = dg[1][3][0] = -2.0 * M * a * (D - r * D_r) / (D * D);
    dg[1][1][1] = (Delta_r * rho2 - Delta * rho2_r) / (rho2 * rho2);
    dg[1][2][2] = -rho2_r / (rho2 * rho2);
    dg[1][3][3] = (Delta_r * D - Nphi * D_r) / (D * D * s2);

    /* d/dtheta */
    const double rho2_t = -2.0 * a * a * c * s;
    const double s2_t = 2.0 * s * c;
    const double AK_t = -a * a * Delta * s2_t;
    const double D_t = rho2_t * Delta;
    const double Nphi_t = -a * a * s2_t;
    const double Den = D * s2, Den_t = D_t * s2 + D * s2_t;
    dg[2][0][0] = -(AK_t * D - AK * D_t) / (D * D);
    dg[2][0][3] = dg[2][3][0] = 2.0 * M * a * r * D_t / (D * D);
    dg[2][1][1] = -Delta * rho2_t / (rho2 * rho2);
    dg[2][2][2] = -rho2_t / (rho2 * rho2);
    dg[2][3][3] = (Nphi_t * Den - Nphi * Den_t) / (Den * Den);
}

/* ------------------------------------------------------------------------ */
/* Manko-Novikov (Sec. 2.2.3)                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    cplx f, omega, e2gamma, rho2, Delta, sin_th;
} mn_fields;

/* The functions of Sec. 2.2.3 evaluated literally, in complex arithmetic so
 * that the same code gives values (zero imaginary part) and complex-step
 * derivatives.  Legendre polynomials P_l take the argument x y / R.
 * READING (B): printed as a product of two brackets; it is the sum of their
 * squares (asymptotic flatness f -> 1 fixes this).
 * READING (gamma'): the printed "beta(-2 sum ...)" with "(-1^{2-l})" is
 * beta(-2 + sum_{l=0}^{2} (x - y + (-1)^{2-l}(x + y)) P_l / R^{l+1})
 * (regularity e^{2 gamma} = 1 on the axis fixes this). */
static void mn_fields_c(const spacetime *st, cplx r, cplx th, mn_fields *o)
{
    const double M = st->M, k = st->k, al = st->alpha, be = st->beta;
    const cplx x = (r - M) / k;
    const cplx y = ccos(th);
    const cplx R = csqrt(x * x + y * y - 1.0);
    const cplx u = x * y / R;
    cplx P[4];
    P[0] = 1.0;
    P[1] = u;
    P[2] = (3.0 * u * u - 1.0) / 2.0;
    P[3] = (5.0 * u * u * u - 3.0 * u) / 2.0;

    cplx sum_a = 0.0, sum_b = 0.0, sum_g = 0.0;
    cplx Rpow = R; /* R^{l+1} */
    for (int l = 0; l <= 2; l++) {
        const double sgn3 = ((3 - l) % 2 == 0) ? 1.0 : -1.0; /* (-1)^{3-l} */
        const double sgn2 = ((2 - l) % 2 == 0) ? 1.0 : -1.0; /* (-1)^{2-l} */
        sum_a += (x - y) * P[l] / Rpow;
        sum_b += sgn3 * (x + y) * P[l] / Rpow;
        sum_g += (x - y + sgn2 * (x + y)) * P[l] / Rpow;
        Rpow *= R;
    }
    const cplx fa = -al * cexp(-2.0 * be * (-1.0 + sum_a)); /* fraktur a */
    const cplx fb = al * cexp(2.0 * be * (1.0 + sum_b));   /* fraktur b */

    const cplx x2m1 = x * x - 1.0, one_m_y2 = 1.0 - y * y;
    const cplx ab = fa * fb;
    const cplx A = x2m1 * (1.0 + ab) * (1.0 + ab) - one_m_y2 * (fb - fa) * (fb - fa);
    const cplx B1 = (x + 1.0) + (x - 1.0) * ab;
    const cplx B2 = (1.0 + y) * fa + (1.0 - y) * fb;
    const cplx B = B1 * B1 + B2 * B2;
    const cplx C = x2m1 * (1.0 + ab) * ((fb - fa) - y * (fa + fb)) +
                   one_m_y2 * (fb - fa) * ((1.0 + ab) + x * (1.0 - ab));
    const cplx R3 = R * R * R;
    const cplx psi = be * P[2] / R3;
    const cplx gammap = clog(csqrt(x2m1 / (x * x - y * y))) +
                        3.0 * be * be / (2.0 * R3 * R3) * (P[3] * P[3] - P[2] * P[2]) +
                        be * (-2.0 + sum_g);

    o->f = cexp(2.0 * psi) * A / B;
    o->omega = 2.0 * k * cexp(-2.0 * psi) * C / A - 4.0 * k * al / (1.0 - al * al);
    o->e2gamma = cexp(2.0 * gammap) * A / (x2m1 * (1.0 - al * al) * (1.0 - al * al));
    o->rho2 = (r - M) * (r - M) - k * k * y * y;
    o->Delta = (r - M) * (r - M) - k * k;
    o->sin_th = csin(th);
}

/* READING (line element): the printed form lacks the square on (dt - w dphi)
 * and the d theta^2; the metric is
 *   -f (dt - w dphi)^2 + e^{2g} rho^2/(f Delta) dr^2 + e^{2g} rho^2/f dtheta^2
 *   + Delta sin^2/f dphi^2,
 * whose inverse is the one the listing's metric function writes out. */
static void mn_lower_c(const spacetime *st, cplx r, cplx th, cplx g[4][4])
{
    mn_fields F;
    mn_fields_c(st, r, th, &F);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) g[i][j] = 0.0;
    const cplx s2 = F.sin_th * F.sin_th;
    g[0][0] = -F.f;
    g[0][3] = g[3][0] = F.f * F.omega;
    g[1][1] = F.e2gamma * F.rho2 / (F.f * F.Delta);
    g[2][2] = F.e2gamma * F.rho2 / F.f;
    g[3][3] = F.Delta * s2 / F.f - F.f * F.omega * F.omega;
}

/* Inverse metric in the form the listing's metric function writes it:
 *   g^tt = -1/f + f w^2/(Delta sin^2),  g^{t phi} = f w/(Delta sin^2),
 *   g^{phi phi} = f/(Delta sin^2),  g^rr = f Delta/(e^{2g} rho^2),
 *   g^{theta theta} = f/(e^{2g} rho^2). */
static void mn_upper_c(const spacetime *st, cplx r, cplx th, cplx g[4][4])
{
    mn_fields F;
    mn_fields_c(st, r, th, &F);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) g[i][j] = 0.0;
    const cplx ds2 = F.Delta * F.sin_th * F.sin_th;
    g[0][0] = -1.0 / F.f + F.f * F.omega * F.omega / ds2;
    g[1][1] = F.f * F.Delta / (F.e2gamma * F.rho2);
    g[2][2] = F.f / (F.e2gamma * F.rho2);
    g[3][3] = F.f / ds2;
    g[0][3] = g[3][0] = F.f * F.omega / ds2;
}

/* ------------------------------------------------------------------------ */
/* Dispatch: metric, inverse, derivatives                                    */
/* ------------------------------------------------------------------------ */

#define CSTEP_H 1e-30

static void metric_lower(const spacetime *st, double r, double th, double g[4][4])
{
    if (!st->is_mn) {
        kerr_lower(st, r, th, g);
        return;
    }
    cplx gc[4][4];
    mn_lower_c(st, r, th, gc);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) g[i][j] = creal(gc[i][j]);
}

static void metric_upper(const spacetime *st, double r, double th, double g[4][4])
{
    if (!st->is_mn) {
        kerr_upper(st, r, th, g);
        return;
    }
    cplx gc[4][4];
    mn_upper_c(st, r, th, gc);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) g[i][j] = creal(gc[i][j]);
}

/* Complex-step derivatives of the inverse metric, d_mu g^{nu sigma}. */
static void dupper_cstep(const spacetime *st, double r, double th, double dg[4][4][4])
{
    cplx gr[4][4], gt[4][4];
    if (st->is_mn) {
        mn_upper_c(st, r + CSTEP_H * I, th, gr);
        mn_upper_c(st, r, th + CSTEP_H * I, gt);
    } else {
        kerr_upper_c(st, r + CSTEP_H * I, th, gr);
        kerr_upper_c(st, r, th + CSTEP_H * I, gt);
    }
    memset(dg, 0, 64 * sizeof(double));
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            dg[1][i][j] = cimag(gr[i][j]) / CSTEP_H;
            dg[2][i][j] = cimag(gt[i][j]) / CSTEP_H;
        }
}

/* The derivative the integrator uses: closed form for Kerr, complex step
 * for Manko-Novikov. */
static void metric_dupper(const spacetime *st, double r, double th, double dg[4][4][4])
{
    if (!st->is_mn)
        kerr_dupper(st, r, th, dg);
    else
        dupper_cstep(st, r, th, dg);
}

/* ------------------------------------------------------------------------ */
/* Hamiltonian vector field (Eq. hamGeodesic)                                */
/* ------------------------------------------------------------------------ */

/* dq^mu = g^{mu nu} p_nu;  dp_mu = -1/2 d_mu g^{nu sigma} p_nu p_sigma.
 * READING: the 1/2 and the minus sign as in Appendix A (the main-text
 * equation drops the 1/2; the listing keeps both). */
/* Forward differences of the inverse metric as in the listing's propagation kernel:
 * d_r g^{mu nu} ~ (g^{mu nu}(r + delta, theta) - g^{mu nu}(r, theta))/delta and likewise
 * in theta, delta = derPrecision = 1e-8; three metric evaluations (the d_t and d_phi
 * rows are zero for a stationary, axisymmetric metric). */
static void dupper_fd(const spacetime *st, double r, double th, double dg[4][4][4])
{
    double g[4][4], gr[4][4], gt[4][4];
    metric_upper(st, r, th, g);
    metric_upper(st, r + OR_FD_DELTA, th, gr);
    metric_upper(st, r, th + OR_FD_DELTA, gt);
    memset(dg, 0, 64 * sizeof(double));
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            dg[1][i][j] = (gr[i][j] - g[i][j]) / OR_FD_DELTA;
            dg[2][i][j] = (gt[i][j] - g[i][j]) / OR_FD_DELTA;
        }
}

static void vector_field_f(const spacetime *st, const double q[4], const double p[4],
                           double dq[4], double dp[4], int flags)
{
    double g[4][4], dg[4][4][4];
    metric_upper(st, q[1], q[2], g);
    if (flags & OR_FLAG_FD_DERIVS)
        dupper_fd(st, q[1], q[2], dg);
    else
        metric_dupper(st, q[1], q[2], dg);
    for (int mu = 0; mu < 4; mu++) {
        double acc = 0.0;
        for (int nu = 0; nu < 4; nu++)
            for (int sg = 0; sg < 4; sg++) acc += -0.5 * dg[mu][nu][sg] * p[nu] * p[sg];
        dp[mu] = acc;
    }
    for (int mu = 0; mu < 4; mu++) {
        double acc = 0.0;
        for (int nu = 0; nu < 4; nu++) acc += g[mu][nu] * p[nu];
        dq[mu] = acc;
    }
}

static void vector_field(const spacetime *st, const double q[4], const double p[4],
                         double dq[4], double dp[4])
{
    vector_field_f(st, q, p, dq, dp, 0);
}

static double hamiltonian(const spacetime *st, const double q[4], const double p[4])
{
    double g[4][4];
    metric_upper(st, q[1], q[2], g);
    double h = 0.0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++) h += g[mu][nu] * p[mu] * p[nu];
    return 0.5 * h;
}

/* ------------------------------------------------------------------------ */
/* Camera (appendix listing + Sec. 3.3.1)                                     */
/* ------------------------------------------------------------------------ */

/* Initial data of one ray leaving the camera at (0, r0, th0, 0) in the direction
 * (alpha, beta) of the camera's (v^phi sin th0, v^theta) plane (Sec. 3.3.1 and the
 * listing's camera block): v = (v^t, -1, beta, alpha/sin th0), v^t the root
 * (-B + sqrt(B^2 - 4AC))/(2A) of g(v, v) = 0, v rescaled so that v^t = -1 (READING),
 * p_mu = g_{mu nu} v^nu. */
static int camera_dir(const spacetime *st, double r0, double th0, double al, double bt, int flags,
                      double q[4], double p[4])
{
    double v[4];
    v[1] = -1.0;
    v[2] = bt;
    v[3] = (flags & OR_FLAG_COMPAT_CAMERA) ? al : al / sin(th0);
    double g[4][4];
    metric_lower(st, r0, th0, g);
    const double A = g[0][0];
    double B = 0.0, C = 0.0;
    for (int m = 1; m < 4; m++) B += 2.0 * g[0][m] * v[m];
    for (int m = 1; m < 4; m++)
        for (int n = 1; n < 4; n++) C += v[m] * g[m][n] * v[n];
    const double disc = B * B - 4.0 * A * C;
    if (!(A < 0.0) || !(disc >= 0.0)) return OR_ERR_INVALID_ARG;
    const double T = (-B + sqrt(disc)) / (2.0 * A);
    v[0] = T;
    const double scale = 1.0 / fabs(T);
    for (int m = 0; m < 4; m++) v[m] *= scale;
    q[0] = 0.0;
    q[1] = r0;
    q[2] = th0;
    q[3] = 0.0;
    for (int m = 0; m < 4; m++) {
        double acc = 0.0;
        for (int n = 0; n < 4; n++) acc += g[m][n] * v[n];
        p[m] = acc;
    }
    return OR_OK;
}

/* Pixel (i, j) of a resX x resY camera, i in [0, resX) along phi, j in [0, resY)
 * along theta: alpha_i, beta_j the inclusive linspaces over [-H, H] and [-V, V],
 * V = tan(FOV/2)/r0, H = atan(tan(V) resX/resY) (listing's camera block); a single
 * pixel sits at 0 (READING). */
static int camera_ray(const spacetime *st, double r0, double th0, double fov_deg, int resX,
                      int resY, int i, int j, int flags, double q[4], double p[4])
{
    const double V = tan(0.5 * fov_deg / 180.0 * M_PI) / r0;
    const double Hh = atan(tan(V) * (double)resX / (double)resY);
    const double al = resX > 1 ? Hh * (double)(2 * i - (resX - 1)) / (double)(resX - 1) : 0.0;
    const double bt = resY > 1 ? V * (double)(2 * j - (resY - 1)) / (double)(resY - 1) : 0.0;
    return camera_dir(st, r0, th0, al, bt, flags, q, p);
}

/* ------------------------------------------------------------------------ */
/* RK4 propagation (Sec. 3.1.2, listing's propagation kernel)                */
/* ------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------ */
/* Ring and redshift (Sec. 3.3.3; the ring renders of Sec. 5)                */
/* ------------------------------------------------------------------------ */

/* The ring of the renders: a region around the equator of small, non-zero
 * thickness (solid, so that a ray stepping into its volume hits it).  READING:
 * r_in <= r <= r_out and |r cos theta| <= half_thickness. */
typedef struct {
    double r_in, r_out, half_thickness;
} disk_t;

static int in_disk(const disk_t *dk, double r, double th)
{
    return r >= dk->r_in && r <= dk->r_out && fabs(r * cos(th)) <= dk->half_thickness;
}

/* Emitter momentum of the ring at (r, theta) (Sec. 3.3.3): a circular orbit,
 * p_r = p_theta = 0 and dp_r/dtau = 0, with p_t = -1, so that
 *     d_r g^{tt} p_t^2 + 2 d_r g^{t phi} p_t p_phi + d_r g^{phi phi} p_phi^2 = 0
 * (READING: the printed equation has lower indices; the Hamiltonian equation of
 * motion it is derived from has the inverse metric's derivatives).  Of its two
 * roots the one with positive angular velocity u^phi/u^t is taken (the ring turns
 * with +phi, the hole's sense for S > 0; READING), then p is rescaled so that
 * g^{mu nu} p_mu p_nu = -1.  Returns OR_ERR_INVALID_ARG where no timelike circular
 * orbit exists (inside the photon orbit). */
static int circular_orbit(const spacetime *st, double r, double th, int flags, double p[4])
{
    double dg[4][4][4], g[4][4];
    if (flags & OR_FLAG_FD_DERIVS)
        dupper_fd(st, r, th, dg);
    else
        metric_dupper(st, r, th, dg);
    metric_upper(st, r, th, g);
    const double A = dg[1][3][3], B = dg[1][0][3], C = dg[1][0][0];
    /* A p_phi^2 - 2 B p_phi + C = 0 for p_t = -1 */
    const double disc = B * B - A * C;
    if (!(disc >= 0.0) || A == 0.0) return OR_ERR_INVALID_ARG;
    const double roots[2] = {(B + sqrt(disc)) / A, (B - sqrt(disc)) / A};
    for (int k = 0; k < 2; k++) {
        const double pph = roots[k];
        const double ut = -g[0][0] + g[0][3] * pph;
        const double uph = -g[3][0] + g[3][3] * pph;
        const double norm = g[0][0] - 2.0 * g[0][3] * pph + g[3][3] * pph * pph;
        if (ut > 0.0 && uph / ut > 0.0 && norm < 0.0) {
            const double lam = 1.0 / sqrt(-norm);
            p[0] = -lam;
            p[1] = 0.0;
            p[2] = 0.0;
            p[3] = lam * pph;
            return OR_OK;
        }
    }
    return OR_ERR_INVALID_ARG;
}

/* Redshift factor z = lambda_O / lambda_S = (g_{mu nu} kappa_S^mu S^nu) /
 * (g_{mu nu} kappa_O^mu O^nu) (Sec. 3.3.3): kappa the traced (backward) ray,
 * S the ring's 4-velocity at the hit, O the observer's.  READING: the paper makes
 * the denominator 1 through the v^t = -1 normalisation; here O is the static
 * observer at the camera, O = (-g_tt(r0, theta0))^(-1/2) d_t, so the denominator
 * is p_t / sqrt(-g_tt) with p_t conserved along the ray.  NaN where no circular
 * orbit exists. */
static double redshift(const spacetime *st, double r0, double th0, const double q[4],
                       const double p[4], int flags)
{
    double pS[4], g[4][4], gl[4][4];
    if (circular_orbit(st, q[1], q[2], flags, pS) != OR_OK) return NAN;
    metric_upper(st, q[1], q[2], g);
    double num = 0.0;
    for (int mu = 0; mu < 4; mu++) {
        double u = 0.0;
        for (int nu = 0; nu < 4; nu++) u += g[mu][nu] * pS[nu];
        num += p[mu] * u;
    }
    metric_lower(st, r0, th0, gl);
    const double den = p[0] / sqrt(-gl[0][0]);
    return num / den;
}

static int all_finite(const double q[4], const double p[4])
{
    for (int m = 0; m < 4; m++)
        if (!isfinite(q[m]) || !isfinite(p[m])) return 0;
    return 1;
}

typedef struct {
    int status;
    int64_t nsteps;
    double min_sin; /* min |sin theta| over the accepted states */
} ray_result;

/* One ray.  Each iteration: k1 = F(x); h = |sp / k1.q^t|; k2 = F(x + h/2 k1);
 * k3 = F(x + h/2 k2); k4 = F(x + h k3); x += h w (k1 + 2 k2 + 2 k3 + k4) with
 * w = 1/6 (READING; the listing uses 0.1667).  Then, in the listing's order:
 * r > 1.5 r_start -> ESCAPED, else h < sp 3e-5 -> HORIZON.  A step whose result
 * is not finite ends the ray as NONFINITE and keeps the last finite state
 * (READING: the paper has no such test).  nsteps counts the terminal step;
 * a ray that never exits is MAXSTEPS with nsteps = n_steps. */
static void trace_ray(const spacetime *st, double q[4], double p[4], double r_start,
                      int64_t n_steps, double sp, int flags, const disk_t *dk, ray_result *res)
{
    const double w = (flags & OR_FLAG_COMPAT_WEIGHTS) ? 0.1667 : 1.0 / 6.0;
    const double r_escape = 1.5 * r_start;
    double k1q[4], k1p[4], k2q[4], k2p[4], k3q[4], k3p[4], k4q[4], k4p[4];
    double xq[4], xp[4];
    double min_sin = fabs(sin(q[2]));
    for (int64_t i = 0; i < n_steps; i++) {
        vector_field_f(st, q, p, k1q, k1p, flags);
        const double h = fabs(sp / k1q[0]);
        double nq[4], np[4];
        if (flags & OR_FLAG_EULER) { /* Sec. 3.1.1: x += h F(x) */
            for (int m = 0; m < 4; m++) {
                nq[m] = q[m] + h * k1q[m];
                np[m] = p[m] + h * k1p[m];
            }
            goto exits;
        }
        for (int m = 0; m < 4; m++) {
            xq[m] = q[m] + 0.5 * h * k1q[m];
            xp[m] = p[m] + 0.5 * h * k1p[m];
        }
        vector_field_f(st, xq, xp, k2q, k2p, flags);
        for (int m = 0; m < 4; m++) {
            xq[m] = q[m] + 0.5 * h * k2q[m];
            xp[m] = p[m] + 0.5 * h * k2p[m];
        }
        vector_field_f(st, xq, xp, k3q, k3p, flags);
        for (int m = 0; m < 4; m++) {
            xq[m] = q[m] + h * k3q[m];
            xp[m] = p[m] + h * k3p[m];
        }
        vector_field_f(st, xq, xp, k4q, k4p, flags);
        for (int m = 0; m < 4; m++) {
            np[m] = p[m] + h * w * (k1p[m] + 2.0 * k2p[m] + 2.0 * k3p[m] + k4p[m]);
            nq[m] = q[m] + h * w * (k1q[m] + 2.0 * k2q[m] + 2.0 * k3q[m] + k4q[m]);
        }
    exits:
        if (!isfinite(h) || !all_finite(nq, np)) {
            res->status = OR_NONFINITE;
            res->nsteps = i + 1;
            res->min_sin = min_sin;
            return;
        }
        memcpy(q, nq, sizeof nq);
        memcpy(p, np, sizeof np);
        const double sn = fabs(sin(q[2]));
        if (sn < min_sin) min_sin = sn;
        if (q[1] > r_escape) {
            res->status = OR_ESCAPED;
            res->nsteps = i + 1;
            res->min_sin = min_sin;
            return;
        }
        if (dk && in_disk(dk, q[1], q[2])) { /* the ring is tested before the horizon */
            res->status = OR_DISK;
            res->nsteps = i + 1;
            res->min_sin = min_sin;
            return;
        }
        if (h < sp * 0.00003) {
            res->status = OR_HORIZON;
            res->nsteps = i + 1;
            res->min_sin = min_sin;
            return;
        }
    }
    res->status = OR_MAXSTEPS;
    res->nsteps = n_steps;
    res->min_sin = min_sin;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (ctypes)                                            */
/* ------------------------------------------------------------------------ */

int or_metric_lower(double M, double S, double Q, double r, double th, double *g16)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK || !g16) return OR_ERR_INVALID_ARG;
    double g[4][4];
    metric_lower(&st, r, th, g);
    memcpy(g16, g, sizeof g);
    return OR_OK;
}

int or_metric_upper(double M, double S, double Q, double r, double th, double *g16)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK || !g16) return OR_ERR_INVALID_ARG;
    double g[4][4];
    metric_upper(&st, r, th, g);
    memcpy(g16, g, sizeof g);
    return OR_OK;
}

/* d64[mu*16 + nu*4 + sigma] = d_mu g^{nu sigma}; method 0 = the integrator's
 * (closed form for Kerr, complex step for Manko-Novikov), 1 = complex step. */
int or_dmetric_upper(double M, double S, double Q, double r, double th, int method, double *d64)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK || !d64) return OR_ERR_INVALID_ARG;
    double dg[4][4][4];
    if (method == 0)
        metric_dupper(&st, r, th, dg);
    else if (method == 1)
        dupper_cstep(&st, r, th, dg);
    else
        return OR_ERR_INVALID_ARG;
    memcpy(d64, dg, sizeof dg);
    return OR_OK;
}

/* Manko-Novikov scalar functions at real (r, theta):
 * out = {f, omega, e^{2 gamma}, rho^2, Delta, alpha, k, beta}. */
int or_mn_fields(double M, double S, double Q, double r, double th, double *out8)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK || !out8) return OR_ERR_INVALID_ARG;
    if (S == 0.0) return OR_ERR_INVALID_ARG;
    if (!st.is_mn) { /* q = 0 Manko-Novikov: constants from the same formulas */
        double sm = S / M;
        st.alpha = (-M + sqrt(M * M - sm * sm)) / sm;
        st.k = M * (1.0 - st.alpha * st.alpha) / (1.0 + st.alpha * st.alpha);
        st.beta = 0.0;
    }
    mn_fields F;
    mn_fields_c(&st, r, th, &F);
    out8[0] = creal(F.f);
    out8[1] = creal(F.omega);
    out8[2] = creal(F.e2gamma);
    out8[3] = creal(F.rho2);
    out8[4] = creal(F.Delta);
    out8[5] = st.alpha;
    out8[6] = st.k;
    out8[7] = st.beta;
    return OR_OK;
}

/* Manko-Novikov inverse metric even at q = 0 (for the q -> 0 Kerr pin). */
int or_mn_metric_upper(double M, double S, double Q, double r, double th, double *g16)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK || !g16 || S == 0.0) return OR_ERR_INVALID_ARG;
    if (!st.is_mn) {
        double sm = S / M;
        st.alpha = (-M + sqrt(M * M - sm * sm)) / sm;
        st.k = M * (1.0 - st.alpha * st.alpha) / (1.0 + st.alpha * st.alpha);
        st.beta = 0.0;
    }
    cplx gc[4][4];
    mn_upper_c(&st, r, th, gc);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) g16[4 * i + j] = creal(gc[i][j]);
    return OR_OK;
}

int or_mn_metric_lower(double M, double S, double Q, double r, double th, double *g16)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK || !g16 || S == 0.0) return OR_ERR_INVALID_ARG;
    if (!st.is_mn) {
        double sm = S / M;
        st.alpha = (-M + sqrt(M * M - sm * sm)) / sm;
        st.k = M * (1.0 - st.alpha * st.alpha) / (1.0 + st.alpha * st.alpha);
        st.beta = 0.0;
    }
    cplx gc[4][4];
    mn_lower_c(&st, r, th, gc);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) g16[4 * i + j] = creal(gc[i][j]);
    return OR_OK;
}

int or_vector_field(double M, double S, double Q, const double *q4, const double *p4, double *dq4,
                    double *dp4)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK) return OR_ERR_INVALID_ARG;
    vector_field(&st, q4, p4, dq4, dp4);
    return OR_OK;
}

int or_hamiltonian(double M, double S, double Q, const double *q4, const double *p4, double *h)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK) return OR_ERR_INVALID_ARG;
    *h = hamiltonian(&st, q4, p4);
    return OR_OK;
}

static int camera_valid(double r0, double th0, double fov_deg, int resX, int resY)
{
    if (!(r0 > 0.0) || !isfinite(r0)) return 0;
    if (!(th0 > 0.0 && th0 < M_PI)) return 0;
    if (!(fov_deg > 0.0 && fov_deg < 180.0)) return 0;
    if (resX < 1 || resY < 1) return 0;
    return 1;
}

int or_camera_ray(double M, double S, double Q, double r0, double th0, double fov_deg, int resX,
                  int resY, int i, int j, int flags, double *q4, double *p4)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK) return OR_ERR_INVALID_ARG;
    if (!camera_valid(r0, th0, fov_deg, resX, resY)) return OR_ERR_INVALID_ARG;
    if (i < 0 || i >= resX || j < 0 || j >= resY) return OR_ERR_INVALID_ARG;
    return camera_ray(&st, r0, th0, fov_deg, resX, resY, i, j, flags, q4, p4);
}

/* Initial (q, p) of a ray in direction (alpha, beta) from a camera at (r0, th0). */
int or_camera_dir(double M, double S, double Q, double r0, double th0, double al, double bt,
                  int flags, double *q4, double *p4)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK) return OR_ERR_INVALID_ARG;
    if (!(r0 > 0.0) || !isfinite(r0) || !(th0 > 0.0 && th0 < M_PI)) return OR_ERR_INVALID_ARG;
    if (!isfinite(al) || !isfinite(bt)) return OR_ERR_INVALID_ARG;
    return camera_dir(&st, r0, th0, al, bt, flags, q4, p4);
}

/* Integrate one ray from an arbitrary initial state (q, p are overwritten by
 * the end state); r_start sets the escape radius 1.5 r_start. */
int or_trace_ray(double M, double S, double Q, double *q4, double *p4, double r_start,
                 int64_t n_steps, double sp, int flags, int *status, int64_t *nsteps,
                 double *min_sin)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK) return OR_ERR_INVALID_ARG;
    if (n_steps < 0 || !(sp > 0.0)) return OR_ERR_INVALID_ARG;
    ray_result res;
    trace_ray(&st, q4, p4, r_start, n_steps, sp, flags, NULL, &res);
    *status = res.status;
    *nsteps = res.nsteps;
    if (min_sin) *min_sin = res.min_sin;
    return OR_OK;
}

/* Record the whole trajectory (states after each accepted step, up to
 * max_states) for the convergence and conservation pins. */
int or_trace_ray_path(double M, double S, double Q, const double *q4, const double *p4,
                      double r_start, int64_t n_steps, double sp, int flags, double *states8,
                      int64_t max_states, int64_t *n_states)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK) return OR_ERR_INVALID_ARG;
    if (n_steps < 0 || !(sp > 0.0) || max_states < 1) return OR_ERR_INVALID_ARG;
    double q[4], p[4];
    memcpy(q, q4, sizeof q);
    memcpy(p, p4, sizeof p);
    int64_t n = 0;
    memcpy(states8, q, sizeof q);
    memcpy(states8 + 4, p, sizeof p);
    n = 1;
    for (int64_t i = 0; i < n_steps && n < max_states; i++) {
        ray_result res;
        trace_ray(&st, q, p, r_start, 1, sp, flags, NULL, &res);
        if (res.status == OR_NONFINITE) break;
        memcpy(states8 + 8 * n, q, sizeof q);
        memcpy(states8 + 8 * n + 4, p, sizeof p);
        n++;
        if (res.status != OR_MAXSTEPS) break;
    }
    *n_states = n;
    return OR_OK;
}

typedef struct {
    const spacetime *st;
    double r0, th0, fov;
    int resX, resY;
    int64_t n_steps;
    double sp;
    int flags;
    const int64_t *pixels;
    int64_t n;
    int64_t next; /* shared work counter */
    double *t, *r, *th, *ph;
    uint8_t *status;
    uint32_t *nsteps;
    double *p_out;   /* optional, 4 per ray */
    double *min_sin; /* optional */
    int err;
    const disk_t *dk; /* optional ring */
    double *z;        /* redshift per ray with the ring (NaN where it was not hit) */
} image_job;

/* float32 rounding of the listing's kernel arguments and outputs (OR_FLAG_F32_IO) */
static double f32(double v) { return (double)(float)v; }

static void *image_worker(void *arg)
{
    image_job *job = (image_job *)arg;
    for (;;) {
        const int64_t k = __atomic_fetch_add(&job->next, 1, __ATOMIC_RELAXED);
        if (k >= job->n) break;
        const int64_t pix = job->pixels ? job->pixels[k] : k;
        const int i = (int)(pix % job->resX), j = (int)(pix / job->resX);
        double q[4], p[4];
        if (camera_ray(job->st, job->r0, job->th0, job->fov, job->resX, job->resY, i, j, job->flags,
                       q, p) != OR_OK) {
            __atomic_store_n(&job->err, 1, __ATOMIC_RELAXED);
            continue;
        }
        if (job->flags & OR_FLAG_F32_IO)
            for (int m = 0; m < 4; m++) {
                q[m] = f32(q[m]);
                p[m] = f32(p[m]);
            }
        ray_result res;
        trace_ray(job->st, q, p, job->r0, job->n_steps, job->sp, job->flags, job->dk, &res);
        if (job->z)
            job->z[k] = res.status == OR_DISK ? redshift(job->st, job->r0, job->th0, q, p, job->flags)
                                              : NAN;
        if (job->flags & OR_FLAG_F32_IO)
            for (int m = 0; m < 4; m++) q[m] = f32(q[m]);
        job->t[k] = q[0];
        job->r[k] = q[1];
        job->th[k] = q[2];
        job->ph[k] = q[3];
        job->status[k] = (uint8_t)res.status;
        job->nsteps[k] = (uint32_t)res.nsteps;
        if (job->p_out) memcpy(job->p_out + 4 * k, p, sizeof p);
        if (job->min_sin) job->min_sin[k] = res.min_sin;
    }
    return NULL;
}

/* Trace the camera's pixels (all of them when pixels == NULL, else the listed
 * flat indices j*resX + i) on n_threads POSIX threads.  Output k belongs to
 * the k-th traced pixel. */
static int trace_image(double M, double S, double Q, double r0, double th0, double fov_deg,
                       int resX, int resY, int64_t n_steps, double sp, int flags,
                       const int64_t *pixels, int64_t n_pixels, int n_threads, double *t,
                       double *r, double *th, double *ph, uint8_t *status, uint32_t *nsteps,
                       double *p_out, double *min_sin, const disk_t *dk, double *z)
{
    spacetime st;
    if (flags & OR_FLAG_F32_IO) { /* the listing passes M, S, q as float32 */
        M = f32(M);
        S = f32(S);
        Q = f32(Q);
    }
    if (spacetime_init(&st, M, S, Q) != OR_OK) return OR_ERR_INVALID_ARG;
    if (!camera_valid(r0, th0, fov_deg, resX, resY)) return OR_ERR_INVALID_ARG;
    if (n_steps < 0 || n_steps > 0xffffffffLL || !(sp > 0.0)) return OR_ERR_INVALID_ARG;
    const int64_t total = (int64_t)resX * (int64_t)resY;
    const int64_t n = pixels ? n_pixels : total;
    if (n < 0) return OR_ERR_INVALID_ARG;
    if (pixels)
        for (int64_t k = 0; k < n; k++)
            if (pixels[k] < 0 || pixels[k] >= total) return OR_ERR_INVALID_ARG;
    if (n == 0) return OR_OK;
    if (!t || !r || !th || !ph || !status || !nsteps) return OR_ERR_INVALID_ARG;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 1024) n_threads = 1024;
    image_job job = {&st,   r0,    th0,     fov_deg, resX, resY, n_steps, sp,  flags,
                     pixels, n,    0,       t,       r,    th,   ph,      status, nsteps,
                     p_out, min_sin, 0, dk, z};
    pthread_t *tids = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    if (!tids) return OR_ERR_INVALID_ARG;
    int started = 0;
    for (int k = 0; k < n_threads; k++) {
        if (pthread_create(&tids[k], NULL, image_worker, &job) != 0) break;
        started++;
    }
    if (started == 0) image_worker(&job);
    for (int k = 0; k < started; k++) pthread_join(tids[k], NULL);
    free(tids);
    return job.err ? OR_ERR_INVALID_ARG : OR_OK;
}

int or_trace_image(double M, double S, double Q, double r0, double th0, double fov_deg, int resX,
                   int resY, int64_t n_steps, double sp, int flags, const int64_t *pixels,
                   int64_t n_pixels, int n_threads, double *t, double *r, double *th, double *ph,
                   uint8_t *status, uint32_t *nsteps, double *p_out, double *min_sin)
{
    return trace_image(M, S, Q, r0, th0, fov_deg, resX, resY, n_steps, sp, flags, pixels,
                       n_pixels, n_threads, t, r, th, ph, status, nsteps, p_out, min_sin, NULL,
                       NULL);
}

/* As or_trace_image with the ring r_in <= r <= r_out, |r cos theta| <= half_thickness
 * as an exit (status 5, tested after the escape and before the horizon) and the
 * redshift factor of each ray that hit it in z (NaN otherwise). */
int or_trace_image_disk(double M, double S, double Q, double r0, double th0, double fov_deg,
                        int resX, int resY, int64_t n_steps, double sp, int flags, double r_in,
                        double r_out, double half_thickness, const int64_t *pixels,
                        int64_t n_pixels, int n_threads, double *t, double *r, double *th,
                        double *ph, uint8_t *status, uint32_t *nsteps, double *z)
{
    if (!(r_in > 0.0) || !(r_out > r_in) || !(half_thickness > 0.0) || !z) return OR_ERR_INVALID_ARG;
    const disk_t dk = {r_in, r_out, half_thickness};
    return trace_image(M, S, Q, r0, th0, fov_deg, resX, resY, n_steps, sp, flags, pixels,
                       n_pixels, n_threads, t, r, th, ph, status, nsteps, NULL, NULL, &dk, z);
}

/* Ring emitter momentum (p_t, p_r, p_theta, p_phi) at (r, theta). */
int or_circular_orbit(double M, double S, double Q, double r, double th, int flags, double *p4)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK || !p4) return OR_ERR_INVALID_ARG;
    return circular_orbit(&st, r, th, flags, p4);
}

/* Redshift factor of a ray with momentum p4 at position q4 against a static observer
 * at (r0, th0). */
int or_redshift(double M, double S, double Q, double r0, double th0, const double *q4,
                const double *p4, int flags, double *z)
{
    spacetime st;
    if (spacetime_init(&st, M, S, Q) != OR_OK || !q4 || !p4 || !z) return OR_ERR_INVALID_ARG;
    *z = redshift(&st, r0, th0, q4, p4, flags);
    return OR_OK;
}
