// spacetime.cuh -- device-side spacetimes for the geodesic integrator (sm_103a).
//
// For a stationary, axisymmetric metric g^{mu nu}(r, theta) the Hamiltonian of
// Eq. hamGeodesic is H = 1/2 g^{mu nu} p_mu p_nu, with p_t and p_phi constants of
// motion.  Rather than the paper's 4x4x4 contraction of finite-difference
// derivatives (appendix listing), each spacetime here writes H in closed form and
// differentiates it exactly:
//
//   Kerr (Sec. 2.2.2), with Sigma = r^2 + a^2 cos^2, Delta = r^2 - 2Mr + a^2:
//     2 Sigma H = K = Delta p_r^2 + p_theta^2 + V^2 - W^2/Delta,
//     W = (r^2 + a^2) p_t + a p_phi,   V = p_phi/sin + a sin p_t,
//   and dq/dtau = dH/dp, dp_r/dtau = -dH/dr, dp_theta/dtau = -dH/dtheta by hand.
//
//   Manko-Novikov (Sec. 2.2.3): the inverse metric of its line element is
//     2H = -p_t^2/f + F (p_phi + w p_t)^2 + G (Delta p_r^2 + p_theta^2),
//     F = f/(Delta sin^2),  G = g^{theta theta} = (1-alpha^2)^2/k^2 exp(2psi - 2gamma'')/B,
//   (gamma'' = gamma' without its logarithm, which cancels against e^{2gamma}'s
//   (x^2-1) factor); the kernels take its r and theta derivatives by a reverse
//   (adjoint) sweep over the same expressions (mn_rates), and a forward-mode form with
//   dual numbers (value, d/dr, d/dtheta) is kept as the reference it is checked
//   against (mn_rates_fwd).
//
// Both are written once over a scalar type T so the FP32-mixed path can reuse them.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#ifndef GT_HD
#define GT_HD __host__ __device__ __forceinline__
#endif

namespace gt {

enum : int { KIND_KERR = 0, KIND_MN = 1 };

// Derived constants of one spacetime (computed on the device by the setup kernel),
// in the working precision T of the field evaluation.
template <class T>
struct SpacetimeT {
    int kind;
    T M, a, a2;           // Kerr: a = S/M
    T r_plus;             // outer horizon (Kerr M + sqrt(M^2 - a^2); MN M + k)
    T k, ik, alpha, beta; // Manko-Novikov
    T two_beta, three_beta2;
    T c_g;                // (1 - alpha^2)^2 / k^2
    T w_inf;              // 4 k alpha / (1 - alpha^2)
    T k2, inv_k2, two_k;
};
using SpacetimeC = SpacetimeT<double>;
using SpacetimeF = SpacetimeT<float>;

// Rounded copy for the FP32 path (done once per ray, not per field evaluation).
template <class T>
GT_HD SpacetimeF to_float(const SpacetimeT<T> &c)
{
    SpacetimeF f;
    f.kind = c.kind;
    f.M = (float)c.M;
    f.a = (float)c.a;
    f.a2 = (float)c.a2;
    f.r_plus = (float)c.r_plus;
    f.k = (float)c.k;
    f.ik = (float)c.ik;
    f.alpha = (float)c.alpha;
    f.beta = (float)c.beta;
    f.two_beta = (float)c.two_beta;
    f.three_beta2 = (float)c.three_beta2;
    f.c_g = (float)c.c_g;
    f.w_inf = (float)c.w_inf;
    f.k2 = (float)c.k2;
    f.inv_k2 = (float)c.inv_k2;
    f.two_k = (float)c.two_k;
    return f;
}

template <class T>
struct Rates {
    T dt, dr, dth, dph, dpr, dpth;
};

// ------------------------------------------------------------------ math helpers
// (device-only; a host-side counting type supplies its own overloads)
#ifdef __CUDACC__
__device__ __forceinline__ void sincos_t(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_t(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float exp_t(float x) { return __expf(x); } // FP32 path: fast
// reciprocal: IEEE in FP64 (the parity path), the fast hardware approximation in FP32
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp_t(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
#endif

// ------------------------------------------------------------------ dual numbers
// (value, d/dr, d/dtheta)
template <class T>
struct D3 {
    T v, r, t;
};

template <class T>
GT_HD D3<T> dc(T v) { return {v, T(0), T(0)}; }
template <class T>
GT_HD D3<T> operator+(D3<T> a, D3<T> b) { return {a.v + b.v, a.r + b.r, a.t + b.t}; }
template <class T>
GT_HD D3<T> operator-(D3<T> a, D3<T> b) { return {a.v - b.v, a.r - b.r, a.t - b.t}; }
template <class T>
GT_HD D3<T> operator-(D3<T> a) { return {-a.v, -a.r, -a.t}; }
template <class T>
GT_HD D3<T> operator+(D3<T> a, T c) { return {a.v + c, a.r, a.t}; }
template <class T>
GT_HD D3<T> operator+(T c, D3<T> a) { return {a.v + c, a.r, a.t}; }
template <class T>
GT_HD D3<T> operator-(D3<T> a, T c) { return {a.v - c, a.r, a.t}; }
template <class T>
GT_HD D3<T> operator-(T c, D3<T> a) { return {c - a.v, -a.r, -a.t}; }
template <class T>
GT_HD D3<T> operator*(D3<T> a, T c) { return {a.v * c, a.r * c, a.t * c}; }
template <class T>
GT_HD D3<T> operator*(T c, D3<T> a) { return {a.v * c, a.r * c, a.t * c}; }
template <class T>
GT_HD D3<T> operator*(D3<T> a, D3<T> b)
{
    return {a.v * b.v, fma_t(a.r, b.v, a.v * b.r), fma_t(a.t, b.v, a.v * b.t)};
}
template <class T>
GT_HD D3<T> dsq(D3<T> a)
{
    const T tv = a.v + a.v;
    return {a.v * a.v, tv * a.r, tv * a.t};
}
template <class T>
GT_HD D3<T> drcp(D3<T> a)
{
    const T iv = rcp_t(a.v);
    const T w = -iv * iv;
    return {iv, a.r * w, a.t * w};
}
template <class T>
GT_HD D3<T> drsqrt(D3<T> a)
{
    const T rs = rsqrt_t(a.v);
    const T w = T(-0.5) * rs * rs * rs;
    return {rs, a.r * w, a.t * w};
}
template <class T>
GT_HD D3<T> dexp(D3<T> a)
{
    const T e = exp_t(a.v);
    return {e, a.r * e, a.t * e};
}

// Value-only stand-in with the dual numbers' interface: the same formulas evaluate
// the metric functions without their derivatives (camera set-up, H re-projection).
template <class T>
struct V1 {
    T v;
};
template <class T>
GT_HD V1<T> operator+(V1<T> a, V1<T> b) { return {a.v + b.v}; }
template <class T>
GT_HD V1<T> operator-(V1<T> a, V1<T> b) { return {a.v - b.v}; }
template <class T>
GT_HD V1<T> operator-(V1<T> a) { return {-a.v}; }
template <class T>
GT_HD V1<T> operator+(V1<T> a, T c) { return {a.v + c}; }
template <class T>
GT_HD V1<T> operator+(T c, V1<T> a) { return {a.v + c}; }
template <class T>
GT_HD V1<T> operator-(V1<T> a, T c) { return {a.v - c}; }
template <class T>
GT_HD V1<T> operator-(T c, V1<T> a) { return {c - a.v}; }
template <class T>
GT_HD V1<T> operator*(V1<T> a, T c) { return {a.v * c}; }
template <class T>
GT_HD V1<T> operator*(T c, V1<T> a) { return {a.v * c}; }
template <class T>
GT_HD V1<T> operator*(V1<T> a, V1<T> b) { return {a.v * b.v}; }
template <class T>
GT_HD V1<T> dsq(V1<T> a) { return {a.v * a.v}; }
template <class T>
GT_HD V1<T> drcp(V1<T> a) { return {rcp_t(a.v)}; }
template <class T>
GT_HD V1<T> drsqrt(V1<T> a) { return {rsqrt_t(a.v)}; }
template <class T>
GT_HD V1<T> dexp(V1<T> a) { return {exp_t(a.v)}; }

// variable constructors: f(r) with d/dr = dr, and f(theta) with d/dtheta = dt
template <class T>
GT_HD void mkvar(D3<T> &o, T v, T dr, T dt) { o = {v, dr, dt}; }
template <class T>
GT_HD void mkvar(V1<T> &o, T v, T, T) { o = {v}; }

// ------------------------------------------------------------------ Kerr
// The rate functions take theta through s = sin(theta) and cs = cos(theta) (the *_sc
// forms), so that a caller that already has them -- the FP32 RK4 step rotates the first
// stage's pair to the later stages -- need not evaluate them again.
template <class T>
GT_HD void kerr_rates_sc(const SpacetimeT<T> &c, T r, T s, T cs, T pr, T pth, T pt, T pph,
                         Rates<T> &o)
{
    const T a = T(c.a), a2 = T(c.a2), M = T(c.M);
    const T r2 = r * r, ra2 = r2 + a2;
    const T s2 = s * s;
    const T Sigma = fma_t(a2, cs * cs, r2);
    const T Delta = fma_t(r, r - T(2) * M, a2);
    const T inv = rcp_t(Sigma * Delta * s2); // one reciprocal for 1/Sigma, 1/Delta, 1/sin^2
    const T iSigma = Delta * s2 * inv;
    const T iDelta = Sigma * s2 * inv;
    const T is2 = Sigma * Delta * inv;
    const T is = s * is2;
    const T W = fma_t(ra2, pt, a * pph);
    const T V = fma_t(pph, is, a * s * pt);
    const T WiD = W * iDelta;
    const T K = fma_t(Delta * pr, pr, fma_t(pth, pth, fma_t(V, V, -W * WiD)));
    o.dr = Delta * pr * iSigma;
    o.dth = pth * iSigma;
    o.dt = (a * V * s - ra2 * WiD) * iSigma;
    o.dph = (V * is - a * WiD) * iSigma;
    const T Kr = T(2) * (r - M) * fma_t(pr, pr, WiD * WiD) - T(4) * r * pt * WiD;
    const T Kth = T(2) * V * cs * (a * pt - pph * is2);
    const T KiS = K * iSigma;
    o.dpr = T(-0.5) * (Kr - T(2) * r * KiS) * iSigma;
    o.dpth = T(-0.5) * fma_t(T(2) * a2 * s * cs, KiS, Kth) * iSigma;
}

template <class T>
GT_HD void kerr_rates(const SpacetimeT<T> &c, T r, T th, T pr, T pth, T pt, T pph, Rates<T> &o)
{
    T s, cs;
    sincos_t(th, &s, &cs);
    kerr_rates_sc<T>(c, r, s, cs, pr, pth, pt, pph, o);
}

#ifdef __CUDACC__
// Inverse-metric components (tt, t phi, phi phi, rr, theta theta) of Kerr.
__device__ __forceinline__ void kerr_upper(const SpacetimeC &c, double r, double th, double g[5])
{
    double s, cs;
    sincos(th, &s, &cs);
    const double a = c.a, a2 = c.a2, M = c.M;
    const double s2 = s * s, ra2 = r * r + a2;
    const double Sigma = r * r + a2 * cs * cs;
    const double Delta = r * r - 2.0 * M * r + a2;
    const double D = Sigma * Delta;
    g[0] = -(ra2 * ra2 - a2 * Delta * s2) / D;
    g[1] = -2.0 * M * a * r / D;
    g[2] = (Delta - a2 * s2) / (D * s2);
    g[3] = Delta / Sigma;
    g[4] = 1.0 / Sigma;
}
#endif

// ------------------------------------------------------------------ Manko-Novikov
template <class N>
struct MNPot {
    N invf, F, om, G, Delta;
};

// N = D3<T> (values and r, theta derivatives) or V1<T> (values only).
template <class T, class N>
GT_HD void mn_potentials(const SpacetimeT<T> &c, T r, T th, MNPot<N> &P)
{
    T s, cs;
    sincos_t(th, &s, &cs);
    const T ik = T(c.ik);
    const T two_beta = T(c.two_beta);
    N x, xm1, y, s2;
    mkvar(x, (r - T(c.M)) * ik, ik, T(0));
    mkvar(xm1, (r - T(c.r_plus)) * ik, ik, T(0)); // x - 1 without cancellation
    mkvar(y, cs, T(0), -s);
    mkvar(s2, s * s, T(0), T(2) * s * cs); // 1 - y^2
    const N xp1 = x + T(1);
    const N x2m1 = xm1 * xp1;
    const N R2 = x2m1 + dsq(y); // x^2 + y^2 - 1
    const N iR = drsqrt(R2);
    const N u = x * y * iR; // Legendre argument x y / R
    const N u2 = dsq(u);
    const N P2 = u2 * T(1.5) - T(0.5);
    const N P3 = u * (u2 * T(2.5) - T(1.5));
    const N iR2 = dsq(iR);
    const N iR3 = iR2 * iR;
    const N uR2 = u * iR2, P2R3 = P2 * iR3;
    // sum_l (+-1) P_l / R^{l+1} with the sign patterns of fraktur a, fraktur b, gamma'
    const N Sa = (x - y) * (iR + uR2 + P2R3);
    const N Sb = (x + y) * (uR2 - iR - P2R3);
    const N Sg = T(2) * (x * iR - y * uR2 + x * P2R3);
    const N fa = dexp((Sa - T(1)) * (-two_beta)) * T(-c.alpha);
    const N fb = dexp((Sb + T(1)) * two_beta) * T(c.alpha);
    const N ab = fa * fb;
    const N opab = ab + T(1);
    const N bma = fb - fa;
    const N A = x2m1 * dsq(opab) - s2 * dsq(bma);
    const N B = dsq(xp1 + xm1 * ab) + dsq((y + T(1)) * fa + (T(1) - y) * fb);
    const N C = x2m1 * opab * (bma - y * (fa + fb)) + s2 * bma * (opab + x * (T(1) - ab));
    const N psi2 = P2R3 * two_beta;                                            // 2 psi
    const N g2 = T(c.three_beta2) * dsq(iR3) * (dsq(P3) - dsq(P2)) + (Sg - T(2)) * two_beta; // 2 gamma''
    const N e2psi = dexp(psi2);
    const N ie2psi = drcp(e2psi);
    const N iA = drcp(A);
    const N iB = drcp(B);
    P.invf = ie2psi * B * iA;
    P.F = e2psi * A * iB * drcp(x2m1 * s2) * T(c.inv_k2);
    P.om = ie2psi * C * iA * T(c.two_k) - T(c.w_inf);
    P.G = dexp(psi2 - g2) * iB * T(c.c_g);
    P.Delta = x2m1 * T(c.k2);
}

// Rates of Manko-Novikov by reverse-mode differentiation: one forward sweep of values
// through the same expressions as mn_potentials, then one backward sweep of adjoints
// (xb = d(2H)/dx for each intermediate x) from 2H down to r and theta.  Exact to
// rounding like the dual-number form below (mn_rates_fwd), with less than half its
// arithmetic: a product costs one multiply forward and two fused multiply-adds backward
// instead of five operations for a value and two derivatives.
// ex (optional) receives the four exponents of the evaluation, -2 beta Ea, 2 beta Eb,
// 2 psi and 2 psi - 2 gamma'': the double-float evaluation checks its range with them.
template <class T, bool TAIL = false>
GT_HD void mn_rates_sc(const SpacetimeT<T> &c, T r, T s, T cs, T pr, T pth, T pt, T pph,
                       Rates<T> &o, T *ex = nullptr)
{
    // ---- forward sweep (values)
    const T ik = T(c.ik), tb = T(c.two_beta), al = T(c.alpha);
    const T x = (r - T(c.M)) * ik;
    const T xm1 = (r - T(c.r_plus)) * ik; // x - 1 without cancellation
    const T y = cs, s2 = s * s;
    const T xp1 = x + T(1);
    const T x2m1 = xm1 * xp1;
    const T R2 = fma_t(y, y, x2m1);
    const T iR = rsqrt_t(R2);
    const T xy = x * y;
    const T u = xy * iR;
    const T u2 = u * u;
    const T P2 = fma_t(T(1.5), u2, T(-0.5));
    const T q3 = fma_t(T(2.5), u2, T(-1.5));
    const T P3 = u * q3;
    const T iR2 = iR * iR;
    const T iR3 = iR2 * iR;
    const T P2R3 = P2 * iR3;
    const T xmy = x - y, xpy = x + y;
    // Ea = Sa - 1, Eb = Sb + 1, Eg = Sg - 2, where Sa, Sb, Sg are the l <= 2 multipole
    // sums of the metric (Sa = (x - y) sum_l P_l(u)/R^(l+1), Sb = -(x + y) sum_l (-1)^l
    // P_l(u)/R^(l+1), Sg = Sa - Sb).  The full series sum to 1/(x - y) and 1/(x + y) (the
    // Legendre generating function with t = 1/R, u R = x y), so Ea and Eb are series tails,
    // small far out, and the direct differences lose about 2 beta ulp(1) in the exponents.
    // TAIL (FP32 kernels on request) writes the tails in closed form, without cancellation:
    //   Ea = -t^3 N(t) / (1 + sa Q(t)),  sa = (x - y) t,  Q(t) = 1 + u t + P2 t^2,
    //   Eb = -t^3 N(-t) / (1 + sb Q(-t)), sb = (x + y) t,
    //   N(t) = 2 P3 - c4 t - c5 t^2 - c6 t^3,
    //   c4 = P2^2 - 4 u^2 P2 + 2 P2 + u^2,  c5 = 2 u P2 (1 - P2),  c6 = P2^2,
    //   Eg = Ea - Eb;
    // at the price of ~45 more operations per evaluation.  FP64 keeps the direct
    // differences (their error there is ~1e-12), and so does the default FP32 path, whose
    // end states stay within the mixed-precision criteria regardless.
    T Ea, Eb, Eg;
    T uR2 = T(0), T1 = T(0), T2 = T(0), iRP = T(0);           // direct form
    T c4 = T(0), c5 = T(0), c6 = T(0), tw1 = T(0), tw2 = T(0);  // tail form
    T tv1 = T(0), tv2 = T(0), Nn = T(0), Np = T(0), sa = T(0), sb = T(0);
    T q1 = T(0), q2 = T(0), Qa = T(0), Qb = T(0), ia = T(0), ib = T(0);
    if constexpr (TAIL) {
        c4 = fma_t(P2, P2 - T(4) * u2 + T(2), u2);
        c5 = T(2) * u * (P2 - P2 * P2);
        c6 = P2 * P2;
        tw1 = fma_t(iR, c6, c5);  // c5 + t c6
        tw2 = fma_t(iR, tw1, c4); // c4 + t tw1
        Nn = fma_t(-iR, tw2, T(2) * P3);
        tv1 = fma_t(-iR, c6, c5); // c5 - t c6
        tv2 = fma_t(-iR, tv1, c4); // c4 - t tv1
        Np = fma_t(iR, tv2, T(2) * P3);
        sa = xmy * iR;
        sb = xpy * iR;
        q1 = fma_t(P2, iR, u);   // u + P2 t
        q2 = fma_t(-P2, iR, u);  // u - P2 t
        Qa = fma_t(iR, q1, T(1));
        Qb = fma_t(-iR, q2, T(1));
        ia = rcp_t(fma_t(sa, Qa, T(1)));
        ib = rcp_t(fma_t(sb, Qb, T(1)));
        Ea = -iR3 * Nn * ia;
        Eb = -iR3 * Np * ib;
        Eg = Ea - Eb;
    } else {
        uR2 = u * iR2;
        T1 = iR + uR2 + P2R3;
        T2 = uR2 - iR - P2R3;
        iRP = iR + P2R3;
        Ea = xmy * T1 - T(1);
        Eb = xpy * T2 + T(1);
        Eg = T(2) * (x * iRP - y * uR2) - T(2);
    }
    const T xa = Ea * (-tb), xb = Eb * tb;
    const T fa = exp_t(xa) * (-al);
    const T fb = exp_t(xb) * al;
    const T ab = fa * fb;
    const T opab = ab + T(1);
    const T bma = fb - fa;
    const T A = x2m1 * (opab * opab) - s2 * (bma * bma);
    const T yp1 = y + T(1), omy = T(1) - y;
    const T Bq1 = fma_t(xm1, ab, xp1);
    const T Bq2 = yp1 * fa + omy * fb;
    const T B = Bq1 * Bq1 + Bq2 * Bq2;
    const T fsum = fa + fb, omab = T(1) - ab;
    const T C1 = bma - y * fsum;
    const T C2 = fma_t(x, omab, opab);
    const T c1 = x2m1 * opab, c2 = s2 * bma;
    const T C = c1 * C1 + c2 * C2;
    const T psi2 = tb * P2R3;
    const T D = P3 * P3 - P2 * P2;
    const T t3 = T(c.three_beta2) * (iR3 * iR3);
    const T g2 = fma_t(t3, D, Eg * tb);
    const T e2psi = exp_t(psi2);
    const T ie2psi = rcp_t(e2psi);
    const T iA = rcp_t(A);
    const T iB = rcp_t(B);
    const T v1 = ie2psi * B;
    const T invf = v1 * iA;
    const T xs = x2m1 * s2;
    const T ixs = rcp_t(xs);
    const T pA = A * iB;
    const T pB = pA * ixs;
    const T W = pB * T(c.inv_k2);
    const T F = e2psi * W;
    const T ieC = ie2psi * C;
    const T om0 = ieC * iA;
    const T om = om0 * T(c.two_k) - T(c.w_inf);
    const T xg = psi2 - g2;
    const T eG = exp_t(xg);
    if (ex) {
        ex[0] = xa;
        ex[1] = xb;
        ex[2] = psi2;
        ex[3] = xg;
    }
    const T iBc = iB * T(c.c_g);
    const T G = eG * iBc;
    const T Delta = x2m1 * T(c.k2);
    const T pw = fma_t(om, pt, pph);
    const T pr2 = pr * pr;
    const T Q = fma_t(Delta, pr2, pth * pth);
    const T Fpw = F * pw;
    o.dt = fma_t(Fpw, om, -pt * invf);
    o.dph = Fpw;
    o.dr = G * Delta * pr;
    o.dth = G * pth;

    // ---- backward sweep: adjoints of 2H = -pt^2 invf + F pw^2 + G Q
    const T invf_b = -pt * pt;
    const T F_b = pw * pw;
    const T om0_b = T(2) * Fpw * pt * T(c.two_k); // through pw = om pt + pph
    const T G_b = Q;
    const T Delta_b = G * pr2;
    // G = eG iB c_g, eG = exp(psi2 - g2)
    const T eG_b = G_b * iBc;
    const T dG = eG_b * eG;
    T psi2_b = dG;
    const T g2_b = -dG;
    T iB_b = G_b * eG * T(c.c_g);
    // om0 = ie2psi C iA
    T ie2psi_b = om0_b * C * iA;
    T C_b = om0_b * ie2psi * iA;
    T iA_b = om0_b * ieC;
    // F = e2psi pB inv_k2, pB = A iB ixs
    T e2psi_b = F_b * W;
    const T pB_b = F_b * e2psi * T(c.inv_k2);
    const T pA_b = pB_b * ixs;
    const T ixs_b = pB_b * pA;
    T A_b = pA_b * iB;
    iB_b = fma_t(pA_b, A, iB_b);
    // invf = ie2psi B iA
    const T v1_b = invf_b * iA;
    iA_b = fma_t(invf_b, v1, iA_b);
    ie2psi_b = fma_t(v1_b, B, ie2psi_b);
    T B_b = v1_b * ie2psi;
    // reciprocals and the exponential of psi
    const T xs_b = -ixs_b * ixs * ixs;
    T x2m1_b = fma_t(Delta_b, T(c.k2), xs_b * s2);
    T s2_b = xs_b * x2m1;
    B_b = fma_t(-iB_b * iB, iB, B_b);
    A_b = fma_t(-iA_b * iA, iA, A_b);
    e2psi_b = fma_t(-ie2psi_b * ie2psi, ie2psi, e2psi_b);
    psi2_b = fma_t(e2psi_b, e2psi, psi2_b);
    // g2 = t3 D + tb (Sg - 2), t3 = 3 beta^2 iR3^2
    const T D_b = g2_b * t3;
    T iR3_b = g2_b * D * T(c.three_beta2) * T(2) * iR3;
    const T Eg_b = g2_b * tb;
    T P3_b = T(2) * P3 * D_b;
    T P2_b = T(-2) * P2 * D_b;
    T P2R3_b = tb * psi2_b;
    // C = c1 C1 + c2 C2
    const T C1_b = C_b * c1, C2_b = C_b * c2;
    const T c1_b = C_b * C1, c2_b = C_b * C2;
    x2m1_b = fma_t(c1_b, opab, x2m1_b);
    T opab_b = c1_b * x2m1 + C2_b;
    s2_b = fma_t(c2_b, bma, s2_b);
    T bma_b = fma_t(c2_b, s2, C1_b);
    T x_b = C2_b * omab;
    T ab_b = -C2_b * x;
    T y_b = -C1_b * fsum;
    T fa_b = -C1_b * y;
    T fb_b = fa_b;
    // B = Bq1^2 + Bq2^2
    const T Bq1_b = T(2) * Bq1 * B_b, Bq2_b = T(2) * Bq2 * B_b;
    y_b = fma_t(Bq2_b, fa - fb, y_b);
    fa_b = fma_t(Bq2_b, yp1, fa_b);
    fb_b = fma_t(Bq2_b, omy, fb_b);
    T xp1_b = Bq1_b;
    T xm1_b = Bq1_b * ab;
    ab_b = fma_t(Bq1_b, xm1, ab_b);
    // A = x2m1 opab^2 - s2 bma^2
    x2m1_b = fma_t(A_b, opab * opab, x2m1_b);
    opab_b = fma_t(A_b * x2m1, T(2) * opab, opab_b);
    s2_b = fma_t(-A_b, bma * bma, s2_b);
    bma_b = fma_t(-A_b * s2, T(2) * bma, bma_b);
    // bma = fb - fa, opab = ab + 1, ab = fa fb
    fb_b = fb_b + bma_b;
    fa_b = fa_b - bma_b;
    ab_b = ab_b + opab_b;
    fa_b = fma_t(ab_b, fb, fa_b);
    fb_b = fma_t(ab_b, fa, fb_b);
    // fa = -alpha exp(-2 beta Ea), fb = alpha exp(2 beta Eb)
    T Ea_b = -fa_b * fa * tb;
    T Eb_b = fb_b * fb * tb;
    T iR_b, u_b, iR2_b;
    if constexpr (TAIL) {
        // Eg = Ea - Eb
        Ea_b = Ea_b + Eg_b;
        Eb_b = Eb_b - Eg_b;
        // Ea = -iR3 Nn ia, ia = 1 / (1 + sa Qa); Eb likewise
        iR3_b = iR3_b - (Nn * ia * Ea_b + Np * ib * Eb_b);
        const T Nn_b = -iR3 * ia * Ea_b, Np_b = -iR3 * ib * Eb_b;
        const T Da_b = -Ea * ia * Ea_b, Db_b = -Eb * ib * Eb_b;
        const T sa_b = Da_b * Qa, Qa_b = Da_b * sa;
        const T sb_b = Db_b * Qb, Qb_b = Db_b * sb;
        // sa = (x - y) t, sb = (x + y) t, t = iR
        x_b = fma_t(iR, sa_b + sb_b, x_b);
        y_b = fma_t(iR, sb_b - sa_b, y_b);
        iR_b = fma_t(xmy, sa_b, xpy * sb_b);
        // Qa = 1 + t q1, q1 = u + P2 t;  Qb = 1 - t q2, q2 = u - P2 t
        const T q1_b = iR * Qa_b, q2_b = -iR * Qb_b;
        iR_b = iR_b + q1 * Qa_b - q2 * Qb_b + P2 * (q1_b - q2_b);
        u_b = q1_b + q2_b;
        P2_b = fma_t(iR, q1_b - q2_b, P2_b);
        // Nn = 2 P3 - t tw2, tw2 = c4 + t tw1, tw1 = c5 + t c6;
        // Np = 2 P3 + t tv2, tv2 = c4 - t tv1, tv1 = c5 - t c6
        P3_b = fma_t(T(2), Nn_b + Np_b, P3_b);
        const T tw2_b = -iR * Nn_b, tv2_b = iR * Np_b;
        const T tw1_b = iR * tw2_b, tv1_b = -iR * tv2_b;
        iR_b = iR_b - tw2 * Nn_b + tv2 * Np_b + tw1 * tw2_b - tv1 * tv2_b + c6 * (tw1_b - tv1_b);
        const T c4_b = tw2_b + tv2_b, c5_b = tw1_b + tv1_b, c6_b = iR * (tw1_b - tv1_b);
        // c4 = P2 (P2 - 4 u2 + 2) + u2, c5 = 2 u (P2 - P2^2), c6 = P2^2
        P2_b = P2_b + c4_b * (T(2) * P2 - T(4) * u2 + T(2)) +
               c5_b * (T(2) * u) * (T(1) - T(2) * P2) + c6_b * (T(2) * P2);
        u_b = u_b + c4_b * (T(2) * u - T(8) * u * P2) + c5_b * (T(2) * (P2 - P2 * P2));
        // P2R3 = P2 iR3 (in psi2), iR3 = iR2 iR, iR2 = iR^2
        P2_b = fma_t(P2R3_b, iR3, P2_b);
        iR3_b = fma_t(P2R3_b, P2, iR3_b);
        iR2_b = iR3_b * iR;
        iR_b = fma_t(iR3_b, iR2, iR_b);
        iR_b = fma_t(T(2) * iR, iR2_b, iR_b);
    } else {
        // Eg = 2 (x (iR + P2R3) - y uR2) - 2
        const T Sg2 = T(2) * Eg_b;
        x_b = fma_t(Sg2, iRP, x_b);
        iR_b = Sg2 * x;
        P2R3_b = fma_t(Sg2, x, P2R3_b);
        y_b = fma_t(-Sg2, uR2, y_b);
        T uR2_b = -Sg2 * y;
        // Ea = (x - y) T1 - 1, Eb = (x + y) T2 + 1
        x_b = x_b + Ea_b * T1 + Eb_b * T2;
        y_b = y_b - Ea_b * T1 + Eb_b * T2;
        const T T1_b = Ea_b * xmy, T2_b = Eb_b * xpy;
        iR_b = iR_b + T1_b - T2_b;
        uR2_b = uR2_b + T1_b + T2_b;
        P2R3_b = P2R3_b + T1_b - T2_b;
        // P2R3 = P2 iR3, uR2 = u iR2, iR3 = iR2 iR, iR2 = iR^2
        P2_b = fma_t(P2R3_b, iR3, P2_b);
        iR3_b = fma_t(P2R3_b, P2, iR3_b);
        u_b = uR2_b * iR2;
        iR2_b = fma_t(uR2_b, u, iR3_b * iR);
        iR_b = fma_t(iR3_b, iR2, iR_b);
        iR_b = fma_t(T(2) * iR, iR2_b, iR_b);
    }
    // P3 = u q3, q3 = 2.5 u2 - 1.5, P2 = 1.5 u2 - 0.5, u2 = u^2
    u_b = fma_t(P3_b, q3, u_b);
    const T u2_b = P3_b * u * T(2.5) + T(1.5) * P2_b;
    u_b = fma_t(T(2) * u, u2_b, u_b);
    // u = xy iR, xy = x y
    const T xy_b = u_b * iR;
    iR_b = fma_t(u_b, xy, iR_b);
    x_b = fma_t(xy_b, y, x_b);
    y_b = fma_t(xy_b, x, y_b);
    // iR = R2^(-1/2), R2 = x2m1 + y^2
    const T R2_b = T(-0.5) * iR_b * iR3;
    x2m1_b = x2m1_b + R2_b;
    y_b = fma_t(T(2) * y, R2_b, y_b);
    // x2m1 = xm1 xp1, xp1 = x + 1
    xm1_b = fma_t(x2m1_b, xp1, xm1_b);
    xp1_b = fma_t(x2m1_b, xm1, xp1_b);
    x_b = x_b + xp1_b;
    // x, x - 1 linear in r; y = cos theta, s2 = sin^2 theta
    const T dHr = (x_b + xm1_b) * ik;
    const T dHth = s * (T(2) * cs * s2_b - y_b);
    o.dpr = T(-0.5) * dHr;
    o.dpth = T(-0.5) * dHth;
}

template <class T, bool TAIL = false>
GT_HD void mn_rates(const SpacetimeT<T> &c, T r, T th, T pr, T pth, T pt, T pph, Rates<T> &o)
{
    T s, cs;
    sincos_t(th, &s, &cs);
    mn_rates_sc<T, TAIL>(c, r, s, cs, pr, pth, pt, pph, o);
}

// The same rates by forward-mode dual numbers (value, d/dr, d/dtheta) through
// mn_potentials: the reference form the reverse sweep above is checked against.
template <class T>
GT_HD void mn_rates_fwd(const SpacetimeT<T> &c, T r, T th, T pr, T pth, T pt, T pph,
                        Rates<T> &o)
{
    MNPot<D3<T>> P;
    mn_potentials<T, D3<T>>(c, r, th, P);
    const D3<T> pw = P.om * pt + pph;                 // p_phi + w p_t
    const D3<T> H2 = P.invf * (-pt * pt) + P.F * dsq(pw) + P.G * (P.Delta * (pr * pr) + pth * pth);
    const T Fpw = P.F.v * pw.v;
    o.dt = fma_t(Fpw, P.om.v, -pt * P.invf.v);
    o.dph = Fpw;
    o.dr = P.G.v * P.Delta.v * pr;
    o.dth = P.G.v * pth;
    o.dpr = T(-0.5) * H2.r;
    o.dpth = T(-0.5) * H2.t;
}

// (t, phi) block of the inverse metric, g^{tt}, g^{t phi}, g^{phi phi}, with N = D3<T>
// (values and r, theta derivatives) or V1<T> (values): the ring emitter's circular orbit
// needs their exact r derivatives.
template <class T, class N>
GT_HD void kerr_upper_tphi(const SpacetimeT<T> &c, T r, T th, N g[3])
{
    T s, cs;
    sincos_t(th, &s, &cs);
    const T a = T(c.a), a2 = T(c.a2), M = T(c.M);
    N R, S2, C2;
    mkvar(R, r, T(1), T(0));
    mkvar(S2, s * s, T(0), T(2) * s * cs);
    mkvar(C2, cs * cs, T(0), T(-2) * s * cs);
    const N r2 = dsq(R);
    const N ra2 = r2 + a2;
    const N Sigma = r2 + C2 * a2;
    const N Delta = r2 - R * (T(2) * M) + a2;
    const N iD = drcp(Sigma * Delta);
    g[0] = -(dsq(ra2) - Delta * S2 * a2) * iD;
    g[1] = R * iD * (T(-2) * M * a);
    g[2] = (Delta - S2 * a2) * iD * drcp(S2);
}

template <class T, class N>
GT_HD void mn_upper_tphi(const SpacetimeT<T> &c, T r, T th, N g[3])
{
    MNPot<N> P;
    mn_potentials<T, N>(c, r, th, P);
    g[0] = -P.invf + dsq(P.om) * P.F;
    g[1] = P.om * P.F;
    g[2] = P.F;
}

#ifdef __CUDACC__
__device__ __forceinline__ void mn_upper(const SpacetimeC &c, double r, double th, double g[5])
{
    MNPot<V1<double>> P;
    mn_potentials<double, V1<double>>(c, r, th, P);
    g[0] = -P.invf.v + P.om.v * P.om.v * P.F.v;
    g[1] = P.om.v * P.F.v;
    g[2] = P.F.v;
    g[3] = P.G.v * P.Delta.v;
    g[4] = P.G.v;
}

template <int KIND, class T>
GT_HD void rates(const SpacetimeT<T> &c, T r, T th, T pr, T pth, T pt, T pph,
                                      Rates<T> &o)
{
    if (KIND == KIND_KERR)
        kerr_rates<T>(c, r, th, pr, pth, pt, pph, o);
    else
        mn_rates<T>(c, r, th, pr, pth, pt, pph, o);
}

__device__ __forceinline__ void upper_metric(const SpacetimeC &c, double r, double th, double g[5])
{
    if (c.kind == KIND_KERR)
        kerr_upper(c, r, th, g);
    else
        mn_upper(c, r, th, g);
}
#endif

} // namespace gt
