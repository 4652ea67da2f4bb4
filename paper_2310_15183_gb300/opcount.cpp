// opcount.cpp -- algorithmic operation count of one RK4 step, taken from the very
// templates the kernels run (spacetime.cuh) instantiated with a counting scalar.
// Host-only program; prints JSON.  Convention: add, sub, mul = 1 flop, fma = 2,
// div, rsqrt, exp = 1 each, sincos = 2 (sin and cos); negation is free.
#include <math.h>
#include <stdio.h>

struct Counts {
    long add = 0, mul = 0, fma = 0, div = 0, rsqrt = 0, exp = 0, sincos = 0;
};

static Counts g_c;

struct CN {
    double v;
    CN(double x = 0.0) : v(x) {}
};
static CN operator+(CN a, CN b) { g_c.add++; return CN(a.v + b.v); }
static CN operator-(CN a, CN b) { g_c.add++; return CN(a.v - b.v); }
static CN operator*(CN a, CN b) { g_c.mul++; return CN(a.v * b.v); }
static CN operator/(CN a, CN b) { g_c.div++; return CN(a.v / b.v); }
static CN operator-(CN a) { return CN(-a.v); }

// found by argument-dependent lookup from the templates in namespace gt
static void sincos_t(CN x, CN *s, CN *c) { g_c.sincos++; *s = CN(sin(x.v)); *c = CN(cos(x.v)); }
static CN exp_t(CN x) { g_c.exp++; return CN(exp(x.v)); }
static CN rsqrt_t(CN x) { g_c.rsqrt++; return CN(1.0 / sqrt(x.v)); }
static CN rcp_t(CN x) { g_c.div++; return CN(1.0 / x.v); }
static CN fma_t(CN a, CN b, CN c) { g_c.fma++; return CN(a.v * b.v + c.v); }

#include "csrc/spacetime.cuh"

static long flops(const Counts &c)
{
    return c.add + c.mul + 2 * c.fma + c.div + c.rsqrt + c.exp + 2 * c.sincos;
}

static void print_counts(const char *name, const Counts &c, bool last)
{
    printf("  \"%s\": {\"add\": %ld, \"mul\": %ld, \"fma\": %ld, \"div\": %ld, \"rsqrt\": %ld, "
           "\"exp\": %ld, \"sincos\": %ld, \"flops\": %ld}%s\n",
           name, c.add, c.mul, c.fma, c.div, c.rsqrt, c.exp, c.sincos, flops(c), last ? "" : ",");
}

int main()
{
    gt::SpacetimeT<CN> st = {};
    st.M = 0.5;
    st.a = 0.48;
    st.a2 = 0.48 * 0.48;
    st.k = 0.14;
    st.ik = 1.0 / 0.14;
    st.alpha = -0.75;
    st.beta = 91.1;
    st.two_beta = 2 * 91.1;
    st.three_beta2 = 3 * 91.1 * 91.1;
    st.c_g = 1.0;
    st.w_inf = 0.1;
    st.k2 = 0.14 * 0.14;
    st.inv_k2 = 1.0 / (0.14 * 0.14);
    st.two_k = 2 * 0.14;
    st.r_plus = 0.5 + 0.14;
    gt::Rates<CN> o;
    g_c = Counts();
    gt::kerr_rates<CN>(st, CN(5.0), CN(1.1), CN(0.2), CN(0.3), CN(0.9), CN(-2.0), o);
    const Counts kerr = g_c;
    g_c = Counts();
    gt::mn_rates<CN>(st, CN(5.0), CN(1.1), CN(0.2), CN(0.3), CN(0.9), CN(-2.0), o);
    const Counts mn = g_c;
    g_c = Counts();
    gt::mn_rates<CN, true>(st, CN(5.0), CN(1.1), CN(0.2), CN(0.3), CN(0.9), CN(-2.0), o);
    const Counts mn_tail = g_c; // closed-form multipole tails (GT_FLAG_PRECISE_MN)
    // RK4 combination outside the four field evaluations (trace.cu, rk4_step64):
    //   h = |sp / k1.dt|: 1 div; hh = 0.5 h: 1 mul; 3 stages x 4 state fma;
    //   hw = h w: 1 mul; 6 components x (k1 + 2k2 + 2k3 + k4: 2 fma + 1 add; x + hw s: 1 fma)
    Counts comb;
    comb.div = 1;
    comb.mul = 2;
    comb.fma = 12 + 6 * 3;
    comb.add = 6;
    // FP32-mixed adds the compensated update (increment into the low part, then Fast2Sum:
    // 4 adds) per component (compensated.cuh, f2_add)
    Counts comp;
    comp.add = 6 * 4;
    printf("{\n");
    print_counts("kerr_field", kerr, false);
    print_counts("mn_field", mn, false);
    print_counts("mn_field_precise", mn_tail, false);
    print_counts("rk4_combination", comb, false);
    print_counts("compensated_update", comp, false);
    printf("  \"kerr_step_flops\": %ld,\n", 4 * flops(kerr) + flops(comb));
    printf("  \"mn_step_flops\": %ld,\n", 4 * flops(mn) + flops(comb));
    printf("  \"kerr_step_flops_mixed\": %ld,\n", 4 * flops(kerr) + flops(comb) + flops(comp));
    printf("  \"mn_step_flops_mixed\": %ld,\n", 4 * flops(mn) + flops(comb) + flops(comp));
    printf("  \"mn_step_flops_mixed_precise\": %ld\n", 4 * flops(mn_tail) + flops(comb) + flops(comp));
    printf("}\n");
    return 0;
}
