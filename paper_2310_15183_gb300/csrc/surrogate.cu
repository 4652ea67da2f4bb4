// surrogate.cu -- the MLP surrogate of the ray tracer: per-pixel (alpha, beta, spin,
// q, theta0) -> (escape logit, end direction), trained on rays the integrator itself
// produces, evaluated with the tcgen05 GEMM, and backed by the integrator for
// low-confidence and photon-ring pixels.
//
// Network: 16 (5 inputs and 5 columns derived from them, zero padded) -> 256 -> 256 ->
// 256 -> 256 -> 16 (4 used: logit and the unit vector of the end direction, which unlike
// (theta, phi) has no jump at phi = +-pi), SiLU between layers.  FP32 master weights and
// AdamW state.  The forward products are split-precision BF16: each layer input x and
// weight w is carried as a bf16 pair (hi, lo), hi = bf16(v), lo = bf16(v - hi), and the
// product is x_hi w_hi + x_lo w_hi + x_hi w_lo -- one tcgen05 GEMM over K' = 3K with the
// input laid out [x_hi | x_lo | x_hi] and the weights [w_hi | w_hi | w_lo] -- which carries
// the layer to about 2^-16 relative instead of bf16's 2^-8 (the dropped x_lo w_lo term is
// 2^-16 of the product); the end direction is read from the last layer, and a single
// 16-bit product leaves a rounding floor of 5e-4 (FP16) to 2e-3 rad (BF16) under it.  The
// backward products take plain BF16, whose range holds gradients scaled by 1/batch.
// Accumulation is FP32 throughout.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/geotrace.h"
#include "internal.cuh"
#include "mlp.cuh"
#include "camera.cuh"
#include "surrogate.cuh"

namespace gt {
namespace sg {

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + __expf(-z)); }

// counter-based normal deviates: splitmix64 -> two uniforms -> Box-Muller
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void init_params_kernel(float *p, int64_t n, const int64_t *offs, const float *scales,
                                   int n_seg, uint64_t seed)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = 0;
    while (s + 1 < n_seg && offs[s + 1] <= i) ++s;
    const float sc = scales[s];
    if (sc == 0.0f) {
        p[i] = 0.0f;
        return;
    }
    const uint64_t a = splitmix64(seed ^ (uint64_t)(2 * i));
    const uint64_t b = splitmix64(seed ^ (uint64_t)(2 * i + 1));
    const double u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0);
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    p[i] = sc * (float)(sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2));
}

// The network's 16 input columns from the 5 inputs (alpha, beta, a/M, q, theta0):
// 0-4 the inputs scaled to about [-1, 1]; 5-7 the pixel direction in polar form
// (rho, cos psi, sin psi) of the scaled (alpha, beta); 8-9 cos and sin of theta0; the
// rest zero.  The derived columns are fixed functions of the inputs.
__device__ __forceinline__ void make_features(double al, double bt, double spin, double q,
                                              double th0, const Norm &nm, float f[16])
{
    const double a = al * nm.inv_h, b = bt * nm.inv_v;
    const double rho = sqrt(a * a + b * b);
    const double irho = 1.0 / fmax(rho, 1e-3);
    f[0] = (float)a;
    f[1] = (float)b;
    f[2] = (float)(spin * nm.spin_scale + nm.spin_shift);
    f[3] = (float)(q * nm.q_scale);
    f[4] = (float)(th0 * nm.th_scale + nm.th_shift);
    f[5] = (float)rho;
    f[6] = (float)(a * irho);
    f[7] = (float)(b * irho);
    f[8] = (float)cos(th0);
    f[9] = (float)sin(th0);
#pragma unroll
    for (int j = 10; j < 16; j++) f[j] = 0.0f;
}

// bf16 pair of v: hi = bf16(v), lo = bf16(v - hi)
__device__ __forceinline__ void split_pair(float v, __nv_bfloat16 *hi, __nv_bfloat16 *lo)
{
    *hi = __float2bfloat16(v);
    *lo = __float2bfloat16(v - __bfloat162float(*hi));
}

// One row of the first layer's split input: columns [hi 0..15 | lo 0..15 | hi 0..15]
__device__ __forceinline__ void store_split_row(const float f[16], __nv_bfloat16 *row)
{
#pragma unroll
    for (int j = 0; j < 16; j++) {
        __nv_bfloat16 hi, lo;
        split_pair(f[j], &hi, &lo);
        row[j] = hi;
        row[16 + j] = lo;
        row[32 + j] = hi;
    }
}

// features of samples [row0, row0 + n): X0[r, 0..47] (split bf16, input of the forward
// product) and optionally X0T (bf16 of the features, transposed, input of the
// weight-gradient product)
__global__ void features_kernel(int64_t n, int64_t row0, const double *alpha, const double *beta,
                                const double *spin, const double *q, const double *theta0,
                                Norm nm, __nv_bfloat16 *X0, __nv_bfloat16 *X0T = nullptr)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t k = row0 + r;
    float f[16];
    make_features(alpha[k], beta[k], spin[k], q[k], theta0[k], nm, f);
    store_split_row(f, X0 + r * 3 * 16);
    if (X0T)
#pragma unroll
        for (int j = 0; j < 16; j++) X0T[j * n + r] = __float2bfloat16(f[j]);
}

// features of camera pixels [pix0, pix0 + n) (flat j*res_x + i), or of the listed pixels
// pixels[pix0 + r]
__global__ void camera_features_kernel(int64_t n, int64_t pix0, const CamDesc *cam, Norm nm,
                                       __nv_bfloat16 *X0, const int64_t *pixels = nullptr)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const CamDesc &c = *cam;
    const int64_t pix = pixels ? pixels[pix0 + r] : pix0 + r;
    const int i = (int)(pix % c.res_x), j = (int)(pix / c.res_x);
    const double al = c.res_x > 1 ? c.H * (double)(2 * i - (c.res_x - 1)) / (double)(c.res_x - 1) : 0.0;
    const double bt = c.res_y > 1 ? c.V * (double)(2 * j - (c.res_y - 1)) / (double)(c.res_y - 1) : 0.0;
    float f[16];
    make_features(al, bt, (c.S / c.M) / c.M, c.Q, c.th0, nm, f);
    store_split_row(f, X0 + r * 3 * 16);
}

// Loss of rows [0, B): BCE(logit, y) + w_dir * y * |d_pred - d|^2, averaged over B.
// labels: [B x 4] = (y, dx, dy, dz).  Writes dZ5 (fp32 and bf16, 16 columns, zeros
// beyond 4) and accumulates the loss sum.
__global__ void head_kernel(int B, const float *Z5, const float *labels, float w_dir, float inv_b,
                            float *dZ5f, __nv_bfloat16 *dZ5b, __nv_bfloat16 *dZ5T, float *loss_acc)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (r < B) {
        const float *z = Z5 + (int64_t)r * 16;
        const float *lab = labels + (int64_t)r * 4;
        const float y = lab[0];
        const float zl = z[0];
        // numerically stable BCE with logits
        l = fmaxf(zl, 0.0f) - zl * y + log1pf(__expf(-fabsf(zl)));
        float g[16];
        g[0] = (sigmoidf(zl) - y) * inv_b;
        for (int j = 1; j < 4; j++) {
            const float d = z[j] - lab[j];
            l += w_dir * y * d * d;
            g[j] = 2.0f * w_dir * y * d * inv_b;
        }
        for (int j = 4; j < 16; j++) g[j] = 0.0f;
        for (int j = 0; j < 16; j++) {
            dZ5f[(int64_t)r * 16 + j] = g[j];
            dZ5b[(int64_t)r * 16 + j] = __float2bfloat16(g[j]);
            dZ5T[(int64_t)j * B + r] = __float2bfloat16(g[j]);
        }
    }
    // warp-reduce the loss, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, l);
}

// dZ = dX * SiLU'(Z), SiLU'(z) = s (1 + z (1 - s)), s = sigmoid(z)
// dZT is the transposed (cols x rows) bf16 copy used by the weight-gradient product.
__global__ void silu_backward_kernel(int64_t rows, int cols, const float *dX, const float *Z,
                                     float *dZf, __nv_bfloat16 *dZb, __nv_bfloat16 *dZT)
{
    // consecutive threads take consecutive rows of one column: coalesced transposed stores
    const int64_t n = rows * cols;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t r = k % rows, c = k / rows;
    const int64_t i = r * cols + c;
    const float z = Z[i];
    const float s = sigmoidf(z);
    const float g = dX[i] * s * (1.0f + z * (1.0f - s));
    dZf[i] = g;
    dZb[i] = __float2bfloat16(g);
    dZT[c * rows + r] = __float2bfloat16(g);
}

// WT[l] = bf16 transpose of the fp32 weights [out][in] -> [in][out]
__global__ void weights_t_kernel(const float *W, int out_dim, int in_dim, __nv_bfloat16 *WT)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= out_dim * in_dim) return;
    const int o = k / in_dim, i = k % in_dim;
    WT[(int64_t)i * out_dim + o] = __float2bfloat16(W[k]);
}

// out[c] += sum_r M[r, c]  (rows x cols, row-major)
__global__ void colsum_kernel(const float *Mx, int64_t rows, int cols, float *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    const int64_t per = (rows + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
    float s = 0.0f;
    for (int64_t r = r0; r < r1; r++) s += Mx[r * cols + c];
    atomicAdd(&out[c], s);
}

__global__ void adamw_kernel(int64_t n, float *p, const float *g, float *m, float *v, float lr,
                             float b1, float b2, float eps, float wd, float bc1, float bc2,
                             const uint8_t *decay_mask)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i];
    if (decay_mask[i]) pi -= lr * wd * pi;
    pi -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
}

// W3 = [w_hi | w_hi | w_lo] per output row (bf16, [out][3 in]) of fp32 weights [out][in]:
// the B operand of the split-precision forward product
__global__ void weights_split_kernel(const float *W, int out_dim, int in_dim, __nv_bfloat16 *W3)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= out_dim * in_dim) return;
    const int o = k / in_dim, i = k % in_dim;
    __nv_bfloat16 hi, lo;
    split_pair(W[k], &hi, &lo);
    __nv_bfloat16 *row = W3 + (int64_t)o * 3 * in_dim;
    row[i] = hi;
    row[in_dim + i] = hi;
    row[2 * in_dim + i] = lo;
}

// Constants of motion of a camera ray in the Kerr picture: E = -p_t, L = p_phi and the
// Carter constant K = p_theta^2 + cos^2 theta0 (-a^2 E^2 + L^2/sin^2 theta0), with a = S/M
// (Manko-Novikov rays take the Kerr values of their M and S: an estimate there).
__device__ __forceinline__ void kerr_constants(const CamDesc &c, const Ray64 &p, double *a,
                                               double *E, double *L, double *K)
{
    *a = c.S / c.M;
    *E = -p.pt;
    *L = p.pph;
    const double ct = cos(c.th0), st = sin(c.th0);
    *K = p.pth * p.pth + ct * ct * (-(*a) * (*a) * (*E) * (*E) + (*L) * (*L) / (st * st));
}

// Photon-ring test for a Kerr pixel: the radial potential of its constants of motion,
//   R(r) = (E (r^2 + a^2) - a L)^2 - Delta ((L - a E)^2 + K),
// has a (near) double root for rays near the critical curve.  Returns
// min over r in (r_+, r0] of R(r) / (E^2 r^4) on a geometric grid.
__device__ double kerr_rmin(const CamDesc &c, const Ray64 &p)
{
    double a, E, L, K;
    kerr_constants(c, p, &a, &E, &L, &K);
    const double M = c.M;
    const double rp = c.st.kind == KIND_KERR ? c.st.r_plus : M + sqrt(fmax(M * M - a * a, 0.0));
    const double lo = log(rp * 1.0001), hi = log(c.r0);
    double best = 1e300;
    for (int k = 0; k <= 96; k++) {
        const double r = exp(lo + (hi - lo) * k / 96.0);
        const double W = E * (r * r + a * a) - a * L;
        const double D = r * r - 2.0 * M * r + a * a;
        const double R = W * W - D * ((L - a * E) * (L - a * E) + K);
        const double v = R / (E * E * r * r * r * r);
        best = v < best ? v : best;
    }
    return best;
}

// Smallest sin^2 theta a Kerr ray can reach: the theta potential
// Theta = K + a^2 E^2 cos^2 - L^2 cot^2 vanishes at u = cos^2 theta solving
// -a^2 E^2 u^2 + (a^2 E^2 - K - L^2) u + K = 0; returns 1 - u for its root in [0, 1].
// Rays that pass close to the axis sweep phi fast and end in directions that change
// abruptly from pixel to pixel.
__device__ double kerr_min_sin2(const CamDesc &c, const Ray64 &p)
{
    double a, E, L, K;
    kerr_constants(c, p, &a, &E, &L, &K);
    const double A = -a * a * E * E, B = a * a * E * E - K - L * L, C = K;
    double u;
    if (fabs(A) < 1e-300) {
        u = (K + L * L) > 0.0 ? K / (K + L * L) : 0.0;
    } else {
        const double disc = sqrt(fmax(B * B - 4.0 * A * C, 0.0));
        const double u1 = (-B + disc) / (2.0 * A), u2 = (-B - disc) / (2.0 * A);
        u = 0.0;
        if (u1 >= 0.0 && u1 <= 1.0) u = fmax(u, u1);
        if (u2 >= 0.0 && u2 <= 1.0) u = fmax(u, u2);
    }
    return 1.0 - u;
}

// Probe pixel columns: k stride for k < n - 1, and the last column (res - 1).
__device__ __forceinline__ int probe_coord(int k, int stride, int n, int res)
{
    return k < n - 1 ? k * stride : res - 1;
}

__device__ __forceinline__ bool is_probe(int i, int j, const ProbeGrid &pg, int res_x, int res_y)
{
    return (i % pg.stride == 0 || i == res_x - 1) && (j % pg.stride == 0 || j == res_y - 1);
}

// The network's answer per pixel (logit, direction) kept for the passes below.
__global__ void net_out_kernel(int64_t n, int64_t pix0, const float *Z5, float4 *net)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float *z = Z5 + k * 16;
    net[pix0 + k] = make_float4(z[0], z[1], z[2], z[3]);
}

// Gates that send a pixel to the integrator whatever the probes say: an unsure logit, the
// Kerr photon-ring band, the axis, an unsettled direction length.
__device__ __forceinline__ bool pixel_gates(const CamDesc &cam, int64_t pix, float4 z, float tau,
                                            double band, double axis, float dir_tol)
{
    if (fabsf(z.x) < tau) return true;
    if ((band > 0.0 && cam.st.kind == KIND_KERR) || axis > 0.0) {
        Ray64 p;
        camera_init(cam, pix, p);
        if (band > 0.0 && cam.st.kind == KIND_KERR && fabs(kerr_rmin(cam, p)) < band) return true;
        if (axis > 0.0 && kerr_min_sin2(cam, p) < axis * axis) return true;
    }
    if (dir_tol > 0.0f && z.x > 0.0f) {
        const float nn = sqrtf(z.y * z.y + z.z * z.z + z.w * z.w);
        if (!(fabsf(nn - 1.0f) <= dir_tol)) return true;
    }
    return false;
}

// The probe cell holding pixel (i, j): corner columns x0 < x1 and rows y0 < y1, and the
// index (kx, ky) of its upper-left probe.
struct Cell {
    int kx, ky, x0, x1, y0, y1;
};

__device__ __forceinline__ Cell cell_of(int i, int j, const ProbeGrid &pg, int res_x, int res_y)
{
    Cell c;
    c.kx = min(i / pg.stride, pg.nx - 2);
    c.ky = min(j / pg.stride, pg.ny - 2);
    c.x0 = probe_coord(c.kx, pg.stride, pg.nx, res_x);
    c.x1 = probe_coord(c.kx + 1, pg.stride, pg.nx, res_x);
    c.y0 = probe_coord(c.ky, pg.stride, pg.ny, res_y);
    c.y1 = probe_coord(c.ky + 1, pg.stride, pg.ny, res_y);
    return c;
}

// First integrator list: the probes, every pixel a gate sends to the integrator, and --
// with probes -- every pixel whose predicted escape differs from the network's prediction
// at one of its cell's corners (such a pixel fails the cell test whatever the integrator
// finds at the corners).  Tracing them in the probes' launch leaves one tail of long rays
// where two passes would leave two.
__device__ __forceinline__ bool first_pass_pixel(const CamDesc &cam, const float4 *net, int64_t pix,
                                                 const ProbeGrid &pg, float tau, double band,
                                                 double axis, float dir_tol)
{
    const int res_x = cam.res_x, res_y = cam.res_y;
    const int i = (int)(pix % res_x), j = (int)(pix / res_x);
    const float4 z = net[pix];
    if (pg.stride > 0) {
        if (is_probe(i, j, pg, res_x, res_y)) return true;
        const Cell c = cell_of(i, j, pg, res_x, res_y);
        const bool esc = z.x > 0.0f;
        const int64_t r0 = (int64_t)c.y0 * res_x, r1 = (int64_t)c.y1 * res_x;
        if ((net[r0 + c.x0].x > 0.0f) != esc || (net[r0 + c.x1].x > 0.0f) != esc ||
            (net[r1 + c.x0].x > 0.0f) != esc || (net[r1 + c.x1].x > 0.0f) != esc)
            return true;
    }
    return pixel_gates(cam, pix, z, tau, band, axis, dir_tol);
}

// warp-aggregated append of the flagged pixels to a list
__device__ __forceinline__ void append_flagged(bool flag, int64_t pix, int64_t *list,
                                               unsigned long long *count)
{
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(mask) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (flag) list[base + __popc(mask & ((1u << lane) - 1u))] = pix;
    }
}

__global__ void select_kernel(int64_t n_pix, const CamDesc *cam, const float4 *net, ProbeGrid pg,
                              float tau, double band, double axis, float dir_tol, int64_t *list,
                              unsigned long long *count)
{
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool flag = pix < n_pix && first_pass_pixel(*cam, net, pix, pg, tau, band, axis, dir_tol);
    append_flagged(flag, pix, list, count);
}

// Probe records from the integrator's results (already in the image) and the network's
// answers at the probes.
__global__ void probe_record_kernel(const CamDesc *cam, ProbeGrid pg, const float4 *net,
                                    const uint8_t *status, const double *th, const double *ph,
                                    ProbeRec *rec)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= pg.nx * pg.ny) return;
    const int kx = k % pg.nx, ky = k / pg.nx;
    const int64_t pix = (int64_t)probe_coord(ky, pg.stride, pg.ny, cam->res_y) * cam->res_x +
                        probe_coord(kx, pg.stride, pg.nx, cam->res_x);
    const float4 z = net[pix];
    ProbeRec o;
    o.exact = status[pix];
    o.net_esc = z.x > 0.0f ? 1 : 0;
    o.pad[0] = o.pad[1] = 0;
    if (o.exact == GT_RAY_ESCAPED) {
        const double s = sin(th[pix]);
        o.err[0] = (float)(s * cos(ph[pix])) - z.y;
        o.err[1] = (float)(s * sin(ph[pix])) - z.z;
        o.err[2] = (float)cos(th[pix]) - z.w;
    } else {
        o.err[0] = o.err[1] = o.err[2] = 0.0f;
    }
    rec[k] = o;
}

// Every pixel the first pass did not trace: with probes, taken from the network only
// inside a probe cell whose four corners the integrator and the network classify alike --
// all escaped, or all not escaping with one common end (all HORIZON, or all MAXSTEPS:
// trapped; the pixel takes that status) -- and, for escaped ones, whose corner error
// vectors differ by less than pg.tol; its end direction is the network's plus the bilinear
// interpolation of the corners' error vectors (the integrator correcting the network
// where it measured it).  The rest go to the second integrator list.
__global__ void gate_kernel(int64_t n_pix, const CamDesc *cam, const float4 *net, ProbeGrid pg,
                            float tau, double band, double axis, float dir_tol, double *t,
                            double *r, double *th, double *ph, uint8_t *status, uint32_t *nsteps,
                            int64_t *fallback, unsigned long long *n_fallback)
{
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool fb = false;
    if (pix < n_pix && !first_pass_pixel(*cam, net, pix, pg, tau, band, axis, dir_tol)) {
        const int res_x = cam->res_x, res_y = cam->res_y;
        const int i = (int)(pix % res_x), j = (int)(pix / res_x);
        const float4 z = net[pix];
        float nx = z.y, ny = z.z, nz = z.w;
        int cap_status = GT_RAY_HORIZON; // status given to a captured network pixel
        if (pg.stride > 0) {
            const Cell cl = cell_of(i, j, pg, res_x, res_y);
            const int kx = cl.kx, ky = cl.ky, x0 = cl.x0, x1 = cl.x1, y0 = cl.y0, y1 = cl.y1;
            const ProbeRec &c00 = pg.rec[ky * pg.nx + kx], &c01 = pg.rec[ky * pg.nx + kx + 1];
            const ProbeRec &c10 = pg.rec[(ky + 1) * pg.nx + kx];
            const ProbeRec &c11 = pg.rec[(ky + 1) * pg.nx + kx + 1];
            const bool esc4 = c00.exact == GT_RAY_ESCAPED && c01.exact == GT_RAY_ESCAPED &&
                              c10.exact == GT_RAY_ESCAPED && c11.exact == GT_RAY_ESCAPED &&
                              c00.net_esc && c01.net_esc && c10.net_esc && c11.net_esc;
            const bool cap4 = (c00.exact == GT_RAY_HORIZON || c00.exact == GT_RAY_MAXSTEPS) &&
                              c01.exact == c00.exact && c10.exact == c00.exact &&
                              c11.exact == c00.exact && !c00.net_esc && !c01.net_esc &&
                              !c10.net_esc && !c11.net_esc;
            cap_status = c00.exact;
            if (z.x > 0.0f) {
                float sp = 0.0f, sq = 0.0f;
#pragma unroll
                for (int m = 0; m < 3; m++) {
                    const float a = c00.err[m] - c11.err[m], b = c01.err[m] - c10.err[m];
                    sp = fmaf(a, a, sp);
                    sq = fmaf(b, b, sq);
                }
                if (!esc4 || !(fmaxf(sp, sq) < pg.tol * pg.tol)) {
                    fb = true;
                } else {
                    const float tx = (float)(i - x0) / (float)(x1 - x0);
                    const float ty = (float)(j - y0) / (float)(y1 - y0);
                    const float w00 = (1.0f - tx) * (1.0f - ty), w01 = tx * (1.0f - ty);
                    const float w10 = (1.0f - tx) * ty, w11 = tx * ty;
                    nx += w00 * c00.err[0] + w01 * c01.err[0] + w10 * c10.err[0] + w11 * c11.err[0];
                    ny += w00 * c00.err[1] + w01 * c01.err[1] + w10 * c10.err[1] + w11 * c11.err[1];
                    nz += w00 * c00.err[2] + w01 * c01.err[2] + w10 * c10.err[2] + w11 * c11.err[2];
                }
            } else if (!cap4) {
                fb = true;
            }
        }
        if (!fb) {
            if (z.x > 0.0f) {
                const float nc = sqrtf(nx * nx + ny * ny + nz * nz);
                th[pix] = acos(fminf(fmaxf(nz / nc, -1.0f), 1.0f));
                ph[pix] = atan2(ny, nx);
                status[pix] = GT_RAY_ESCAPED;
            } else {
                th[pix] = nan("");
                ph[pix] = nan("");
                status[pix] = (uint8_t)cap_status;
            }
            t[pix] = nan("");
            r[pix] = nan("");
            nsteps[pix] = 0;
        }
    }
    append_flagged(fb, pix, fallback, n_fallback);
}

} // namespace sg
} // namespace gt

// ====================================================================== host side
namespace {

using namespace gt;
using namespace gt::sg;

__global__ void labels_kernel(int64_t n, int64_t row0, const uint8_t *status, const double *th,
                              const double *ph, float *lab)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t k = row0 + r;
    const bool esc = status[k] == GT_RAY_ESCAPED;
    float y = esc ? 1.0f : 0.0f, dx = 0.f, dy = 0.f, dz = 0.f;
    if (esc) {
        const double s = sin(th[k]);
        dx = (float)(s * cos(ph[k]));
        dy = (float)(s * sin(ph[k]));
        dz = (float)cos(th[k]);
    }
    lab[r * 4 + 0] = y;
    lab[r * 4 + 1] = dx;
    lab[r * 4 + 2] = dy;
    lab[r * 4 + 3] = dz;
}

inline unsigned blocks_for(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

} // namespace

struct gt_surrogate {
    int device = 0;
    Norm norm = {};
    int64_t w_off[N_LAYERS] = {}, b_off[N_LAYERS] = {};
    int64_t n_params = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr; // fp32 params, grads, Adam
    uint8_t *decay = nullptr;
    __nv_bfloat16 *w3 = nullptr; // split bf16 weights of the forward products, [out][3 in] per layer
    int64_t w3_off[N_LAYERS] = {};
    int64_t step = 0;
    // workspace for `rows` rows
    int64_t rows = 0;
    __nv_bfloat16 *X[N_LAYERS] = {};  // split inputs of each layer (rows x 3 in, forward products)
    __nv_bfloat16 *XT[N_LAYERS] = {}; // the same in bf16, transposed (in_dim x rows)
    __nv_bfloat16 *WT = nullptr;      // transposed bf16 weights ([in][out] per layer)
    __nv_bfloat16 *dZT = nullptr;     // transposed bf16 gradient (cols x rows)
    float *Z[N_LAYERS] = {};         // pre-activations (fp32)
    float *dXf = nullptr, *dZf = nullptr, *lab = nullptr, *loss = nullptr;
    __nv_bfloat16 *dZb = nullptr;
    int *err = nullptr;
};

namespace {

void free_ws(gt_surrogate *s)
{
    for (int l = 0; l < N_LAYERS; l++) {
        cudaFree(s->X[l]);
        cudaFree(s->XT[l]);
        cudaFree(s->Z[l]);
        s->X[l] = nullptr;
        s->XT[l] = nullptr;
        s->Z[l] = nullptr;
    }
    cudaFree(s->dZT);
    s->dZT = nullptr;
    cudaFree(s->dXf);
    cudaFree(s->dZf);
    cudaFree(s->dZb);
    cudaFree(s->lab);
    s->dXf = s->dZf = s->lab = nullptr;
    s->dZb = nullptr;
    s->rows = 0;
}

int ensure_ws(gt_surrogate *s, int64_t rows)
{
    if (s->rows >= rows) return GT_OK;
    free_ws(s);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < N_LAYERS && e == cudaSuccess; l++) {
        e = cudaMalloc(&s->X[l], rows * 3 * IN_DIM[l] * sizeof(__nv_bfloat16));
        if (e == cudaSuccess) e = cudaMalloc(&s->XT[l], rows * IN_DIM[l] * sizeof(__nv_bfloat16));
        if (e == cudaSuccess) e = cudaMalloc(&s->Z[l], rows * OUT_DIM[l] * sizeof(float));
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->dXf, rows * 256 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s->dZf, rows * 256 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s->dZb, rows * 256 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&s->dZT, rows * 256 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&s->lab, rows * 4 * sizeof(float));
    if (e != cudaSuccess) {
        free_ws(s);
        return e == cudaErrorMemoryAllocation ? GT_ERR_OOM : GT_ERR_CUDA;
    }
    s->rows = rows;
    return GT_OK;
}

struct Dev {
    int prev = -1;
    bool ok = false;
    explicit Dev(int d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(d) == cudaSuccess;
    }
    ~Dev()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// split: C16 receives the [hi | lo | hi] split of the output (3 N columns)
cudaError_t gemm(const void *A, int64_t a_sm, int64_t a_sk, const void *B, int64_t b_sn,
                 int64_t b_sk, int M, int N, int K, const float *bias, int act, float *pre,
                 float *C32, int64_t ldc, bool atomic, void *C16, int splits, int *err,
                 cudaStream_t st, __nv_bfloat16 *C16T = nullptr, bool split = false)
{
    GemmArgs g = {};
    g.c16_split = split ? 1 : 0;
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = static_cast<const __nv_bfloat16 *>(A);
    g.a_sm = a_sm;
    g.a_sk = a_sk;
    g.B = static_cast<const __nv_bfloat16 *>(B);
    g.b_sn = b_sn;
    g.b_sk = b_sk;
    g.bias = bias;
    g.act = act;
    g.pre = pre;
    g.ld_pre = N;
    g.C32 = C32;
    g.ldc = ldc;
    g.atomic = atomic ? 1 : 0;
    g.C16 = static_cast<__nv_bfloat16 *>(C16);
    g.ldc16 = split ? 3 * (int64_t)N : N;
    g.C16T = C16T;
    g.ldt = M;
    g.err = err;
    // 256-wide tiles read each A row block once when there are many of them (inference
    // chunks); 128-wide ones give a training batch twice as many tiles to spread over SMs
    const int bn = (N >= 256 && M >= 65536) ? 256 : N >= 128 ? 128 : (N >= 64 ? 64 : (N >= 32 ? 32 : 16));
    return launch_gemm(g, bn, splits, st);
}

// Forward pass of `B` rows whose features are in X[0]; leaves Z[4] = network output.
// keep_pre: also store the hidden pre-activations (needed by the backward pass only).
cudaError_t forward(gt_surrogate *s, int B, cudaStream_t st, bool keep_pre = true)
{
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < N_LAYERS && e == cudaSuccess; l++) {
        const bool last = (l == N_LAYERS - 1);
        const int K3 = 3 * IN_DIM[l];
        e = gemm(s->X[l], K3, 1, s->w3 + s->w3_off[l], K3, 1, B, OUT_DIM[l], K3,
                 s->p + s->b_off[l], last ? 0 : 1, (last || !keep_pre) ? nullptr : s->Z[l],
                 last ? s->Z[l] : nullptr, OUT_DIM[l], false, last ? nullptr : s->X[l + 1], 1,
                 s->err, st, (last || !keep_pre) ? nullptr : s->XT[l + 1], true);
    }
    return e;
}

// Backward pass of B rows with labels in s->lab: gradients (zeroed here) into s->g.
cudaError_t backward(gt_surrogate *s, int B, float w_dir, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(s->g, 0, s->n_params * sizeof(float), st);
    if (e != cudaSuccess) return e;
    head_kernel<<<blocks_for(B), 256, 0, st>>>(B, s->Z[N_LAYERS - 1], s->lab, w_dir, 1.0f / B,
                                               s->dZf, s->dZb, s->dZT, s->loss);
    for (int l = N_LAYERS - 1; l >= 0 && e == cudaSuccess; l--) {
        const int N = OUT_DIM[l], K = IN_DIM[l];
        // dW_l[n, k] = sum_b dZ[b, n] X_l[b, k] from the transposed copies (K-contiguous
        // in the batch), split over the batch
        const int splits = B >= 512 ? (B / 256 < 128 ? B / 256 : 128) : 1;
        e = gemm(s->dZT, B, 1, s->XT[l], B, 1, N, K, B, nullptr, 0, nullptr, s->g + s->w_off[l], K,
                 true, nullptr, splits, s->err, st);
        if (e != cudaSuccess) break;
        // db_l = column sums of dZ
        colsum_kernel<<<dim3(blocks_for(N, 128), 64), 128, 0, st>>>(s->dZf, B, N, s->g + s->b_off[l]);
        if (l == 0) break;
        // dX[b, k] = sum_n dZ[b, n] W_l[n, k] = dZ . (W_l^T)^T
        e = gemm(s->dZb, N, 1, s->WT + s->w_off[l], N, 1, B, K, N, nullptr, 0, nullptr, s->dXf, K,
                 false, nullptr, 1, s->err, st);
        if (e != cudaSuccess) break;
        silu_backward_kernel<<<blocks_for((int64_t)B * K), 256, 0, st>>>(B, K, s->dXf, s->Z[l - 1],
                                                                         s->dZf, s->dZb, s->dZT);
        e = cudaGetLastError();
    }
    return e;
}

int check_err(gt_surrogate *s, cudaStream_t st)
{
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, s->err, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return GT_ERR_CUDA;
    return h ? GT_ERR_TIMEOUT : GT_OK;
}

// split bf16 weights (forward products) and transposed bf16 weights (backward products)
// after an update
cudaError_t refresh_copies(gt_surrogate *s, cudaStream_t st)
{
    for (int l = 0; l < N_LAYERS; l++) {
        const int64_t n = (int64_t)OUT_DIM[l] * IN_DIM[l];
        weights_split_kernel<<<blocks_for(n), 256, 0, st>>>(s->p + s->w_off[l], OUT_DIM[l],
                                                           IN_DIM[l], s->w3 + s->w3_off[l]);
        weights_t_kernel<<<blocks_for(n), 256, 0, st>>>(s->p + s->w_off[l], OUT_DIM[l], IN_DIM[l],
                                                        s->WT + s->w_off[l]);
    }
    return cudaGetLastError();
}

} // namespace

extern "C" {

int gt_surrogate_num_params(int64_t *out)
{
    if (!out) return GT_ERR_INVALID_ARG;
    int64_t n = 0;
    for (int l = 0; l < N_LAYERS; l++) n += (int64_t)OUT_DIM[l] * IN_DIM[l] + OUT_DIM[l];
    *out = n;
    return GT_OK;
}

int gt_surrogate_create(int device, const gt_surrogate_norm *nrm, uint64_t seed, gt_surrogate **out)
{
    if (!out || !nrm) return GT_ERR_INVALID_ARG;
    if (!(nrm->r0 > 0) || !(nrm->fov_deg > 0 && nrm->fov_deg < 180) || !(nrm->spin_max > 0) ||
        !(nrm->theta0_max > nrm->theta0_min) || !(nrm->q_max > 0))
        return GT_ERR_INVALID_ARG;
    *out = nullptr;
    Dev d(device);
    if (!d.ok) return GT_ERR_CUDA;
    gt_surrogate *s = new (std::nothrow) gt_surrogate();
    if (!s) return GT_ERR_OOM;
    s->device = device;
    const double V = tan(0.5 * nrm->fov_deg / 180.0 * M_PI) / nrm->r0;
    const double H = atan(tan(V));
    s->norm.inv_h = 1.0 / H;
    s->norm.inv_v = 1.0 / V;
    s->norm.spin_scale = 2.0 / nrm->spin_max;
    s->norm.spin_shift = -1.0;
    s->norm.q_scale = 1.0 / nrm->q_max;
    s->norm.th_scale = 2.0 / (nrm->theta0_max - nrm->theta0_min);
    s->norm.th_shift = -(nrm->theta0_max + nrm->theta0_min) / (nrm->theta0_max - nrm->theta0_min);
    int64_t off = 0;
    std::vector<int64_t> offs;
    std::vector<float> scales;
    std::vector<uint8_t> decay;
    for (int l = 0; l < N_LAYERS; l++) {
        s->w_off[l] = off;
        offs.push_back(off);
        // LeCun-normal weights (the 6 zero-padded input columns do not count)
        const int fan_in = l == 0 ? 10 : IN_DIM[l];
        scales.push_back((float)(1.0 / sqrt((double)fan_in)));
        off += (int64_t)OUT_DIM[l] * IN_DIM[l];
        s->b_off[l] = off;
        offs.push_back(off);
        scales.push_back(0.0f);
        off += OUT_DIM[l];
    }
    s->n_params = off;
    decay.assign(off, 0);
    for (int l = 0; l < N_LAYERS; l++)
        for (int64_t i = s->w_off[l]; i < s->b_off[l]; i++) decay[i] = 1;
    int64_t *d_offs = nullptr;
    float *d_scales = nullptr;
    cudaError_t e = cudaMalloc(&s->p, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s->g, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s->m, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s->v, off * sizeof(float));
    int64_t off3 = 0;
    for (int l = 0; l < N_LAYERS; l++) {
        s->w3_off[l] = off3;
        off3 += (int64_t)OUT_DIM[l] * 3 * IN_DIM[l];
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->w3, off3 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&s->WT, off * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&s->decay, off);
    if (e == cudaSuccess) e = cudaMalloc(&s->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&d_offs, offs.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_scales, scales.size() * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpy(d_offs, offs.data(), offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_scales, scales.data(), scales.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->decay, decay.data(), off, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s->m, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(s->v, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(s->err, 0, sizeof(int));
    if (e == cudaSuccess) {
        init_params_kernel<<<blocks_for(off), 256>>>(s->p, off, d_offs, d_scales, (int)offs.size(), seed);
        e = refresh_copies(s, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(d_offs);
    cudaFree(d_scales);
    if (e != cudaSuccess) {
        gt_surrogate_destroy(s);
        return e == cudaErrorMemoryAllocation ? GT_ERR_OOM : GT_ERR_CUDA;
    }
    *out = s;
    return GT_OK;
}

int gt_surrogate_destroy(gt_surrogate *s)
{
    if (!s) return GT_ERR_INVALID_ARG;
    Dev d(s->device);
    cudaDeviceSynchronize();
    free_ws(s);
    cudaFree(s->p);
    cudaFree(s->g);
    cudaFree(s->m);
    cudaFree(s->v);
    cudaFree(s->w3);
    cudaFree(s->WT);
    cudaFree(s->decay);
    cudaFree(s->loss);
    cudaFree(s->err);
    delete s;
    return GT_OK;
}

int gt_surrogate_get_params(gt_surrogate *s, float *host, int64_t n)
{
    if (!s || !host || n != s->n_params) return GT_ERR_INVALID_ARG;
    Dev d(s->device);
    return cudaMemcpy(host, s->p, n * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? GT_OK
                                                                                           : GT_ERR_CUDA;
}

int gt_surrogate_get_grads(gt_surrogate *s, float *host, int64_t n)
{
    if (!s || !host || n != s->n_params) return GT_ERR_INVALID_ARG;
    Dev d(s->device);
    return cudaMemcpy(host, s->g, n * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? GT_OK
                                                                                           : GT_ERR_CUDA;
}

int gt_surrogate_set_params(gt_surrogate *s, const float *host, int64_t n)
{
    if (!s || !host || n != s->n_params) return GT_ERR_INVALID_ARG;
    Dev d(s->device);
    cudaError_t e = cudaMemcpy(s->p, host, n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = refresh_copies(s, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? GT_OK : GT_ERR_CUDA;
}

int gt_surrogate_eval(gt_ctx *ctx, gt_surrogate *s, int64_t n, const double *alpha,
                      const double *beta, const double *spin, const double *q,
                      const double *theta0, float *out)
{
    if (!ctx || !s || n < 0 || !alpha || !beta || !spin || !q || !theta0 || !out)
        return GT_ERR_INVALID_ARG;
    Dev d(s->device);
    cudaStream_t st = gt_internal_stream(ctx);
    const int64_t chunk = 1 << 18;
    int rc = ensure_ws(s, n < chunk ? (n > 0 ? n : 1) : chunk);
    if (rc != GT_OK) return rc;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t B = n - r0 < chunk ? n - r0 : chunk;
        features_kernel<<<blocks_for(B), 256, 0, st>>>(B, r0, alpha, beta, spin, q, theta0, s->norm,
                                                       s->X[0]);
        cudaError_t e = forward(s, (int)B, st, false);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(out + r0 * 4, 4 * sizeof(float), s->Z[N_LAYERS - 1], 16 * sizeof(float),
                                  4 * sizeof(float), B, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return GT_ERR_CUDA;
    }
    return check_err(s, st);
}

int gt_surrogate_grad(gt_ctx *ctx, gt_surrogate *s, int64_t n, const double *alpha,
                      const double *beta, const double *spin, const double *q,
                      const double *theta0, const uint8_t *status, const double *th_end,
                      const double *ph_end, float dir_weight, float *grads_host, float *loss_host)
{
    if (!ctx || !s || n < 1 || n > (1 << 20) || !grads_host || !loss_host) return GT_ERR_INVALID_ARG;
    Dev d(s->device);
    cudaStream_t st = gt_internal_stream(ctx);
    int rc = ensure_ws(s, n);
    if (rc != GT_OK) return rc;
    features_kernel<<<blocks_for(n), 256, 0, st>>>(n, 0, alpha, beta, spin, q, theta0, s->norm, s->X[0],
                                                   s->XT[0]);
    labels_kernel<<<blocks_for(n), 256, 0, st>>>(n, 0, status, th_end, ph_end, s->lab);
    cudaError_t e = cudaMemsetAsync(s->loss, 0, sizeof(float), st);
    if (e == cudaSuccess) e = forward(s, (int)n, st);
    if (e == cudaSuccess) e = backward(s, (int)n, dir_weight, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grads_host, s->g, s->n_params * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss_host, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return GT_ERR_CUDA;
    rc = check_err(s, st);
    if (rc == GT_OK) *loss_host /= (float)n;
    return rc;
}

int gt_surrogate_train(gt_ctx *ctx, gt_surrogate *s, const gt_train_cfg *cfg, int64_t n,
                       const double *alpha, const double *beta, const double *spin,
                       const double *q, const double *theta0, const uint8_t *status,
                       const double *th_end, const double *ph_end, float *loss_per_epoch)
{
    if (!ctx || !s || !cfg || n < 1 || cfg->epochs < 1 || cfg->batch < 128 || cfg->batch % 128 ||
        cfg->batch > (1 << 20) || !(cfg->lr > 0))
        return GT_ERR_INVALID_ARG;
    Dev d(s->device);
    cudaStream_t st = gt_internal_stream(ctx);
    const int B = cfg->batch;
    int rc = ensure_ws(s, B);
    if (rc != GT_OK) return rc;
    const int64_t nb = n / B; // full batches only
    if (nb < 1) return GT_ERR_INVALID_ARG;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < cfg->epochs; ep++) {
        cudaError_t e = cudaMemsetAsync(s->loss, 0, sizeof(float), st);
        // cosine learning-rate schedule over the whole run
        for (int64_t b = 0; b < nb && e == cudaSuccess; b++) {
            const double prog = ((double)ep * nb + b) / ((double)cfg->epochs * nb);
            const float lr = (float)(cfg->lr * 0.5 * (1.0 + cos(M_PI * prog)));
            features_kernel<<<blocks_for(B), 256, 0, st>>>(B, b * B, alpha, beta, spin, q, theta0,
                                                           s->norm, s->X[0], s->XT[0]);
            labels_kernel<<<blocks_for(B), 256, 0, st>>>(B, b * B, status, th_end, ph_end, s->lab);
            e = forward(s, B, st);
            if (e == cudaSuccess) e = backward(s, B, (float)cfg->dir_weight, st);
            if (e != cudaSuccess) break;
            s->step++;
            const float bc1 = 1.0f - powf(b1, (float)s->step), bc2 = 1.0f - powf(b2, (float)s->step);
            adamw_kernel<<<blocks_for(s->n_params), 256, 0, st>>>(s->n_params, s->p, s->g, s->m, s->v,
                                                                  lr, b1, b2, eps,
                                                                  (float)cfg->weight_decay, bc1, bc2,
                                                                  s->decay);
            e = refresh_copies(s, st);
        }
        if (e != cudaSuccess) return GT_ERR_CUDA;
        if (loss_per_epoch) {
            float l = 0;
            e = cudaMemcpyAsync(&l, s->loss, sizeof l, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return GT_ERR_CUDA;
            loss_per_epoch[ep] = l / (float)(nb * B);
        }
    }
    return check_err(s, st);
}

} // extern "C"

// Inference with gating (declared in geotrace.h); needs the context's camera, so it is
// implemented next to the context in capi.cu through these helpers.
namespace gt {
namespace sg {

// The network on every pixel of the camera; its answers to `net` (float4 per pixel).
int net_pass(gt_surrogate *s, const CamDesc *d_cam, int64_t n_pix, float4 *net, cudaStream_t st)
{
    const int64_t chunk = 1 << 19;
    int rc = ensure_ws(s, n_pix < chunk ? n_pix : chunk);
    if (rc != GT_OK) return rc;
    for (int64_t p0 = 0; p0 < n_pix; p0 += chunk) {
        const int64_t B = n_pix - p0 < chunk ? n_pix - p0 : chunk;
        camera_features_kernel<<<blocks_for(B), 256, 0, st>>>(B, p0, d_cam, s->norm, s->X[0]);
        if (forward(s, (int)B, st, false) != cudaSuccess) return GT_ERR_CUDA;
        net_out_kernel<<<blocks_for(B), 256, 0, st>>>(B, p0, s->Z[N_LAYERS - 1], net);
        if (cudaGetLastError() != cudaSuccess) return GT_ERR_CUDA;
    }
    return check_err(s, st);
}

int select_first(const CamDesc *d_cam, int64_t n_pix, const float4 *net, const ProbeGrid &pg,
                 float tau, double band, double axis, float dir_tol, int64_t *list,
                 unsigned long long *count, cudaStream_t st)
{
    select_kernel<<<blocks_for(n_pix), 256, 0, st>>>(n_pix, d_cam, net, pg, tau, band, axis,
                                                     dir_tol, list, count);
    return cudaGetLastError() == cudaSuccess ? GT_OK : GT_ERR_CUDA;
}

int probe_records(const CamDesc *d_cam, const ProbeGrid &pg, const float4 *net,
                  const uint8_t *status, const double *th, const double *ph, ProbeRec *rec,
                  cudaStream_t st)
{
    const int n = pg.nx * pg.ny;
    probe_record_kernel<<<blocks_for(n), 256, 0, st>>>(d_cam, pg, net, status, th, ph, rec);
    return cudaGetLastError() == cudaSuccess ? GT_OK : GT_ERR_CUDA;
}

int gate_rest(const CamDesc *d_cam, int64_t n_pix, const float4 *net, const ProbeGrid &pg,
              float tau, double band, double axis, float dir_tol, double *t, double *r, double *th,
              double *ph, uint8_t *status, uint32_t *nsteps, int64_t *list,
              unsigned long long *count, cudaStream_t st)
{
    gate_kernel<<<blocks_for(n_pix), 256, 0, st>>>(n_pix, d_cam, net, pg, tau, band, axis, dir_tol,
                                                   t, r, th, ph, status, nsteps, list, count);
    return cudaGetLastError() == cudaSuccess ? GT_OK : GT_ERR_CUDA;
}

} // namespace sg
} // namespace gt
