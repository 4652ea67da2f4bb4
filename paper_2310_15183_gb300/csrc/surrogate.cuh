// surrogate.cuh -- shared definitions of the surrogate network (device and host).
#pragma once

#include <stdint.h>

namespace gt {
namespace sg {

// Feature normalisation: x0 = alpha inv_h, x1 = beta inv_v, x2 = (a/M) spin_scale + spin_shift,
// x3 = q q_scale, x4 = theta0 th_scale + th_shift (all near [-1, 1] over the training ranges).
struct Norm {
    double inv_h, inv_v, spin_scale, spin_shift, q_scale, th_scale, th_shift;
};

// Integrator probes of gated inference: pixels (k stride, l stride) (the last column and
// row included) traced exactly; per probe the network's error vector (exact end direction
// minus the predicted one) and both classifications.
struct ProbeRec {
    float err[3];
    uint8_t exact;   // integrator status
    uint8_t net_esc; // network predicts escape (logit > 0)
    uint8_t pad[2];
};

struct ProbeGrid {
    int stride;  // 0 = no probes
    int nx, ny;  // probes per row and per column
    float tol;   // largest accepted spread of the error vectors over a cell's corners
    const ProbeRec *rec; // ny x nx, row-major
};

constexpr int N_LAYERS = 5;
constexpr int IN_DIM[N_LAYERS] = {16, 256, 256, 256, 256};
constexpr int OUT_DIM[N_LAYERS] = {256, 256, 256, 256, 16};

} // namespace sg
} // namespace gt
