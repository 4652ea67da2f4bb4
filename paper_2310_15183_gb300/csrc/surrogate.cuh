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

constexpr int N_LAYERS = 5;
constexpr int IN_DIM[N_LAYERS] = {16, 256, 256, 256, 256};
constexpr int OUT_DIM[N_LAYERS] = {256, 256, 256, 256, 16};

} // namespace sg
} // namespace gt
