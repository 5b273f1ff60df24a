// bsi_weights.cuh -- per-offset cubic B-spline weights in constant memory.
//
// With integer spacing d the fractional offset u of Eq. 1 (Sec. 2.1) takes
// only the d values r/d, r = 0..d-1, so the four weights B_0..B_3 of every
// offset are tabulated once (Sec. 3.4: look-up tables of the scalar B-spline
// coefficients).  The table covers every spacing 1..64; the weights of
// spacing d start at weight_base(d) = 2d(d-1), four per offset r.
//
// Values are computed at compile time in FP64 from the uniform cubic B-spline
// polynomials and rounded once to FP32, so the table needs no run-time set-up
// and a compile-time spacing turns every weight into a constant-bank operand.
#pragma once

#include "bsi_geometry.h"

namespace bsi {

struct WeightTable {
    float w[kWeightCount];
};

constexpr WeightTable make_weight_table() {
    WeightTable t{};
    for (int d = 1; d <= kMaxSpacing; ++d) {
        for (int r = 0; r < d; ++r) {
            const double u = static_cast<double>(r) / static_cast<double>(d);
            const double om = 1.0 - u;
            // B_0 = (1-u)^3/6, B_1 = (3u^3 - 6u^2 + 4)/6,
            // B_2 = (-3u^3 + 3u^2 + 3u + 1)/6, B_3 = u^3/6
            const double b0 = om * om * om / 6.0;
            const double b1 = ((3.0 * u - 6.0) * u * u + 4.0) / 6.0;
            const double b2 = (((-3.0 * u + 3.0) * u + 3.0) * u + 1.0) / 6.0;
            const double b3 = u * u * u / 6.0;
            const int o = weight_base(d) + 4 * r;
            t.w[o + 0] = static_cast<float>(b0);
            t.w[o + 1] = static_cast<float>(b1);
            t.w[o + 2] = static_cast<float>(b2);
            t.w[o + 3] = static_cast<float>(b3);
        }
    }
    return t;
}

// One copy in the constant bank of every translation unit that includes this header.
static __constant__ WeightTable c_lut = make_weight_table();

}  // namespace bsi
