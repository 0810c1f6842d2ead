// Exact fixed-point slicing of the tensor-core stage 5 (see covmv_tcx.cu): a kernel value g
// with |g| <= 1 becomes digits a_s on the grids 2^-8(s+1) (|a_0|, |a_3| <= 256, the others
// <= 128), stored as the bfloat16 slices a_s 2^-8(s+1); a scaled right-hand-side value x = u / sigma with |x| <= 1 becomes digits b_t
// stored as b_t 2^-8t.  Every step is exact, so the slices sum to the value up to the dropped
// remainder.  Host builds of the same code let the exactness be checked without a GPU.
#pragma once

#include <cmath>

#include "df64.cuh"

namespace kl {
namespace tcs {

// x rounded to the grid 2^-k (|x| < 2^(22-k)) by the shifter 1.5 * 2^(23-k), and the exact
// remainder: the slice a 2^-k of digit a
KL_HD float digit(float& x, float shifter) {
    const float p = df::sub(df::add(x, shifter), shifter);
    x = df::sub(x, p);
    return p;
}

// six slices a_s 2^(-8(s+1)) of a double-float g with |g| <= 1; the tail joins the remainder
// after the three head digits
KL_HD void slices6(df::F2 g, float* out) {
    float x = g.h;
    out[0] = digit(x, 49152.f);                     // 1.5 * 2^15: grid 2^-8
    out[1] = digit(x, 192.f);                       // grid 2^-16
    out[2] = digit(x, 0.75f);                       // grid 2^-24
    x = df::add(x, g.l);                            // |x| <= 2^-25 after three digits
    out[3] = digit(x, 0.0029296875f);               // 1.5 * 2^-9: grid 2^-32
    out[4] = digit(x, 1.1444091796875e-05f);        // 1.5 * 2^-17: grid 2^-40
    out[5] = digit(x, 4.4703483581542969e-08f);     // 1.5 * 2^-25: grid 2^-48
}

// three slices of a float g with |g| <= 1
KL_HD void slices3(float g, float* out) {
    float x = g;
    out[0] = digit(x, 49152.f);
    out[1] = digit(x, 192.f);
    out[2] = digit(x, 0.75f);
}

// S slices b_t 2^-8t of a scaled right-hand-side value x (|x| <= 1): b_t = round(256 x_t) with
// x_{t+1} = 256 x_t - b_t, every step exact in float64, |b_0| <= 256 and |b_t| <= 128 after
template <int S>
KL_HD void u_slices(double x, float* out) {
    double w = 1.0;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const double p = rint(x * 256.0);
        x = fma(x, 256.0, -p);   // exact
        out[q] = float(p * w);   // |p| <= 256: exact in bfloat16 after scaling
        w *= 0.00390625;
    }
}

// acc += x for a float x (exact two-sum into the head, tail accumulated): the drain of a level
// accumulator into a row's double-float sum
KL_HD void df_acc(df::F2& acc, float x) {
    const df::F2 s = df::two_sum(acc.h, x);
    acc.h = s.h;
    acc.l = df::add(acc.l, s.l);
}

}  // namespace tcs
}  // namespace kl
