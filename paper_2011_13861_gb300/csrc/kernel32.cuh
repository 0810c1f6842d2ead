// Float32 kernel values Gamma(x_k, x_l)/sigma^2 from float32 coordinates pre-scaled so that one
// ex2.approx gives the exponential (exp, separable exp: log2(e)/L; Gaussian: sqrt(log2(e))/L),
// MUFU rsqrt for the distance; the polynomial test kernel from unscaled coordinates.
#pragma once

#include "kl_internal.h"

namespace kl {

template <int KIND>
__device__ __forceinline__ float kernel32(float dx, float dy, float dz, float x0, float y0, float z0,
                                          float x1, float y1, float z1, int pm) {
    if (KIND == KL_K_EXP) {
        float s = fmaxf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), 1e-30f);
        float rs, g;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(s));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(-s * rs));
        return g;
    } else if (KIND == KL_K_GAUSS) {
        float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        float g;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(-s));
        return g;
    } else if (KIND == KL_K_EXP_SEPARABLE) {
        float g;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(-(fabsf(dx) + fabsf(dy) + fabsf(dz))));
        return g;
    } else {
        float f = fmaf(x0, x1, 1.f) * fmaf(y0, y1, 1.f) * fmaf(z0, z1, 1.f), r = 1.f;
        for (int i = 0; i < pm; ++i) r *= f;
        return r;
    }
}

// Packed float32 pairs (fma.rn.f32x2): one instruction performs two IEEE float32 FMAs, each
// rounded exactly as fmaf, on the two halves of 64-bit registers (low half = first element).
// The FMA pipe's throughput is the same as for scalar FFMA (measured: kl_pipe_rates), but one
// issue slot serves two FMAs, which is what the issue-bound float32 stage-5 loop is short of.
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long f2_dup(float g) {
    unsigned long long d;
    asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(g));
    return d;
}

__device__ __forceinline__ float f2_lo(unsigned long long x) { return __uint_as_float(unsigned(x)); }
__device__ __forceinline__ float f2_hi(unsigned long long x) { return __uint_as_float(unsigned(x >> 32)); }

}  // namespace kl
