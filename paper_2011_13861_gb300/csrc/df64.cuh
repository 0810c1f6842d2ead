// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two float32
// numbers with |lo| <= ulp(hi)/2, giving about 48 significant bits (the point coordinates are
// the exception: a grid form with larger tails, which `kernel_df` below differences exactly or
// renormalises).  Built from the
// error-free transformations of Knuth (TwoSum), Dekker (Fast2Sum) and the FMA-based exact
// product; the exponential follows Tang's table-driven method.
//
// GB300 executes float32 FMAs about 70x faster than float64 ones, so evaluating the kernel
// in df64 gives float64-level results (relative error ~1e-14) at a fraction of the cost of
// the float64 pipe.  Every operation below is written with explicit round-to-nearest
// intrinsics so the compiler cannot contract or reassociate them.
#pragma once

#if defined(__CUDACC__)
#include <cuda_runtime.h>

#include "kl.h"
#else
#include <cmath>
#endif

#if defined(__CUDACC__)
#define KL_HD __host__ __device__ __forceinline__
#else
#define KL_HD inline
#endif

namespace kl {
namespace df {

#if defined(__CUDA_ARCH__)
KL_HD float add(float a, float b) { return __fadd_rn(a, b); }
KL_HD float sub(float a, float b) { return __fsub_rn(a, b); }
KL_HD float mul(float a, float b) { return __fmul_rn(a, b); }
KL_HD float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
KL_HD float add(float a, float b) { volatile float r = a + b; return r; }
KL_HD float sub(float a, float b) { volatile float r = a - b; return r; }
KL_HD float mul(float a, float b) { volatile float r = a * b; return r; }
KL_HD float fma_(float a, float b, float c) { return __builtin_fmaf(a, b, c); }
#endif

struct F2 {
    float h, l;
};

// s + e == a + b exactly (Knuth)
KL_HD F2 two_sum(float a, float b) {
    float s = add(a, b);
    float bb = sub(s, a);
    float e = add(sub(a, sub(s, bb)), sub(b, bb));
    return {s, e};
}

// s + e == a + b exactly when |a| >= |b| or a == 0 (Dekker)
KL_HD F2 fast_two_sum(float a, float b) {
    float s = add(a, b);
    float e = sub(b, sub(s, a));
    return {s, e};
}

// p + e == a * b exactly
KL_HD F2 two_prod(float a, float b) {
    float p = mul(a, b);
    float e = fma_(a, b, -p);
    return {p, e};
}

KL_HD F2 add(F2 a, F2 b) {
    F2 s = two_sum(a.h, b.h);
    float e = add(s.l, add(a.l, b.l));
    return fast_two_sum(s.h, e);
}

KL_HD F2 sub(F2 a, F2 b) { return add(a, F2{-b.h, -b.l}); }

KL_HD F2 mul(F2 a, F2 b) {
    F2 p = two_prod(a.h, b.h);
    float e = fma_(a.h, b.l, p.l);
    e = fma_(a.l, b.h, e);
    return fast_two_sum(p.h, e);
}

KL_HD F2 abs(F2 a) { return a.h < 0.f ? F2{-a.h, -a.l} : a; }

// a^2 for a double-float a
KL_HD F2 sqr(F2 a) {
    F2 p = two_prod(a.h, a.h);
    float e = fma_(add(a.h, a.h), a.l, p.l);
    return fast_two_sum(p.h, e);
}

// sqrt(a), a >= 0: float32 reciprocal-square-root seed, one float32 Newton step, then one
// double-float Heron correction r = r0 + (a - r0^2) y / 2.  The correction is about 2^-22 of
// the root and y is good to about 2^-22.4 after the float step, so the root carries a relative
// error of about 2^-44.5 (4e-14 measured on the host against long double).
KL_HD F2 sqrt(F2 a, float rs_seed) {
    if (a.h <= 0.f) return F2{0.f, 0.f};
    float y = rs_seed;
    y = mul(y, fma_(mul(-0.5f, a.h), mul(y, y), 1.5f));
    float r0 = mul(a.h, y);
    F2 p = two_prod(r0, r0);
    float d = add(sub(sub(a.h, p.h), p.l), a.l);   // a - r0^2 (a.h - p.h exact: they are close)
    float c = mul(d, mul(0.5f, y));
    return fast_two_sum(r0, c);
}

// 2^(-j/64), j = 0..63, as double-float pairs (filled by the host)
struct ExpTable {
    float h[64], l[64];
};

// bit pattern of a float
KL_HD int float_bits(float x) {
#if defined(__CUDA_ARCH__)
    return __float_as_int(x);
#else
    int b;
    __builtin_memcpy(&b, &x, 4);
    return b;
#endif
}

// e^(-x) for a double-float x >= 0, Tang's method: n = round(64 x / ln2), j = n mod 64,
// m = n div 64, r = x - n ln2/64 (|r| <= ln2/128) in double-float, e^(-x) = 2^-m 2^(-j/64) e^(-r),
// e^(-r) - 1 by its Taylor polynomial (degree 5).  Arguments above 44 are clamped (the
// result, below 8e-20, then carries an absolute error below 1e-19).
KL_HD F2 exp_neg(F2 x, const float* tab_h, const float* tab_l) {
    // ln2/64 split into three floats: c1 has 12 significant bits, so n*c1 is exact for n < 4096
    const float c1 = 0.0108299255371093750f;          // 0x3C317000: 12-bit head of ln2/64
    const float c2 = 4.9915911404241342e-07f;         // next 24 bits
    const float c3 = 2.5728046402313451e-14f;         // remainder (|ln2/64 - c1 - c2 - c3| < 2e-22)
    const float inv_step = 92.332482616893656f;       // 64 / ln2
    const float shifter = 12582912.f;                 // 1.5 * 2^23: x + shifter keeps round(x) in its low bits
    if (x.h > 44.f) x = F2{44.f, 0.f};
    const float tn = fma_(x.h, inv_step, shifter);
    const float nf = sub(tn, shifter);
    const int n = float_bits(tn) - 0x4B400000;        // 0 <= n <= 4063
    // r = x - n*(c1 + c2 + c3) in double-float.  a is exact (Sterbenz) and, unless zero, a
    // multiple of ulp(x.h) (n*c1 lies on a grid of 2^-18), so |a| >= |x.l| and Fast2Sum is exact.
    float a = fma_(-nf, c1, x.h);
    F2 t = fast_two_sum(a, x.l);
    F2 q = two_prod(nf, c2);
    F2 b = two_sum(t.h, -q.h);
    float bl = add(add(b.l, t.l), -add(q.l, mul(nf, c3)));
    F2 r = fast_two_sum(b.h, bl);
    // s = -r ; e^s - 1 = s + s^2/2 + s^3/6 + s^4/24 + s^5/120
    const float c = -r.h, sl = -r.l;
    F2 c2p = two_prod(c, c);
    float f = fma_(c, 1.0f / 120.0f, 1.0f / 24.0f);
    f = fma_(c, f, 1.0f / 6.0f);
    float u = mul(mul(c2p.h, c), f);                  // s^3/6 + ... (float accuracy suffices)
    F2 h = fast_two_sum(c, mul(0.5f, c2p.h));          // |c| <= ln2/128, so |c| >= c^2/2
    float lo = add(add(h.l, fma_(c, sl, sl)), fma_(0.5f, c2p.l, u));
    F2 P = fast_two_sum(h.h, lo);                     // e^s - 1
    // 2^(-j/64) * (1 + P)
    const int j = n & 63;
    const float th = tab_h[j], tl = tab_l[j];
    F2 tp = two_prod(th, P.h);
    float tpe = fma_(th, P.l, fma_(tl, P.h, tp.l));
    F2 R = fast_two_sum(th, tp.h);
    R.l = add(R.l, add(tl, tpe));
    R = fast_two_sum(R.h, R.l);
    // 2^-m, m = n >> 6 in [0, 63]
    const int m = n >> 6;
    const int sbits = (127 - m) << 23;
#if defined(__CUDA_ARCH__)
    const float scale = __int_as_float(sbits);
#else
    float scale;
    __builtin_memcpy(&scale, &sbits, 4);
#endif
    return F2{mul(R.h, scale), mul(R.l, scale)};
}

// A float64 value as a double-float h + l by integer operations on its bit pattern (no float64
// instruction): h is the value truncated to 24 significant bits, l the rest truncated to 24, so
// h + l equals x to within 2^-47 |x|.  Magnitudes below 2^-73 (where l could leave the normal
// float range) or from 2^128 on use the float conversion instead.
KL_HD F2 split_double_bits(double x) {
    unsigned long long u;
#if defined(__CUDA_ARCH__)
    u = static_cast<unsigned long long>(__double_as_longlong(x));
#else
    __builtin_memcpy(&u, &x, 8);
#endif
    const unsigned sign = unsigned(u >> 32) & 0x80000000u;
    const int e = int((u >> 52) & 0x7FF) - 1023;
    if (e < -73 || e > 127) {
        const float h = float(x);
        return F2{h, float(x - double(h))};
    }
    const unsigned hb = sign | (unsigned(e + 127) << 23) | (unsigned(u >> 29) & 0x7FFFFFu);
    const unsigned m29 = unsigned(u) & 0x1FFFFFFFu;   // the 29 bits below h's last
    unsigned lb = 0;
    if (m29 != 0) {
#if defined(__CUDA_ARCH__)
        const int lz = __clz(int(m29)) - 3;             // leading zeros within the 29 bits
#else
        const int lz = __builtin_clz(m29) - 3;
#endif
        const int el = e - 52 + 28 - lz;                // exponent of l's leading bit
        lb = sign | (unsigned(el + 127) << 23) | (((m29 << lz) >> 5) & 0x7FFFFFu);   // el >= e - 52 >= -125
    }
    float h, l;
#if defined(__CUDA_ARCH__)
    h = __uint_as_float(hb);
    l = __uint_as_float(lb);
#else
    __builtin_memcpy(&h, &hb, 4);
    __builtin_memcpy(&l, &lb, 4);
#endif
    return F2{h, l};
}

// |a|^2 + |b|^2 + |c|^2 of three normalised double-floats: exact head squares, their sum by
// Fast2Sum on ordered (non-negative) operands, and one tail of the product errors, the cross
// terms 2 h l and the two sums' errors (the l^2 terms are below 2^-48 of the result).
KL_HD F2 sum_sq3(F2 a, F2 b, F2 c) {
    const F2 pa = two_prod(a.h, a.h), pb = two_prod(b.h, b.h), pc = two_prod(c.h, c.h);
    const float ea = fma_(add(a.h, a.h), a.l, pa.l);
    const float eb = fma_(add(b.h, b.h), b.l, pb.l);
    const float ec = fma_(add(c.h, c.h), c.l, pc.l);
    const F2 s1 = fast_two_sum(fmaxf(pa.h, pb.h), fminf(pa.h, pb.h));
    const F2 s2 = fast_two_sum(fmaxf(s1.h, pc.h), fminf(s1.h, pc.h));
    const float t = add(add(s1.l, s2.l), add(add(ea, eb), ec));
    return fast_two_sum(s2.h, t);
}

#if defined(__CUDACC__)
// ---- kernel values Gamma(x_k, x_l) in double-float (device only) ----

// a - b for two coordinates in the grid form of the double-float coordinate arrays: each
// head is a multiple of one power of two q with |head| <= 2^23 q, and each tail has |tail| <= q/2.
// The heads' difference (at most 2^24 q) is then exact, and unless it is zero it is at least q
// >= |al - bl|, so one Fast2Sum normalises the result.
__device__ __forceinline__ F2 diff(float ah, float al, float bh, float bl) {
    return fast_two_sum(sub(ah, bh), sub(al, bl));
}

template <int KIND>
__device__ __forceinline__ F2 kernel_df(const float* r, const float* c, int pm, const float* th,
                                        const float* tl) {
    // r, c: {xh, yh, zh, xl, yl, zl} of the row and column point
    if (KIND == KL_K_POLY_TEST) {
        F2 f{1.f, 0.f};
        for (int k = 0; k < 3; ++k) {
            // grid-form coordinates are not normalised: renormalise before multiplying
            F2 p = mul(two_sum(r[k], r[3 + k]), two_sum(c[k], c[3 + k]));
            f = mul(f, add(p, F2{1.f, 0.f}));
        }
        F2 g{1.f, 0.f};
        for (int i = 0; i < pm; ++i) g = mul(g, f);
        return g;
    }
    const F2 dx = diff(r[0], r[3], c[0], c[3]);
    const F2 dy = diff(r[1], r[4], c[1], c[4]);
    const F2 dz = diff(r[2], r[5], c[2], c[5]);
    if (KIND == KL_K_EXP_SEPARABLE) {
        F2 s = add(add(abs(dx), abs(dy)), abs(dz));
        return exp_neg(s, th, tl);
    }
    F2 s = sum_sq3(dx, dy, dz);
    if (KIND == KL_K_GAUSS) return exp_neg(s, th, tl);
    float seed;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(seed) : "f"(fmaxf(s.h, 1e-30f)));
    return exp_neg(sqrt(s, seed), th, tl);
}
#endif

}  // namespace df
}  // namespace kl
