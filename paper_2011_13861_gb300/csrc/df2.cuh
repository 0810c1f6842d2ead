// Double-float arithmetic on pairs of values at once: the two float32 lanes of a 64-bit register
// pair go through one packed instruction (add/sub/mul/fma .rn.f32x2, Blackwell), each lane
// rounded exactly as the scalar float32 operation.  Every function below performs, lane by lane,
// the same operations in the same order as its scalar counterpart in df64.cuh (negations folded
// into exact sign flips, Fast2Sum on ordered operands replaced by TwoSum, which yields the same
// unique sum and error), so the results are bit-identical to evaluating the two values one
// after the other; kl_df2_selftest checks that on the GPU.
//
// The FMA pipe's throughput is the same for packed and scalar instructions; what a pair saves is
// issue slots, which bound the tensor-core float64-class producers (about 190 float32
// instructions per kernel value, most of them these add/sub/mul/fma).  The steps that have no
// packed form (table lookups, the exponent of 2^-m, the clamp) run per lane.
#pragma once

#include "df64.cuh"

namespace kl {
namespace df2 {

struct V {
    unsigned long long x;   // low half: first value, high half: second
};

__device__ __forceinline__ V mk(float a, float b) {
    V r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.x) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ V dup(float a) { return mk(a, a); }
__device__ __forceinline__ float lo(V a) { return __uint_as_float(unsigned(a.x)); }
__device__ __forceinline__ float hi(V a) { return __uint_as_float(unsigned(a.x >> 32)); }

__device__ __forceinline__ V add(V a, V b) {
    V r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.x) : "l"(a.x), "l"(b.x));
    return r;
}
__device__ __forceinline__ V sub(V a, V b) {
    V r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.x) : "l"(a.x), "l"(b.x));
    return r;
}
__device__ __forceinline__ V mul(V a, V b) {
    V r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.x) : "l"(a.x), "l"(b.x));
    return r;
}
__device__ __forceinline__ V fma_(V a, V b, V c) {
    V r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.x) : "l"(a.x), "l"(b.x), "l"(c.x));
    return r;
}
__device__ __forceinline__ V neg(V a) { return V{a.x ^ 0x8000000080000000ull}; }

// A product that an addition or subtraction then consumes, lane by lane in scalar float32.
// The code generator (CUDA 13.0) fuses a packed mul.rn.f32x2 whose result a packed add/sub
// uses into one packed FMA, although the explicit rounding modifier asks it not to contract:
// the sum then skips the product's rounding and differs in the last bit from the scalar code
// (measured on GB300 by kl_df2_selftest).  Scalar mul.rn.f32 is not fused.
__device__ __forceinline__ V mul_nc(V a, V b) { return mk(__fmul_rn(lo(a), lo(b)), __fmul_rn(hi(a), hi(b))); }

struct P {
    V h, l;   // two double-float values: (lo(h) + lo(l), hi(h) + hi(l))
};

__device__ __forceinline__ P two_sum(V a, V b) {
    const V s = add(a, b);
    const V bb = sub(s, a);
    const V e = add(sub(a, sub(s, bb)), sub(b, bb));
    return {s, e};
}

// two_sum(a, -b) of df64.cuh, written with subtractions (every operation negated exactly)
__device__ __forceinline__ P two_diff(V a, V b) {
    const V s = sub(a, b);
    const V bb = sub(s, a);
    const V e = sub(sub(a, sub(s, bb)), add(b, bb));
    return {s, e};
}

__device__ __forceinline__ P fast_two_sum(V a, V b) {
    const V s = add(a, b);
    const V e = sub(b, sub(s, a));
    return {s, e};
}

__device__ __forceinline__ P two_prod(V a, V b) {
    const V p = mul(a, b);
    const V e = fma_(a, b, neg(p));
    return {p, e};
}

__device__ __forceinline__ P add(P a, P b) {
    const P s = two_sum(a.h, b.h);
    const V e = add(s.l, add(a.l, b.l));
    return fast_two_sum(s.h, e);
}

// lanes where `lane_mask` is all ones take b, the others a (whole 64-bit words: no half is
// rewritten on its own)
__device__ __forceinline__ V select(unsigned long long lane_mask, V a, V b) {
    return V{(a.x & ~lane_mask) | (b.x & lane_mask)};
}

// all-ones in the lanes whose value satisfies `pred`
template <typename Pred>
__device__ __forceinline__ unsigned long long lanes(V a, Pred pred) {
    return (pred(lo(a)) ? 0x00000000FFFFFFFFull : 0ull) | (pred(hi(a)) ? 0xFFFFFFFF00000000ull : 0ull);
}

__device__ __forceinline__ P abs(P a) {
    // per lane: the sign of the head decides both parts (an exact sign flip of both)
    const unsigned long long sign = a.h.x & 0x8000000080000000ull;
    return {V{a.h.x ^ sign}, V{a.l.x ^ sign}};
}

// df64.cuh diff: heads and tails of grid-form coordinates
__device__ __forceinline__ P diff(V ah, V al, V bh, V bl) { return fast_two_sum(sub(ah, bh), sub(al, bl)); }

// df64.cuh sum_sq3; the two ordered Fast2Sums become TwoSums (same sum, same exact error)
__device__ __forceinline__ P sum_sq3(P a, P b, P c) {
    const P pa = two_prod(a.h, a.h), pb = two_prod(b.h, b.h), pc = two_prod(c.h, c.h);
    const V ea = fma_(add(a.h, a.h), a.l, pa.l);
    const V eb = fma_(add(b.h, b.h), b.l, pb.l);
    const V ec = fma_(add(c.h, c.h), c.l, pc.l);
    const P s1 = two_sum(pa.h, pb.h);
    const P s2 = two_sum(s1.h, pc.h);
    const V t = add(add(s1.l, s2.l), add(add(ea, eb), ec));
    return fast_two_sum(s2.h, t);
}

// df64.cuh sqrt (seeds per lane from MUFU rsqrt); a zero or negative head gives 0 in its lane
__device__ __forceinline__ P sqrt(P a, V seed) {
    V y = seed;
    y = mul(y, fma_(mul(dup(-0.5f), a.h), mul(y, y), dup(1.5f)));
    const V r0 = mul(a.h, y);
    const P p = two_prod(r0, r0);
    const V d = add(sub(sub(a.h, p.h), p.l), a.l);
    const V c = mul_nc(d, mul(dup(0.5f), y));
    const P r = fast_two_sum(r0, c);
    const unsigned long long keep = ~lanes(a.h, [](float v) { return v <= 0.f; });
    return {V{r.h.x & keep}, V{r.l.x & keep}};
}

// df64.cuh exp_neg: e^(-x) for two double-floats x >= 0 (Tang's method, the same constants)
__device__ __forceinline__ P exp_neg(P x, const float* tab_h, const float* tab_l) {
    const float c1 = 0.0108299255371093750f;
    const float c2 = 4.9915911404241342e-07f;
    const float c3 = 2.5728046402313451e-14f;
    const float inv_step = 92.332482616893656f;
    const float shifter = 12582912.f;
    {
        const unsigned long long big = lanes(x.h, [](float v) { return v > 44.f; });
        x = {select(big, x.h, dup(44.f)), V{x.l.x & ~big}};
    }
    const V tn = fma_(x.h, dup(inv_step), dup(shifter));
    const V nf = sub(tn, dup(shifter));
    const int n0 = __float_as_int(lo(tn)) - 0x4B400000, n1 = __float_as_int(hi(tn)) - 0x4B400000;
    const V a = fma_(nf, dup(-c1), x.h);
    const P t = fast_two_sum(a, x.l);
    const P q = two_prod(nf, dup(c2));
    const P b = two_diff(t.h, q.h);
    const V bl = sub(add(b.l, t.l), add(q.l, mul_nc(nf, dup(c3))));
    const P r = fast_two_sum(b.h, bl);
    const V c = neg(r.h), sl = neg(r.l);
    const P c2p = two_prod(c, c);
    V f = fma_(c, dup(1.0f / 120.0f), dup(1.0f / 24.0f));
    f = fma_(c, f, dup(1.0f / 6.0f));
    const V u = mul(mul(c2p.h, c), f);
    const P h = fast_two_sum(c, mul(dup(0.5f), c2p.h));
    const V lw = add(add(h.l, fma_(c, sl, sl)), fma_(dup(0.5f), c2p.l, u));
    const P Pm = fast_two_sum(h.h, lw);
    const int j0 = n0 & 63, j1 = n1 & 63;
    const V th = mk(tab_h[j0], tab_h[j1]), tl = mk(tab_l[j0], tab_l[j1]);
    const V tph = mul_nc(th, Pm.h);   // two_prod(th, Pm.h); its head then joins a sum
    const P tp{tph, fma_(th, Pm.h, neg(tph))};
    const V tpe = fma_(th, Pm.l, fma_(tl, Pm.h, tp.l));
    P R = fast_two_sum(th, tp.h);
    R.l = add(R.l, add(tl, tpe));
    R = fast_two_sum(R.h, R.l);
    const V scale = mk(__int_as_float((127 - (n0 >> 6)) << 23), __int_as_float((127 - (n1 >> 6)) << 23));
    return {mul(R.h, scale), mul(R.l, scale)};
}

// df64.cuh kernel_df for the kernels the tensor-core producers evaluate in pairs (exponential,
// Gaussian, separable exponential): r = the row point's {xh, yh, zh, xl, yl, zl} in both lanes,
// c = the two column points' coordinates lane by lane
template <int KIND>
__device__ __forceinline__ P kernel_df(const V* r, const V* c, const float* th, const float* tl) {
    const P dx = diff(r[0], r[3], c[0], c[3]);
    const P dy = diff(r[1], r[4], c[1], c[4]);
    const P dz = diff(r[2], r[5], c[2], c[5]);
    if (KIND == KL_K_EXP_SEPARABLE) return exp_neg(add(add(abs(dx), abs(dy)), abs(dz)), th, tl);
    const P s = sum_sq3(dx, dy, dz);
    if (KIND == KL_K_GAUSS) return exp_neg(s, th, tl);
    float s0, s1;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(s0) : "f"(fmaxf(lo(s.h), 1e-30f)));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(s1) : "f"(fmaxf(hi(s.h), 1e-30f)));
    return exp_neg(sqrt(s, mk(s0, s1)), th, tl);
}

// kernel32.cuh kernel values for two columns (float32 class, coordinates pre-scaled so that one
// MUFU ex2 gives the exponential): the differences and squares packed, the MUFU steps per lane
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KIND>
__device__ __forceinline__ V kernel32(V dx, V dy, V dz) {
    if (KIND == KL_K_EXP_SEPARABLE) {
        const unsigned long long m = 0x7FFFFFFF7FFFFFFFull;   // |.| of both lanes
        const V s = add(add(V{dx.x & m}, V{dy.x & m}), V{dz.x & m});
        return mk(ex2_approx(-lo(s)), ex2_approx(-hi(s)));
    }
    const V s = fma_(dz, dz, fma_(dy, dy, mul(dx, dx)));
    if (KIND == KL_K_GAUSS) return mk(ex2_approx(-lo(s)), ex2_approx(-hi(s)));
    const float s0 = fmaxf(lo(s), 1e-30f), s1 = fmaxf(hi(s), 1e-30f);
    return mk(ex2_approx(-s0 * rsqrt_approx(s0)), ex2_approx(-s1 * rsqrt_approx(s1)));
}

// tc_slices.cuh digit and slices6 on pairs
__device__ __forceinline__ V digit(V& x, float shifter) {
    const V sh = dup(shifter);
    const V p = sub(add(x, sh), sh);
    x = sub(x, p);
    return p;
}

__device__ __forceinline__ void slices6(P g, V* out) {
    V x = g.h;
    out[0] = digit(x, 49152.f);
    out[1] = digit(x, 192.f);
    out[2] = digit(x, 0.75f);
    x = add(x, g.l);
    out[3] = digit(x, 0.0029296875f);
    out[4] = digit(x, 1.1444091796875e-05f);
    out[5] = digit(x, 4.4703483581542969e-08f);
}

// tc_slices.cuh slices3 on pairs
__device__ __forceinline__ void slices3(V g, V* out) {
    V x = g;
    out[0] = digit(x, 49152.f);
    out[1] = digit(x, 192.f);
    out[2] = digit(x, 0.75f);
}

// tc_slices.cuh df_acc for two sums at once: acc += x, then the final renormalisation
__device__ __forceinline__ void acc_add(P& acc, V x) {
    const P s = two_sum(acc.h, x);
    acc.h = s.h;
    acc.l = add(acc.l, s.l);
}

}  // namespace df2
}  // namespace kl
