// Host build of the double-float header's arithmetic (exp, sum of squares, grid-form point
// differences) checked against long double.  Prints one JSON object of maximum errors.
#include <cmath>
#include <cstdio>
#include <random>

#include "df64.cuh"

using namespace kl::df;

static long double val(F2 a) { return (long double)a.h + (long double)a.l; }
static F2 split(long double x) {
    const float h = (float)x;
    return {h, (float)(x - (long double)h)};
}

int main() {
    float th[64], tl[64];
    for (int j = 0; j < 64; ++j) {
        const long double t = exp2l(-(long double)j / 64);
        th[j] = (float)t;
        tl[j] = (float)(t - (long double)th[j]);
    }
    std::mt19937_64 rng(2011);
    std::uniform_real_distribution<double> U(0.0, 1.0);

    // e^-x for x in [0, 44]: uniform, small, and log-spread arguments
    double exp_rel = 0, exp_abs = 0;
    int exp_unnormalised = 0;
    for (int i = 0; i < 300000; ++i) {
        const long double x = (i % 3 == 0) ? U(rng) * 44 : (i % 3 == 1 ? U(rng) * 0.02 : std::pow(10.0, -8 + 9.6 * U(rng)));
        const F2 xf = split(x);
        const long double ref = expl(-val(xf));
        const F2 r = exp_neg(xf, th, tl);
        exp_rel = std::fmax(exp_rel, (double)fabsl((val(r) - ref) / ref));
        exp_abs = std::fmax(exp_abs, (double)fabsl(val(r) - ref));
        if (r.h != 0.f && std::fabs(r.l) > std::ldexp(1.0f, std::ilogb(r.h) - 24)) ++exp_unnormalised;
    }

    // grid-form coordinates in [-8, 8): heads on q = 2^-20, tails the remainders
    const double q = std::ldexp(1.0, 3 - 23);
    int inexact_heads = 0;
    double diff_abs = 0, sq_rel = 0;
    for (int i = 0; i < 300000; ++i) {
        const double scale = (i % 3 == 0) ? 1e-7 : (i % 3 == 1 ? 1e-3 : 1.0);
        F2 d[3];
        long double s = 0;
        for (int k = 0; k < 3; ++k) {
            const double a = U(rng) * 16 - 8;
            double b = a + (U(rng) * 2 - 1) * scale;
            if (std::fabs(b) >= 8) b = a;
            const double ah = std::rint(a / q) * q, bh = std::rint(b / q) * q;
            const float al = (float)(a - ah), bl = (float)(b - bh);
            const float hd = sub((float)ah, (float)bh);
            if ((double)hd != ah - bh) ++inexact_heads;
            d[k] = fast_two_sum(hd, sub(al, bl));   // the device difference of two grid-form points
            const long double exact = ((long double)ah + al) - ((long double)bh + bl);
            diff_abs = std::fmax(diff_abs, (double)fabsl(val(d[k]) - exact));
            s += val(d[k]) * val(d[k]);
        }
        const F2 ss = sum_sq3(d[0], d[1], d[2]);
        if (s > 0) sq_rel = std::fmax(sq_rel, (double)fabsl((val(ss) - s) / s));
    }
    // sqrt of a double-float from a float seed with a relative error up to 2^-21 (the device
    // seed is rsqrt.approx, good to about 2^-22.9)
    double sqrt_rel = 0;
    for (int i = 0; i < 300000; ++i) {
        const long double a = std::pow(10.0, -12 + 16 * U(rng));
        const F2 af = split(a);
        const float seed = (float)(1.0 / std::sqrt((double)af.h)) * (float)(1.0 + (2 * U(rng) - 1) * std::ldexp(1.0, -21));
        const F2 r = kl::df::sqrt(af, seed);
        const long double ref = sqrtl(val(af));
        sqrt_rel = std::fmax(sqrt_rel, (double)fabsl((val(r) - ref) / ref));
    }
    // float64 -> double-float by bit operations: magnitudes from 2^-72 to 2^127, both signs,
    // exact powers of two and values with few significant bits
    double split_rel = 0;
    int split_head_wrong = 0;
    for (int i = 0; i < 600000; ++i) {
        double x = std::ldexp(0.5 + 0.5 * U(rng), int(-71 + 198 * U(rng)));
        if (i % 7 == 1) x = -x;
        if (i % 11 == 2) x = std::ldexp(1.0, int(-72 + 199 * U(rng)));
        if (i % 13 == 3) x = std::ldexp(std::floor(U(rng) * 4096.0) + 1.0, int(-60 + 120 * U(rng)));
        const F2 f = split_double_bits(x);
        const long double v = (long double)f.h + (long double)f.l;
        split_rel = std::fmax(split_rel, (double)fabsl((v - (long double)x) / (long double)x));
        // the head is x truncated to 24 significant bits: |x - h| < ulp(h), same sign
        const long double r = (long double)x - (long double)f.h;
        if (fabsl(r) >= std::ldexp(std::fabs((double)f.h), -23) || (r != 0 && (r > 0) != (x > 0))) ++split_head_wrong;
    }
    const F2 z = split_double_bits(0.0), tiny = split_double_bits(1e-300), big = split_double_bits(-3e300);
    const int split_edges_ok = (z.h == 0.f && z.l == 0.f && tiny.h == 0.f && std::isinf(big.h) && big.h < 0) ? 1 : 0;
    std::printf("{\"exp_rel\": %.6e, \"exp_abs\": %.6e, \"exp_unnormalised\": %d, \"inexact_heads\": %d, "
                "\"diff_abs\": %.6e, \"sum_sq_rel\": %.6e, \"sqrt_rel\": %.6e, \"split_rel\": %.6e, "
                "\"split_head_wrong\": %d, \"split_edges_ok\": %d}\n",
                exp_rel, exp_abs, exp_unnormalised, inexact_heads, diff_abs, sq_rel, sqrt_rel, split_rel,
                split_head_wrong, split_edges_ok);
    return 0;
}
