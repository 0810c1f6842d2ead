// Host build of the float64 stage-5 kernel's exponential and square root, checked against long
// double.  The device draws the square root's seed from an approximate reciprocal square root;
// here the exact one is perturbed by up to 2^-21.  Prints one JSON object of maximum errors.
#include <cmath>
#include <cstdio>
#include <random>

#include "fp64_math.cuh"

int main() {
    double tab[1024];   // 2^(j/1024), as the library builds it on the host
    for (int j = 0; j < 1024; ++j) tab[j] = std::exp2(double(j) / 1024.0);
    std::mt19937_64 rng(2011);
    std::uniform_real_distribution<double> U(0.0, 1.0);

    // e^x on [-37, 0] (values above 1e-16 of the diagonal), relative; on [-745, -37] absolute
    double rel = 0, abs_tail = 0;
    int not_zero_below = 0;
    for (int i = 0; i < 400000; ++i) {
        const double x = (i % 4 == 0) ? -37.0 * U(rng) : (i % 4 == 1 ? -1e-3 * U(rng)
                         : (i % 4 == 2 ? -std::pow(10.0, -12 + 13.5 * U(rng)) : -37.0 - 708.0 * U(rng)));
        const double e = kl::f64::exp_nonpos(x, float(x), tab);
        const long double ref = expl((long double)x);
        if (x >= -37.0) rel = std::fmax(rel, (double)fabsl((e - ref) / ref));
        else abs_tail = std::fmax(abs_tail, (double)fabsl(e - ref));
        if (x < -700.5 && e != 0.0) ++not_zero_below;
    }
    // the argument's float copy may differ from x (the kernel passes the float32 distance)
    double rel_fx = 0;
    for (int i = 0; i < 200000; ++i) {
        const double x = -30.0 * U(rng);
        const float xf = float(x) * float(1.0 + (2 * U(rng) - 1) * 1e-6);
        const long double ref = expl((long double)x);
        rel_fx = std::fmax(rel_fx, (double)fabsl((kl::f64::exp_nonpos(x, xf, tab) - ref) / ref));
    }
    // sqrt from a seed with a relative error up to 2^-21 (the device seed is good to ~2^-22.9)
    double sq = 0, sqf = 0;
    for (int i = 0; i < 400000; ++i) {
        const double s = std::pow(10.0, -20 + 24 * U(rng));
        const float sf = std::fmax(float(s), 1e-30f);
        const float yf = float(1.0 / std::sqrt(double(sf))) * float(1.0 + (2 * U(rng) - 1) * std::ldexp(1.0, -21));
        float df;
        const double r = kl::f64::sqrt_from_seed(s, sf, yf, &df);
        const long double ref = sqrtl((long double)s);
        sq = std::fmax(sq, (double)fabsl((r - ref) / ref));
        sqf = std::fmax(sqf, (double)fabsl((df - ref) / ref));
    }
    std::printf("{\"exp_rel\": %.6e, \"exp_abs_tail\": %.6e, \"exp_not_zero_below_700\": %d, "
                "\"exp_rel_float_index\": %.6e, \"sqrt_rel\": %.6e, \"sqrt_float_rel\": %.6e}\n",
                rel, abs_tail, not_zero_below, rel_fx, sq, sqf);
    return 0;
}
