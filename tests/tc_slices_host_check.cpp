// Host emulation of the tensor-core stage 5's exact slicing (csrc/tc_slices.cuh, the code the
// kernels run): kernel values and scaled right-hand sides cut into bfloat16 slices, the slice
// products summed per level in float32 over 128-column drain blocks (the tensor core's
// accumulators), the levels drained into a double-float row sum, all against long double.
// Prints one JSON object.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "tc_slices.cuh"

using kl::df::F2;

static bool bf16_exact(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    return (b & 0xffffu) == 0;
}

int main() {
    std::mt19937_64 rng(2011);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    // the float64 class: 6 x 6 slices, levels 0-3 exact, levels 4-5 in one accumulator, 21 products
    const int S[21] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5};
    const int T[21] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0};
    auto acc_of = [](int q) { return q == 0 ? 0 : q < 3 ? 1 : q < 6 ? 2 : q < 10 ? 3 : 4; };
    int not_bf16 = 0, inexact_levels = 0, big_digit = 0;
    double slice_rem = 0, rel64 = 0, rel32 = 0;
    const int blocks = 16, cols = 128;                 // 2048 columns, drained every 128
    for (int trial = 0; trial < 200; ++trial) {
        // a row of kernel values in (0, 1] (double-float) and one right-hand side with sigma
        static double g[blocks * cols], u[blocks * cols];
        double umax = 0;
        for (int j = 0; j < blocks * cols; ++j) {
            g[j] = std::exp(-6.0 * U(rng));
            u[j] = (2 * U(rng) - 1) * std::pow(10.0, -3 * U(rng));
            umax = std::fmax(umax, std::fabs(u[j]));
        }
        int e;
        std::frexp(umax, &e);
        const double sigma = std::ldexp(1.0, e);
        F2 row64{0.f, 0.f}, row32{0.f, 0.f};
        long double exact = 0, absum = 0, exact32 = 0;
        for (int b = 0; b < blocks; ++b) {
            float lev[5] = {0, 0, 0, 0, 0}, lev32[3] = {0, 0, 0};
            long double lev_exact[5] = {0, 0, 0, 0, 0};
            for (int j = b * cols; j < (b + 1) * cols; ++j) {
                const float gh = float(g[j]);
                const F2 gd{gh, float(g[j] - double(gh))};
                float a[6], bb[6], a3[3];
                kl::tcs::slices6(gd, a);
                kl::tcs::u_slices<6>(u[j] / sigma, bb);
                kl::tcs::slices3(gh, a3);
                long double sa = 0;
                for (int s = 0; s < 6; ++s) {
                    not_bf16 += !bf16_exact(a[s]) + !bf16_exact(bb[s]);
                    sa += (long double)a[s];
                    // digit bounds: 256 for the leading digits and for a_3, where the double-float
                    // tail joins the remainder; 128 elsewhere (round-to-nearest remainders)
                    const double dig_a = std::ldexp(a[s], 8 * (s + 1)), dig_b = std::ldexp(bb[s], 8 * s);
                    big_digit += (std::fabs(dig_a) > (s == 0 || s == 3 ? 256 : 128)) + (std::fabs(dig_b) > (s ? 128 : 256));
                }
                slice_rem = std::fmax(slice_rem, (double)fabsl(sa - ((long double)gd.h + gd.l)));
                for (int q = 0; q < 21; ++q) {
                    const float pr = a[S[q]] * bb[T[q]];   // exact: two 8-bit significands
                    lev[acc_of(q)] += pr;
                    lev_exact[acc_of(q)] += (long double)pr;
                }
                for (int q = 0; q < 6; ++q) lev32[acc_of(q)] += a3[S[q]] * bb[T[q]];
                exact += (long double)g[j] * u[j];
                exact32 += (long double)gh * u[j];
                absum += fabsl((long double)g[j] * u[j]);
            }
            for (int d = 0; d < 4; ++d) inexact_levels += ((long double)lev[d] != lev_exact[d]);
            for (int d = 0; d < 5; ++d) kl::tcs::df_acc(row64, lev[d]);
            row64 = kl::df::fast_two_sum(row64.h, row64.l);
            for (int d = 0; d < 3; ++d) kl::tcs::df_acc(row32, lev32[d]);
            row32 = kl::df::fast_two_sum(row32.h, row32.l);
        }
        const long double got64 = ((long double)row64.h + row64.l) * sigma * 0.00390625L;
        const long double got32 = ((long double)row32.h + row32.l) * sigma * 0.00390625L;
        rel64 = std::fmax(rel64, (double)(fabsl(got64 - exact) / absum));
        rel32 = std::fmax(rel32, (double)(fabsl(got32 - exact32) / absum));
    }
    std::printf("{\"not_bf16\": %d, \"big_digits\": %d, \"inexact_levels\": %d, \"slice_remainder\": %.6e, "
                "\"rel_err_float64_class\": %.6e, \"rel_err_float32_class\": %.6e}\n",
                not_bf16, big_digit, inexact_levels, slice_rem, rel64, rel32);
    return 0;
}
