// Self-test of the bounded waits that every tensor-core kernel uses (failure detection without a
// GPU fault): one thread waits on an mbarrier that nothing ever completes, gives up after the
// requested time, records KL_ERR_TIMEOUT in a device status word and returns, so the host sees
// the same error status a stalled pipeline would produce and the context stays usable.
#include <cmath>
#include <vector>

#include "df2.cuh"
#include "kernel32.cuh"
#include "kl_internal.h"
#include "tc_common.cuh"
#include "tc_slices.cuh"

namespace kl {
namespace {

__global__ void wait_selftest_kernel(long long max_clocks, int* status) {
    using namespace tc;
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);                         // one arrival expected, none ever made
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const bool ok = mbar_wait(b, 0, max_clocks);
    *status = ok ? int(KL_OK) : int(KL_ERR_TIMEOUT);
}

// splitmix64 (Steele, Lea, Flood 2014) of a counter: uniform 64-bit words
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// a double in [0, span) from a counter, as a normalised double-float (head, tail)
__device__ __forceinline__ void rand_df(unsigned long long seed, unsigned long long ctr, double span, float* h,
                                        float* l) {
    const double x = double(mix64(seed ^ mix64(ctr)) >> 11) * 0x1.0p-53 * span;
    *h = float(x);
    *l = float(x - double(*h));
}

// Packed pair evaluation (df2.cuh) against the scalar one (df64.cuh, tc_slices.cuh), bit by bit:
// pair i draws a row point and two column points with coordinates in [0, span_i) (span_i from
// 1/4 to 64, so arguments reach the exponential's clamp), evaluates the three kernels the
// packed producers handle, slices each value and adds the slices into a running double-float
// sum, and counts the words that differ.
__global__ void df2_selftest_kernel(long long n, unsigned long long seed, const float* __restrict__ tab,
                                    unsigned long long* __restrict__ mismatches) {
    __shared__ float stab[128];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) stab[i] = tab[i];
    __syncthreads();
    unsigned long long bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double span = 0.25 * double(1 << (i % 9));
        float r[6], c0[6], c1[6];
        for (int k = 0; k < 3; ++k) {
            rand_df(seed, 9ull * i + k, span, &r[k], &r[3 + k]);
            rand_df(seed, 9ull * i + 3 + k, span, &c0[k], &c0[3 + k]);
            rand_df(seed, 9ull * i + 6 + k, span, &c1[k], &c1[3 + k]);
        }
        df2::V r2[6], cc[6];
        for (int k = 0; k < 6; ++k) {
            r2[k] = df2::dup(r[k]);
            cc[k] = df2::mk(c0[k], c1[k]);
        }
        for (int kind = 0; kind < 3; ++kind) {
            df::F2 g0, g1;
            df2::P g;
            if (kind == 0) {
                g0 = df::kernel_df<KL_K_EXP>(r, c0, 0, stab, stab + 64);
                g1 = df::kernel_df<KL_K_EXP>(r, c1, 0, stab, stab + 64);
                g = df2::kernel_df<KL_K_EXP>(r2, cc, stab, stab + 64);
            } else if (kind == 1) {
                g0 = df::kernel_df<KL_K_GAUSS>(r, c0, 0, stab, stab + 64);
                g1 = df::kernel_df<KL_K_GAUSS>(r, c1, 0, stab, stab + 64);
                g = df2::kernel_df<KL_K_GAUSS>(r2, cc, stab, stab + 64);
            } else {
                g0 = df::kernel_df<KL_K_EXP_SEPARABLE>(r, c0, 0, stab, stab + 64);
                g1 = df::kernel_df<KL_K_EXP_SEPARABLE>(r, c1, 0, stab, stab + 64);
                g = df2::kernel_df<KL_K_EXP_SEPARABLE>(r2, cc, stab, stab + 64);
            }
            bad += (__float_as_uint(g0.h) != __float_as_uint(df2::lo(g.h))) + (__float_as_uint(g0.l) != __float_as_uint(df2::lo(g.l)));
            bad += (__float_as_uint(g1.h) != __float_as_uint(df2::hi(g.h))) + (__float_as_uint(g1.l) != __float_as_uint(df2::hi(g.l)));
            float o0[6], o1[6];
            df2::V o[6];
            tcs::slices6(g0, o0);
            tcs::slices6(g1, o1);
            df2::slices6(g, o);
            df::F2 a0{0.f, 0.f}, a1{0.f, 0.f};
            df2::P a{df2::dup(0.f), df2::dup(0.f)};
            for (int q = 0; q < 6; ++q) {
                bad += (__float_as_uint(o0[q]) != __float_as_uint(df2::lo(o[q]))) +
                       (__float_as_uint(o1[q]) != __float_as_uint(df2::hi(o[q])));
                tcs::df_acc(a0, o0[q]);
                tcs::df_acc(a1, o1[q]);
                df2::acc_add(a, o[q]);
            }
            a0 = df::fast_two_sum(a0.h, a0.l);
            a1 = df::fast_two_sum(a1.h, a1.l);
            a = df2::fast_two_sum(a.h, a.l);
            bad += (__float_as_uint(a0.h) != __float_as_uint(df2::lo(a.h))) + (__float_as_uint(a0.l) != __float_as_uint(df2::lo(a.l)));
            bad += (__float_as_uint(a1.h) != __float_as_uint(df2::hi(a.h))) + (__float_as_uint(a1.l) != __float_as_uint(df2::hi(a.l)));
            // float32 class (the heads as float32 coordinates): kernel values and three slices
            float f0, f1;
            df2::V f;
            const df2::V dx = df2::sub(df2::dup(r[0]), df2::mk(c0[0], c1[0]));
            const df2::V dy = df2::sub(df2::dup(r[1]), df2::mk(c0[1], c1[1]));
            const df2::V dz = df2::sub(df2::dup(r[2]), df2::mk(c0[2], c1[2]));
            if (kind == 0) {
                f0 = kernel32<KL_K_EXP>(r[0] - c0[0], r[1] - c0[1], r[2] - c0[2], r[0], r[1], r[2], c0[0], c0[1], c0[2], 0);
                f1 = kernel32<KL_K_EXP>(r[0] - c1[0], r[1] - c1[1], r[2] - c1[2], r[0], r[1], r[2], c1[0], c1[1], c1[2], 0);
                f = df2::kernel32<KL_K_EXP>(dx, dy, dz);
            } else if (kind == 1) {
                f0 = kernel32<KL_K_GAUSS>(r[0] - c0[0], r[1] - c0[1], r[2] - c0[2], r[0], r[1], r[2], c0[0], c0[1], c0[2], 0);
                f1 = kernel32<KL_K_GAUSS>(r[0] - c1[0], r[1] - c1[1], r[2] - c1[2], r[0], r[1], r[2], c1[0], c1[1], c1[2], 0);
                f = df2::kernel32<KL_K_GAUSS>(dx, dy, dz);
            } else {
                f0 = kernel32<KL_K_EXP_SEPARABLE>(r[0] - c0[0], r[1] - c0[1], r[2] - c0[2], r[0], r[1], r[2], c0[0], c0[1],
                                                  c0[2], 0);
                f1 = kernel32<KL_K_EXP_SEPARABLE>(r[0] - c1[0], r[1] - c1[1], r[2] - c1[2], r[0], r[1], r[2], c1[0], c1[1],
                                                  c1[2], 0);
                f = df2::kernel32<KL_K_EXP_SEPARABLE>(dx, dy, dz);
            }
            bad += (__float_as_uint(f0) != __float_as_uint(df2::lo(f))) + (__float_as_uint(f1) != __float_as_uint(df2::hi(f)));
            float t0[3], t1[3];
            df2::V t[3];
            tcs::slices3(f0, t0);
            tcs::slices3(f1, t1);
            df2::slices3(f, t);
            for (int q = 0; q < 3; ++q)
                bad += (__float_as_uint(t0[q]) != __float_as_uint(df2::lo(t[q]))) +
                       (__float_as_uint(t1[q]) != __float_as_uint(df2::hi(t[q])));
        }
    }
    if (bad) atomicAdd(mismatches, bad);
}

}  // namespace
}  // namespace kl

using namespace kl;

extern "C" kl_status kl_df2_selftest(int64_t n, uint64_t seed, int64_t* mismatches, void* stream) {
    if (n < 0 || !mismatches) return fail(KL_ERR_INVALID_ARG, "df2 self-test: n >= 0 and a result pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<float> tab(128);
    for (int j = 0; j < 64; ++j) {
        const double t = exp2(-double(j) / 64.0);
        tab[j] = float(t);
        tab[64 + j] = float(t - double(tab[j]));
    }
    DevBuf dt, dm;
    KL_TRY(ensure(dt, 128 * sizeof(float)));
    KL_TRY(ensure(dm, sizeof(unsigned long long)));
    unsigned long long h = 0;
    cudaError_t e = cudaMemcpyAsync(dt.ptr, tab.data(), 128 * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dm.ptr, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess && n > 0) {
        df2_selftest_kernel<<<num_sms() * 4, 256, 0, s>>>(n, seed, static_cast<const float*>(dt.ptr),
                                                         static_cast<unsigned long long*>(dm.ptr));
        e = cudaGetLastError();
        count_launches(1);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, dm.ptr, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release(dt);
    release(dm);
    if (e != cudaSuccess) return cuda_fail(e, "df2 self-test");
    *mismatches = int64_t(h);
    return KL_OK;
}

extern "C" kl_status kl_wait_selftest(double seconds, void* stream) {
    if (!(seconds > 0.0) || seconds > 2.0) return fail(KL_ERR_INVALID_ARG, "wait self-test: 0 < seconds <= 2");
    int dev = 0, khz = 0;
    KL_CUDA(cudaGetDevice(&dev));
    KL_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const long long max_clocks = (long long)(seconds * double(khz) * 1e3);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf st;
    KL_TRY(ensure(st, sizeof(int)));
    int h = -1;
    wait_selftest_kernel<<<1, 1, 0, s>>>(max_clocks, static_cast<int*>(st.ptr));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st.ptr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release(st);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    count_launches(1);
    if (h == int(KL_ERR_TIMEOUT)) return fail(KL_ERR_TIMEOUT, "wait self-test: the bounded wait gave up as intended");
    return fail(KL_ERR_NUMERIC, "wait self-test: an mbarrier nothing arrives at completed");
}
