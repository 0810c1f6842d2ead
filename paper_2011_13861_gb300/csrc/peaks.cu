// Throughput of the arithmetic pipes that bound the stage-5 kernels: float64 FMA (DFMA),
// float32 FMA (FFMA, and the packed pair form FFMA2), and the special-function unit's ex2 and
// rsqrt (MUFU).  These measured
// rates are the denominators of the roofline fractions the stage-5 kernels report (the kernels
// are compute-bound: a few MB of points and vectors against Ntilde^2 kernel evaluations).
//
// Each kernel runs a persistent grid of full-occupancy CTAs; every thread advances independent
// dependency chains, unrolled so that the loop's own counter and branch are a small fraction of
// the issued instructions.  The chains stay bounded and finite (a tiny increment or a
// contraction for FMA, x -> 2^-x and x -> 1/sqrt(x) for the MUFU functions) and their sum is
// stored only under a condition the compiler cannot decide, so no operation is removed.
#include "kl_internal.h"

namespace kl {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float mufu_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float mufu_rsqrt(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// CTA 0's first thread records the SM clock counter and the global nanosecond timer around its
// loop (sink[1..4]), from which the host derives the SM clock the launch ran at
__device__ __forceinline__ void stamp(double* sink, int at) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long c = clock64();
        unsigned long long ns;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
        sink[1 + at] = double(c);
        sink[3 + at] = double(ns);
    }
}

// four independent chains a thread, each with its own multiplicands (more chains measured
// slower on GB300: 1.60 DFMA per SM and cycle with 16 chains, 1.90 with 4, against a pipe peak of 2)
__global__ void __launch_bounds__(kThreads) dfma_rate_kernel(int iters, double a, double b, double* sink) {
    double x[4], p[4], q[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        x[i] = 0.5 + 1e-3 * i + 1e-9 * threadIdx.x;
        p[i] = a * (1.0 + 1e-3 * i);
        q[i] = b * (1.0 + 1e-4 * i);
    }
    stamp(sink, 0);
#pragma unroll 16
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = fma(p[i], q[i], x[i]);
    }
    stamp(sink, 1);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) s += x[i];
    if (s == -1.0) sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) ffma_rate_kernel(int iters, float a, float b, double* sink) {
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = 0.5f + 1e-3f * i + 1e-7f * threadIdx.x;
    stamp(sink, 0);
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = fmaf(x[i], a, b);
    }
    stamp(sink, 1);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += x[i];
    if (s == -1.f) sink[0] = s;
}

// packed float32 pair FMA (fma.rn.f32x2, Blackwell): two FMAs per lane and instruction; the
// rate counts FMAs, so it compares directly with the scalar FFMA rate above
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    return (static_cast<unsigned long long>(__float_as_uint(hi)) << 32) | __float_as_uint(lo);
}

__global__ void __launch_bounds__(kThreads) ffma2_rate_kernel(int iters, float a, float b, double* sink) {
    unsigned long long x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = pack2(0.5f + 1e-3f * i + 1e-7f * threadIdx.x, 0.25f + 1e-3f * i);
    const unsigned long long a2 = pack2(a, a), b2 = pack2(b, b);
    stamp(sink, 0);
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = ffma2(x[i], a2, b2);
    }
    stamp(sink, 1);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += __uint_as_float(unsigned(x[i])) + __uint_as_float(unsigned(x[i] >> 32));
    if (s == -1.f) sink[0] = s;
}

template <int FN>   // 0: ex2 of the negated value, 1: rsqrt
__global__ void __launch_bounds__(kThreads) mufu_rate_kernel(int iters, float a, double* sink) {
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = a + 1e-3f * i + 1e-7f * threadIdx.x;
    stamp(sink, 0);
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = FN == 0 ? mufu_ex2(-x[i]) : mufu_rsqrt(x[i]);
    }
    stamp(sink, 1);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += x[i];
    if (s == -1.f) sink[0] = s;
}

}  // namespace
}  // namespace kl

using namespace kl;

extern "C" kl_status kl_pipe_rates(double* rates_host, int n, void* stream) {
    if (!rates_host || n < 4) return fail(KL_ERR_INVALID_ARG, "kl_pipe_rates: rates_host needs 4 entries");
    const int nops = n >= 10 ? 5 : 4;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = num_sms() * (2048 / kThreads);
    const double threads = double(grid) * kThreads;
    DevBuf sink;
    KL_TRY(ensure(sink, 5 * sizeof(double)));
    double* snk = static_cast<double*>(sink.ptr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // operations per launch: chains x iterations x threads
    const int iters[5] = {4096, 32768, 8192, 4096, 32768};
    const double ops[5] = {4.0 * iters[0] * threads, 16.0 * iters[1] * threads, 16.0 * iters[2] * threads,
                           16.0 * iters[3] * threads, 16.0 * iters[4] * threads};
    int launches = 0;
    for (int op = 0; op < nops && e == cudaSuccess; ++op) {
        float best = 0.f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first launch is a warm-up
            e = cudaEventRecord(e0, s);
            if (e != cudaSuccess) break;
            switch (op) {
                case 0: dfma_rate_kernel<<<grid, kThreads, 0, s>>>(iters[0], 1e-9, 1e-9, snk); break;
                case 1: ffma_rate_kernel<<<grid, kThreads, 0, s>>>(iters[1], 0.9999f, 1e-5f, snk); break;
                case 2: mufu_rate_kernel<0><<<grid, kThreads, 0, s>>>(iters[2], 0.5f, snk); break;
                case 3: mufu_rate_kernel<1><<<grid, kThreads, 0, s>>>(iters[3], 0.7f, snk); break;
                default: ffma2_rate_kernel<<<grid, kThreads, 0, s>>>(iters[4], 0.9999f, 1e-5f, snk); break;
            }
            ++launches;
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) {
                best = ms;
                double st[5];
                e = cudaMemcpy(st, snk, sizeof(st), cudaMemcpyDeviceToHost);
                const int at = op < 4 ? 4 + op : 9;
                if (e == cudaSuccess && n >= 8 && st[4] > st[3]) rates_host[at] = 1e3 * (st[2] - st[1]) / (st[4] - st[3]);
            }
        }
        if (e == cudaSuccess) rates_host[op < 4 ? op : 8] = ops[op] / (double(best) * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    release(sink);
    count_launches(launches);
    if (e != cudaSuccess) return cuda_fail(e, "pipe-rate microbenchmark");
    return KL_OK;
}
