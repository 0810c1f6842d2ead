// Stage 5 of Algorithm 1 in double-float ("df64") arithmetic: float64-level accuracy
// (kernel values to ~1e-14 relative, sums to ~1e-15) computed entirely on the float32 pipe.
//
// Same N-body tiling as the float32/float64 kernels in covmv.cu: 128 rows per CTA (one per
// thread, coordinates as hi/lo float pairs in registers), column tiles of coordinates and of
// the u block (split into hi/lo floats while staging) in shared memory, a contiguous column
// range per CTA, partial sums combined in a fixed order by covmv_reduce.  Per pair the kernel
// value is formed once in double-float (distance with exact TwoSum differences, squared
// norm, Heron square root, Tang exponential) and reused for every vector of the block; each
// vector accumulates Gamma*u with an exact product and a TwoSum into a hi/lo accumulator
// that is renormalised once per tile.
#include "df64.cuh"
#include "kl_internal.h"

namespace kl {
namespace {

constexpr int kDfThreads = 128;
constexpr int kDfTile = 128;

using df::F2;

__device__ __forceinline__ F2 diff(float ah, float al, float bh, float bl) {
    F2 s = df::two_sum(ah, -bh);
    float e = df::add(s.l, df::sub(al, bl));
    return df::fast_two_sum(s.h, e);
}

template <int KIND>
__device__ __forceinline__ F2 kernel_df(const float* r, const float* c, int pm, const float* th,
                                        const float* tl) {
    // r, c: {xh, yh, zh, xl, yl, zl} of the row and column point
    if (KIND == KL_K_POLY_TEST) {
        F2 f{1.f, 0.f};
        for (int k = 0; k < 3; ++k) {
            F2 p = df::mul(F2{r[k], r[3 + k]}, F2{c[k], c[3 + k]});
            f = df::mul(f, df::add(p, F2{1.f, 0.f}));
        }
        F2 g{1.f, 0.f};
        for (int i = 0; i < pm; ++i) g = df::mul(g, f);
        return g;
    }
    const F2 dx = diff(r[0], r[3], c[0], c[3]);
    const F2 dy = diff(r[1], r[4], c[1], c[4]);
    const F2 dz = diff(r[2], r[5], c[2], c[5]);
    if (KIND == KL_K_EXP_SEPARABLE) {
        F2 s = df::add(df::add(df::abs(dx), df::abs(dy)), df::abs(dz));
        return df::exp_neg(s, th, tl);
    }
    F2 s = df::add(df::add(df::sqr(dx), df::sqr(dy)), df::sqr(dz));
    if (KIND == KL_K_GAUSS) return df::exp_neg(s, th, tl);
    float seed;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(seed) : "f"(fmaxf(s.h, 1e-30f)));
    return df::exp_neg(df::sqrt(s, seed), th, tl);
}

template <int KIND, int NV>
__global__ void __launch_bounds__(kDfThreads)
covmv_df_kernel(CovParams cp, const double* __restrict__ U, int64_t ldu, double* __restrict__ part,
                int64_t cols_per_split) {
    __shared__ float sp[6][kDfTile];
    __shared__ float2 su[kDfTile][NV];
    __shared__ float stab[128];
    if (threadIdx.x < 128) stab[threadIdx.x] = cp.tabdf[threadIdx.x];

    const int64_t Nt = cp.Nt;
    const int64_t row = int64_t(blockIdx.x) * kDfThreads + threadIdx.x;
    const bool valid = row < Nt;
    float rp[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) rp[k] = valid ? cp.Pdf[k * cp.ldp + row] : 0.f;

    const int64_t c_begin = int64_t(blockIdx.y) * cols_per_split;
    int64_t c_end = c_begin + cols_per_split;
    if (c_end > Nt) c_end = Nt;

    float ah[NV], al[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        ah[v] = 0.f;
        al[v] = 0.f;
    }
    for (int64_t c0 = c_begin; c0 < c_end; c0 += kDfTile) {
        __syncthreads();
        const int64_t c = c0 + threadIdx.x;
        if (c < c_end) {
#pragma unroll
            for (int k = 0; k < 6; ++k) sp[k][threadIdx.x] = cp.Pdf[k * cp.ldp + c];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const double u = U[v * ldu + c];
                const float uh = __double2float_rn(u);
                su[threadIdx.x][v] = make_float2(uh, __double2float_rn(u - double(uh)));
            }
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) sp[k][threadIdx.x] = 0.f;
#pragma unroll
            for (int v = 0; v < NV; ++v) su[threadIdx.x][v] = make_float2(0.f, 0.f);   // adds 0
        }
        __syncthreads();
#pragma unroll 1
        for (int j = 0; j < kDfTile; ++j) {
            float cpj[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) cpj[k] = sp[k][j];
            const F2 g = kernel_df<KIND>(rp, cpj, cp.poly_m, stab, stab + 64);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float2 u = su[j][v];
                const float ph = df::mul(g.h, u.x);
                float pe = df::fma_(g.h, u.x, -ph);
                pe = df::fma_(g.h, u.y, pe);
                pe = df::fma_(g.l, u.x, pe);
                const F2 s = df::two_sum(ah[v], ph);
                ah[v] = s.h;
                al[v] = df::add(al[v], df::add(s.l, pe));
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const F2 r = df::fast_two_sum(ah[v], al[v]);
            ah[v] = r.h;
            al[v] = r.l;
        }
    }
    if (valid) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
            part[(int64_t(blockIdx.y) * NV + v) * Nt + row] = double(ah[v]) + double(al[v]);
    }
}

__global__ void covmv_df_reduce(const double* __restrict__ part, int splits, int64_t Nt, int nv,
                                double* __restrict__ Z, int64_t ldz, double scale2,
                                const double* __restrict__ J) {
    const int64_t total = Nt * nv;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t v = idx / Nt, row = idx - v * Nt;
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp) s += part[(int64_t(sp) * nv + v) * Nt + row];
        s *= scale2;
        if (J) s *= J[row];
        Z[v * ldz + row] = s;
    }
}

template <int NV>
cudaError_t dispatch_df(const CovParams& cp, const double* U, int64_t ldu, double* part, dim3 grid,
                        int64_t cps, cudaStream_t s) {
    switch (cp.kind) {
        case KL_K_EXP: covmv_df_kernel<KL_K_EXP, NV><<<grid, kDfThreads, 0, s>>>(cp, U, ldu, part, cps); break;
        case KL_K_GAUSS: covmv_df_kernel<KL_K_GAUSS, NV><<<grid, kDfThreads, 0, s>>>(cp, U, ldu, part, cps); break;
        case KL_K_EXP_SEPARABLE: covmv_df_kernel<KL_K_EXP_SEPARABLE, NV><<<grid, kDfThreads, 0, s>>>(cp, U, ldu, part, cps); break;
        default: covmv_df_kernel<KL_K_POLY_TEST, NV><<<grid, kDfThreads, 0, s>>>(cp, U, ldu, part, cps); break;
    }
    return cudaGetLastError();
}

int group_df(int left) { return left >= 32 ? 32 : left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1; }

}  // namespace

int covmv_df_splits(int64_t Nt) {
    const int64_t rowblocks = (Nt + kDfThreads - 1) / kDfThreads;
    int64_t splits = (152 * 8 * 4 + rowblocks - 1) / rowblocks;
    int64_t maxs = Nt / (4 * kDfTile);
    if (maxs < 1) maxs = 1;
    if (splits > maxs) splits = maxs;
    if (splits > 64) splits = 64;
    if (splits < 1) splits = 1;
    return int(splits);
}

cudaError_t launch_covmv_df(const CovParams& cp, const double* U, int64_t ldu, int nvec, double* Z,
                            int64_t ldz, double scale2, const double* J, double* part, int splits,
                            cudaStream_t s) {
    const int64_t Nt = cp.Nt;
    if (Nt == 0 || nvec == 0) return cudaSuccess;
    int64_t cps = (Nt + splits - 1) / splits;
    cps = (cps + kDfTile - 1) / kDfTile * kDfTile;
    const int used = int((Nt + cps - 1) / cps);
    dim3 grid(unsigned((Nt + kDfThreads - 1) / kDfThreads), unsigned(used));
    for (int v0 = 0; v0 < nvec;) {
        const int g = group_df(nvec - v0);
        cudaError_t e;
        const double* Ug = U + int64_t(v0) * ldu;
        switch (g) {
            case 32: e = dispatch_df<32>(cp, Ug, ldu, part, grid, cps, s); break;
            case 16: e = dispatch_df<16>(cp, Ug, ldu, part, grid, cps, s); break;
            case 8: e = dispatch_df<8>(cp, Ug, ldu, part, grid, cps, s); break;
            case 4: e = dispatch_df<4>(cp, Ug, ldu, part, grid, cps, s); break;
            case 2: e = dispatch_df<2>(cp, Ug, ldu, part, grid, cps, s); break;
            default: e = dispatch_df<1>(cp, Ug, ldu, part, grid, cps, s); break;
        }
        if (e != cudaSuccess) return e;
        count_launches(2);
        int64_t tot = Nt * g;
        int blocks = int((tot + 255) / 256);
        if (blocks > 152 * 8) blocks = 152 * 8;
        covmv_df_reduce<<<blocks, 256, 0, s>>>(part, used, Nt, g, Z + int64_t(v0) * ldz, ldz, scale2, J);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        v0 += g;
    }
    return cudaSuccess;
}

}  // namespace kl
