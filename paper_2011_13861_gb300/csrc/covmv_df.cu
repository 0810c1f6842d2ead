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

using df::kernel_df;

template <int KIND, int NV>
__global__ void __launch_bounds__(kDfThreads)
covmv_df_kernel(CovParams cp, const double* __restrict__ U, int64_t ldu, double* __restrict__ part,
                int64_t cols_per_split, int nv) {
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
                const double u = (v < nv) ? U[v * ldu + c] : 0.0;   // inactive lanes add 0
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
            if (v < nv) part[(int64_t(blockIdx.y) * nv + v) * Nt + row] = double(ah[v]) + double(al[v]);
    }
}

// ---- symmetric tiling: Gamma(x_k, x_l) = Gamma(x_l, x_k), so each kernel value is evaluated once
// for both products.  Points are cut into tiles of 256 and each 256 x 256 block is evaluated
// once; thread t owns row I*256+t.  Off the diagonal the block is walked in 32-column chunks in a
// rotated order: at step s lane l evaluates the pair (row l, column (l+s) mod 32) of the chunk,
// adds g*u_col to its row accumulator and g*u_row to a travelling column accumulator that is
// handed to lane l-1 after every step, so after 32 steps lane l holds the warp's sum for column l.
// The 8 warps' column sums are combined in shared memory.  The diagonal block (I, I) is
// evaluated in full, row side only.  Schedules (SymPlan): BAND = false, CTA b takes the pair
// (I, J), I <= J, of the triangular index b, row sums to slot J and column sums to slot I, so
// every output row receives exactly one partial per tile index; BAND = true, CTA (I, s) walks its
// bands of the launch, adding column sums into slot S + (d - d0) and its row sums into slot s.
constexpr int kSymTile = kSymTileSize;

__device__ __forceinline__ void sym_decode_tri_df(int64_t bidx, int* I, int* J) {
    int j = int((sqrt(8.0 * double(bidx) + 1.0) - 1.0) * 0.5);
    while (int64_t(j) * (j + 1) / 2 > bidx) --j;
    while (int64_t(j + 1) * (j + 2) / 2 <= bidx) ++j;
    *J = j;
    *I = int(bidx - int64_t(j) * (j + 1) / 2);
}

template <int KIND, int NV, bool BAND>
__global__ void __launch_bounds__(kSymTile)
covmv_df_sym_kernel(CovParams cp, const double* __restrict__ U, int64_t ldu, double* __restrict__ part,
                    int nv, SymBand bd) {
    extern __shared__ float smem_sym[];
    float* sc = smem_sym;                                   // [6][256] column coordinates
    float2* su = reinterpret_cast<float2*>(smem_sym + 6 * kSymTile);   // [256][NV] column u
    float2* cpart = su + kSymTile * NV;                     // [8 warps][32][NV] column partials
    __shared__ float stab[128];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 128) stab[tid] = cp.tabdf[tid];

    int I, J0;
    if (BAND) {
        I = blockIdx.x;
        J0 = 0;
    } else {
        sym_decode_tri_df(blockIdx.x, &I, &J0);
    }
    const int nsteps = BAND ? bd.nd : 1;

    const int64_t Nt = cp.Nt;
    const int64_t row = int64_t(I) * kSymTile + tid;
    const bool rvalid = row < Nt;
    float rp[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) rp[k] = rvalid ? cp.Pdf[k * cp.ldp + row] : 0.f;
    float2 ur[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double u = (rvalid && v < nv) ? U[v * ldu + row] : 0.0;
        const float uh = __double2float_rn(u);
        ur[v] = make_float2(uh, __double2float_rn(u - double(uh)));
    }
    float ah[NV], al[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        ah[v] = 0.f;
        al[v] = 0.f;
    }
    double rsum[NV];   // row sums across the blocks of a band launch
#pragma unroll
    for (int v = 0; v < NV; ++v) rsum[v] = 0.0;

    for (int step = 0; step < nsteps; ++step) {
        int J = J0, d = 0;
        if (BAND && !sym_band_pair(bd, I, blockIdx.y, step, &J, &d)) continue;
        const bool diag = BAND ? (d == 0) : (I == J);
        const int cslot = BAND ? bd.S + (d - bd.d0) : I;
        __syncthreads();
        // stage the column tile J
        {
            const int64_t c = int64_t(J) * kSymTile + tid;
            const bool cvalid = c < Nt;
#pragma unroll
            for (int k = 0; k < 6; ++k) sc[k * kSymTile + tid] = cvalid ? cp.Pdf[k * cp.ldp + c] : 0.f;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const double u = (cvalid && v < nv) ? U[v * ldu + c] : 0.0;
                const float uh = __double2float_rn(u);
                su[tid * NV + v] = make_float2(uh, __double2float_rn(u - double(uh)));
            }
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            ah[v] = 0.f;
            al[v] = 0.f;
        }
        if (diag) {
#pragma unroll 1
            for (int j = 0; j < kSymTile; ++j) {
                float cpj[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) cpj[k] = sc[k * kSymTile + j];
                const F2 g = kernel_df<KIND>(rp, cpj, cp.poly_m, stab, stab + 64);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const float2 u = su[j * NV + v];
                    const float ph = df::mul(g.h, u.x);
                    float pe = df::fma_(g.h, u.x, -ph);
                    pe = df::fma_(g.h, u.y, pe);
                    pe = df::fma_(g.l, u.x, pe);
                    const F2 sm = df::two_sum(ah[v], ph);
                    ah[v] = sm.h;
                    al[v] = df::add(al[v], df::add(sm.l, pe));
                }
            }
        } else {
            const int64_t col0 = int64_t(J) * kSymTile;
#pragma unroll 1
            for (int q = 0; q < kSymTile / 32; ++q) {
                float ch[NV], cl[NV];   // travelling column accumulator
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    ch[v] = 0.f;
                    cl[v] = 0.f;
                }
#pragma unroll 1
                for (int st = 0; st < 32; ++st) {
                    const int j = q * 32 + ((lane + st) & 31);
                    float cpj[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) cpj[k] = sc[k * kSymTile + j];
                    const F2 g = kernel_df<KIND>(rp, cpj, cp.poly_m, stab, stab + 64);
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        // row side: g * u_col
                        const float2 u = su[j * NV + v];
                        float ph = df::mul(g.h, u.x);
                        float pe = df::fma_(g.h, u.x, -ph);
                        pe = df::fma_(g.h, u.y, pe);
                        pe = df::fma_(g.l, u.x, pe);
                        F2 sm = df::two_sum(ah[v], ph);
                        ah[v] = sm.h;
                        al[v] = df::add(al[v], df::add(sm.l, pe));
                        // column side: g * u_row
                        ph = df::mul(g.h, ur[v].x);
                        pe = df::fma_(g.h, ur[v].x, -ph);
                        pe = df::fma_(g.h, ur[v].y, pe);
                        pe = df::fma_(g.l, ur[v].x, pe);
                        sm = df::two_sum(ch[v], ph);
                        ch[v] = sm.h;
                        cl[v] = df::add(cl[v], df::add(sm.l, pe));
                        ch[v] = __shfl_sync(0xffffffffu, ch[v], (lane + 1) & 31);
                        cl[v] = __shfl_sync(0xffffffffu, cl[v], (lane + 1) & 31);
                    }
                }
                // lane holds this warp's partial for column q*32 + lane
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const F2 r = df::fast_two_sum(ch[v], cl[v]);
                    cpart[(warp * 32 + lane) * NV + v] = make_float2(r.h, r.l);
                }
                __syncthreads();
                for (int e = tid; e < 32 * NV; e += kSymTile) {
                    const int cl_ = e / NV, v = e - cl_ * NV;
                    double acc = 0.0;
                    for (int w = 0; w < kSymTile / 32; ++w) {
                        const float2 p = cpart[(w * 32 + cl_) * NV + v];
                        acc += double(p.x) + double(p.y);
                    }
                    const int64_t c = col0 + q * 32 + cl_;
                    if (c < Nt && v < nv) {
                        double* dst = part + (int64_t(cslot) * nv + v) * Nt + c;
                        *dst = BAND ? *dst + acc : acc;
                    }
                }
                __syncthreads();
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const F2 r = df::fast_two_sum(ah[v], al[v]);
                    ah[v] = r.h;
                    al[v] = r.l;
                }
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) rsum[v] += double(ah[v]) + double(al[v]);
    }
    if (rvalid) {
        const int rslot = BAND ? int(blockIdx.y) : J0;
#pragma unroll
        for (int v = 0; v < NV; ++v)
            if (v < nv) {
                double* dst = part + (int64_t(rslot) * nv + v) * Nt + row;
                *dst = BAND ? *dst + rsum[v] : rsum[v];
            }
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
                        int64_t cps, int nv, cudaStream_t s) {
    switch (cp.kind) {
        case KL_K_EXP: covmv_df_kernel<KL_K_EXP, NV><<<grid, kDfThreads, 0, s>>>(cp, U, ldu, part, cps, nv); break;
        case KL_K_GAUSS: covmv_df_kernel<KL_K_GAUSS, NV><<<grid, kDfThreads, 0, s>>>(cp, U, ldu, part, cps, nv); break;
        case KL_K_EXP_SEPARABLE: covmv_df_kernel<KL_K_EXP_SEPARABLE, NV><<<grid, kDfThreads, 0, s>>>(cp, U, ldu, part, cps, nv); break;
        default: covmv_df_kernel<KL_K_POLY_TEST, NV><<<grid, kDfThreads, 0, s>>>(cp, U, ldu, part, cps, nv); break;
    }
    return cudaGetLastError();
}

// instantiated block widths; a group of n active vectors runs in the smallest width >= n so
// that the kernel value of a pair is evaluated once for the whole group
int width_df(int n) {
    static const int w[] = {1, 2, 4, 8, 12, 16, 20, 24, 32};
    for (int x : w)
        if (n <= x) return x;
    return 32;
}

constexpr int kSymMaxNV = 8;   // widest block that takes the symmetric path

template <int KIND, int NV>
cudaError_t sym_df_kind(const CovParams& cp, const double* U, int64_t ldu, double* part, const SymPlan& pl, int nv,
                        cudaStream_t s) {
    const size_t smem = (size_t(6) * kSymTile + 2 * size_t(kSymTile) * NV + 2 * size_t(kSymTile) * NV) * sizeof(float);
    if (!pl.band) {
        SymBand bd{pl.T, pl.D, 0, 1, 0};
        const unsigned pairs = unsigned(int64_t(pl.T) * (pl.T + 1) / 2);
        covmv_df_sym_kernel<KIND, NV, false><<<pairs, kSymTile, smem, s>>>(cp, U, ldu, part, nv, bd);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(part, 0, size_t(pl.slots) * nv * cp.Nt * sizeof(double), s);
    for (int t = 0; t < pl.launches && e == cudaSuccess; ++t) {
        SymBand bd{pl.T, pl.D, t * kSymBandW, kSymBandW / kSymBandS, kSymBandS};
        covmv_df_sym_kernel<KIND, NV, true><<<dim3(unsigned(pl.T), unsigned(kSymBandS)), kSymTile, smem, s>>>(
            cp, U, ldu, part, nv, bd);
        e = cudaGetLastError();
    }
    return e;
}

template <int NV>
cudaError_t launch_sym(const CovParams& cp, const double* U, int64_t ldu, double* part, const SymPlan& pl, int nv,
                       cudaStream_t s) {
    switch (cp.kind) {
        case KL_K_EXP: return sym_df_kind<KL_K_EXP, NV>(cp, U, ldu, part, pl, nv, s);
        case KL_K_GAUSS: return sym_df_kind<KL_K_GAUSS, NV>(cp, U, ldu, part, pl, nv, s);
        case KL_K_EXP_SEPARABLE: return sym_df_kind<KL_K_EXP_SEPARABLE, NV>(cp, U, ldu, part, pl, nv, s);
        default: return sym_df_kind<KL_K_POLY_TEST, NV>(cp, U, ldu, part, pl, nv, s);
    }
}

}  // namespace

// partial-sum scratch (doubles) of the non-symmetric double-float stage 5 (column splits, groups
// of up to 32 vectors); the symmetric path needs sym_part_doubles
size_t covmv_df_part_doubles(int64_t Nt, int nvec) {
    (void)nvec;
    return size_t(covmv_df_splits(Nt)) * 32 * size_t(Nt);
}

int covmv_df_splits(int64_t Nt) {
    const int64_t rowblocks = (Nt + kDfThreads - 1) / kDfThreads;
    int64_t splits = (int64_t(num_sms()) * 8 * 4 + rowblocks - 1) / rowblocks;
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
    const int nt_tiles = int((Nt + kSymTile - 1) / kSymTile);
    for (int v0 = 0; v0 < nvec;) {
        const int g = (nvec - v0) < 32 ? (nvec - v0) : 32;   // active vectors in this launch
        cudaError_t e;
        const double* Ug = U + int64_t(v0) * ldu;
        if (g <= kSymMaxNV && nt_tiles >= 2) {
            // narrow blocks: symmetric tiles halve the kernel evaluations
            const int w = width_df(g);
            const SymPlan pl = sym_plan(Nt, g);
            switch (w) {
                case 8: e = launch_sym<8>(cp, Ug, ldu, part, pl, g, s); break;
                case 4: e = launch_sym<4>(cp, Ug, ldu, part, pl, g, s); break;
                case 2: e = launch_sym<2>(cp, Ug, ldu, part, pl, g, s); break;
                default: e = launch_sym<1>(cp, Ug, ldu, part, pl, g, s); break;
            }
            if (e != cudaSuccess) return e;
            count_launches(1 + pl.launches);
            int64_t tot = Nt * g;
            int blocks = int((tot + 255) / 256);
            if (blocks > num_sms() * 8) blocks = num_sms() * 8;
            covmv_df_reduce<<<blocks, 256, 0, s>>>(part, pl.slots, Nt, g, Z + int64_t(v0) * ldz, ldz, scale2, J);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            v0 += g;
            continue;
        }
        switch (width_df(g)) {
            case 32: e = dispatch_df<32>(cp, Ug, ldu, part, grid, cps, g, s); break;
            case 24: e = dispatch_df<24>(cp, Ug, ldu, part, grid, cps, g, s); break;
            case 20: e = dispatch_df<20>(cp, Ug, ldu, part, grid, cps, g, s); break;
            case 16: e = dispatch_df<16>(cp, Ug, ldu, part, grid, cps, g, s); break;
            case 12: e = dispatch_df<12>(cp, Ug, ldu, part, grid, cps, g, s); break;
            case 8: e = dispatch_df<8>(cp, Ug, ldu, part, grid, cps, g, s); break;
            case 4: e = dispatch_df<4>(cp, Ug, ldu, part, grid, cps, g, s); break;
            case 2: e = dispatch_df<2>(cp, Ug, ldu, part, grid, cps, g, s); break;
            default: e = dispatch_df<1>(cp, Ug, ldu, part, grid, cps, g, s); break;
        }
        if (e != cudaSuccess) return e;
        count_launches(2);
        int64_t tot = Nt * g;
        int blocks = int((tot + 255) / 256);
        if (blocks > num_sms() * 8) blocks = num_sms() * 8;
        covmv_df_reduce<<<blocks, 256, 0, s>>>(part, used, Nt, g, Z + int64_t(v0) * ldz, ldz, scale2, J);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        v0 += g;
    }
    return cudaSuccess;
}

}  // namespace kl
