// Float64 block linear algebra of the eigensolver: tall-skinny Gram products and updates,
// block Cholesky-QR, counter-based random blocks, the small symmetric eigenproblem of the
// Rayleigh-Ritz step, residual norms and restart bookkeeping.  Every reduction is
// two-stage with a fixed combination order, so repeated runs are bit-identical.
#include <math.h>

#include "df64.cuh"
#include "kl_internal.h"

namespace kl {
namespace {

constexpr int kGramThreads = 256;
constexpr int kGramRows = 32;
constexpr int kGramMaxP = 192;
constexpr int kGramMaxQ = 32;

// shared-memory row stride for a staged chunk of c columns: odd, so that the rows of a warp's
// coalesced stores fall into distinct banks
__host__ __device__ constexpr int gram_ld(int c) { return c | 1; }

// part[g][i*q + j] = sum over this CTA's rows r of A[r, i] * B[r, j]; rows are staged 32 at a
// time (coalesced along r) and every thread accumulates up to 24 of the p*q outputs
__global__ void __launch_bounds__(kGramThreads)
gram_partial(const double* __restrict__ A, int64_t lda, int p, const double* __restrict__ B,
             int64_t ldb, int q, int64_t N, int64_t rows_per_part, double* __restrict__ part) {
    extern __shared__ double sgram[];
    const int la = gram_ld(p), lb = gram_ld(q);
    double* sA = sgram;                       // [kGramRows][la]
    double* sB = sgram + kGramRows * la;      // [kGramRows][lb]
    const int outs = p * q;
    constexpr int kMaxPer = (kGramMaxP * kGramMaxQ + kGramThreads - 1) / kGramThreads;
    double acc[kMaxPer];
#pragma unroll
    for (int t = 0; t < kMaxPer; ++t) acc[t] = 0.0;
    const int64_t r_begin = int64_t(blockIdx.x) * rows_per_part;
    int64_t r_end = r_begin + rows_per_part;
    if (r_end > N) r_end = N;
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kGramRows) {
        __syncthreads();
        for (int e = threadIdx.x; e < kGramRows * p; e += kGramThreads) {
            const int c = e / kGramRows, rl = e - c * kGramRows;
            const int64_t r = r0 + rl;
            sA[rl * la + c] = (r < r_end) ? A[c * lda + r] : 0.0;
        }
        for (int e = threadIdx.x; e < kGramRows * q; e += kGramThreads) {
            const int c = e / kGramRows, rl = e - c * kGramRows;
            const int64_t r = r0 + rl;
            sB[rl * lb + c] = (r < r_end) ? B[c * ldb + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kMaxPer; ++t) {
            const int e = threadIdx.x + t * kGramThreads;
            if (e < outs) {
                const int i = e / q, j = e - i * q;
                double s = acc[t];
#pragma unroll 8
                for (int rr = 0; rr < kGramRows; ++rr) s = fma(sA[rr * la + i], sB[rr * lb + j], s);
                acc[t] = s;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < kMaxPer; ++t) {
        const int e = threadIdx.x + t * kGramThreads;
        if (e < outs) part[int64_t(blockIdx.x) * outs + e] = acc[t];
    }
}

// out = sum over the parts, 32 outputs per CTA: thread (g, o) adds parts g, g+8, ... of output o
// (coalesced along o), then the 8 group sums are added in a fixed order
__global__ void __launch_bounds__(256) gram_reduce(const double* __restrict__ part, int parts, int p, int q,
                                                   double* __restrict__ out, int ldo) {
    __shared__ double red[8][33];
    const int outs = p * q;
    const int o = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + o;
    double s = 0.0;
    if (e < outs)
        for (int k = g; k < parts; k += 8) s += part[int64_t(k) * outs + e];
    red[g][o] = s;
    __syncthreads();
    if (g == 0 && e < outs) {
        double t = red[0][o];
        for (int k = 1; k < 8; ++k) t += red[k][o];
        const int i = e / q, j = e - i * q;
        out[i + int64_t(j) * ldo] = t;
    }
}

// C[r, j0:j0+QB] = alpha * A[r, 0:p] B[:, j0:j0+QB] + beta * C[r, j0:j0+QB] for every row r and
// column group j0 (QB columns, the last group zero-padded); items (row, group) with the row
// fastest, so a warp reads 32 consecutive entries of each column of A; B in shared memory
template <int QB>
__global__ void __launch_bounds__(128)
gemm_tall_kernel(double alpha, const double* __restrict__ A, int64_t lda, int64_t N, int p,
                 const double* __restrict__ B, int ldb, int q, double beta, double* __restrict__ C,
                 int64_t ldc) {
    extern __shared__ double sBm[];   // p x (ng * QB), row-major
    const int ng = (q + QB - 1) / QB, lq = ng * QB;
    for (int e = threadIdx.x; e < p * lq; e += blockDim.x) {
        const int i = e / lq, j = e - i * lq;
        sBm[e] = (j < q) ? B[i + int64_t(j) * ldb] : 0.0;
    }
    __syncthreads();
    const int64_t items = N * ng;
    for (int64_t it = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; it < items;
         it += int64_t(gridDim.x) * blockDim.x) {
        const int64_t g = it / N, r = it - g * N;
        const int j0 = int(g) * QB;
        double acc[QB];
#pragma unroll
        for (int j = 0; j < QB; ++j) acc[j] = 0.0;
        for (int i = 0; i < p; ++i) {
            const double a = A[i * lda + r];
#pragma unroll
            for (int j = 0; j < QB; ++j) acc[j] = fma(a, sBm[i * lq + j0 + j], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < QB; ++j) {
            if (j0 + j < q) {
                double* c = C + (j0 + j) * ldc + r;
                *c = (beta == 0.0) ? alpha * acc[j] : fma(alpha, acc[j], beta * (*c));
            }
        }
    }
}

// ---- the same two products in double-float arithmetic on the float32 pipe ----
// For a phase whose operator is float32-accurate: every float64 input is split by integer
// operations into a double-float (split_double_bits, within 2^-47), each product term is the
// exact float32 product of the heads plus the two cross terms, and the sums are double-float
// (TwoSum into the head, tail accumulated, renormalised every staged chunk of rows), so a Gram
// entry or an updated basis entry carries about 2^-46 of its magnitude's error.  GB300's float32
// pipe runs ~65x the float64 pipe's FMA rate; a term costs 12 float32 operations.
__device__ __forceinline__ void df_madd(float& sh, float& sl, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float pe = __fmaf_rn(ah, bh, -p);
    const float cr = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, pe));
    const float s = __fadd_rn(sh, p);
    const float bb = __fsub_rn(s, sh);
    const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(e, cr));
}

__device__ __forceinline__ void df_renorm(float& sh, float& sl) {
    const float s = __fadd_rn(sh, sl);
    sl = __fsub_rn(sl, __fsub_rn(s, sh));
    sh = s;
}

__global__ void __launch_bounds__(kGramThreads)
gram_partial_df(const double* __restrict__ A, int64_t lda, int p, const double* __restrict__ B,
                int64_t ldb, int q, int64_t N, int64_t rows_per_part, double* __restrict__ part) {
    extern __shared__ float2 sgdf[];
    const int la = gram_ld(p), lb = gram_ld(q);
    float2* sA = sgdf;                        // [kGramRows][la] (head, tail)
    float2* sB = sgdf + kGramRows * la;       // [kGramRows][lb]
    const int outs = p * q;
    constexpr int kMaxPer = (kGramMaxP * kGramMaxQ + kGramThreads - 1) / kGramThreads;
    float acch[kMaxPer], accl[kMaxPer];
#pragma unroll
    for (int t = 0; t < kMaxPer; ++t) acch[t] = accl[t] = 0.f;
    const int64_t r_begin = int64_t(blockIdx.x) * rows_per_part;
    int64_t r_end = r_begin + rows_per_part;
    if (r_end > N) r_end = N;
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kGramRows) {
        __syncthreads();
        for (int e = threadIdx.x; e < kGramRows * p; e += kGramThreads) {
            const int c = e / kGramRows, rl = e - c * kGramRows;
            const int64_t r = r0 + rl;
            const df::F2 v = df::split_double_bits((r < r_end) ? A[c * lda + r] : 0.0);
            sA[rl * la + c] = make_float2(v.h, v.l);
        }
        for (int e = threadIdx.x; e < kGramRows * q; e += kGramThreads) {
            const int c = e / kGramRows, rl = e - c * kGramRows;
            const int64_t r = r0 + rl;
            const df::F2 v = df::split_double_bits((r < r_end) ? B[c * ldb + r] : 0.0);
            sB[rl * lb + c] = make_float2(v.h, v.l);
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kMaxPer; ++t) {
            const int e = threadIdx.x + t * kGramThreads;
            if (e < outs) {
                const int i = e / q, j = e - i * q;
                float sh = acch[t], sl = accl[t];
#pragma unroll 4
                for (int rr = 0; rr < kGramRows; ++rr) {
                    const float2 a = sA[rr * la + i], b = sB[rr * lb + j];
                    df_madd(sh, sl, a.x, a.y, b.x, b.y);
                }
                df_renorm(sh, sl);
                acch[t] = sh;
                accl[t] = sl;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < kMaxPer; ++t) {
        const int e = threadIdx.x + t * kGramThreads;
        if (e < outs) part[int64_t(blockIdx.x) * outs + e] = double(acch[t]) + double(accl[t]);
    }
}

template <int QB>
__global__ void __launch_bounds__(128)
gemm_tall_df_kernel(double alpha, const double* __restrict__ A, int64_t lda, int64_t N, int p,
                    const double* __restrict__ B, int ldb, int q, double beta, double* __restrict__ C,
                    int64_t ldc) {
    extern __shared__ float2 sBdf[];   // p x (ng * QB), row-major (head, tail)
    const int ng = (q + QB - 1) / QB, lq = ng * QB;
    for (int e = threadIdx.x; e < p * lq; e += blockDim.x) {
        const int i = e / lq, j = e - i * lq;
        const df::F2 v = df::split_double_bits((j < q) ? B[i + int64_t(j) * ldb] : 0.0);
        sBdf[e] = make_float2(v.h, v.l);
    }
    __syncthreads();
    const int64_t items = N * ng;
    for (int64_t it = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; it < items;
         it += int64_t(gridDim.x) * blockDim.x) {
        const int64_t g = it / N, r = it - g * N;
        const int j0 = int(g) * QB;
        float sh[QB], sl[QB];
#pragma unroll
        for (int j = 0; j < QB; ++j) sh[j] = sl[j] = 0.f;
        for (int i = 0; i < p; ++i) {
            const df::F2 a = df::split_double_bits(A[i * lda + r]);
#pragma unroll
            for (int j = 0; j < QB; ++j) {
                const float2 b = sBdf[i * lq + j0 + j];
                df_madd(sh[j], sl[j], a.h, a.l, b.x, b.y);
            }
            if ((i & 15) == 15) {
#pragma unroll
                for (int j = 0; j < QB; ++j) df_renorm(sh[j], sl[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < QB; ++j) {
            if (j0 + j < q) {
                double* c = C + (j0 + j) * ldc + r;
                const double v = double(sh[j]) + double(sl[j]);
                *c = (beta == 0.0) ? alpha * v : fma(alpha, v, beta * (*c));
            }
        }
    }
}

// G (b x b, column-major) = R^T R with R upper triangular; also R^{-1}.  One CTA.
// flag is set to 1 when a pivot is not positive (rank-deficient block).
__global__ void chol_inv_kernel(const double* __restrict__ G, int ldg, int b, double* __restrict__ Rinv,
                                double* __restrict__ R, int* flag) {
    extern __shared__ double sR[];   // b x b, column-major
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) sR[e] = 0.0;
    __syncthreads();
    double gmax = 0.0;
    for (int i = 0; i < b; ++i) gmax = fmax(gmax, G[i + int64_t(i) * ldg]);
    for (int j = 0; j < b; ++j) {
        if (threadIdx.x == 0) {
            double s = G[j + int64_t(j) * ldg];
            for (int k = 0; k < j; ++k) s -= sR[k + j * b] * sR[k + j * b];
            if (!(s > 1e-28 * gmax) || !isfinite(s)) {
                bad = 1;
                s = 1e-28 * gmax + 1e-300;
            }
            sR[j + j * b] = sqrt(s);
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) {
            double s = G[j + int64_t(i) * ldg];
            for (int k = 0; k < j; ++k) s -= sR[k + j * b] * sR[k + i * b];
            sR[j + i * b] = s / sR[j + j * b];
        }
        __syncthreads();
    }
    // R^{-1}: column c solves R x = e_c by back substitution
    for (int c = threadIdx.x; c < b; c += blockDim.x) {
        for (int i = b - 1; i >= 0; --i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = i + 1; k <= c; ++k) s -= sR[i + k * b] * Rinv[k + c * b];
            Rinv[i + c * b] = (i <= c) ? s / sR[i + i * b] : 0.0;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) R[e] = sR[e];
    if (threadIdx.x == 0) *flag = bad;
}

// splitmix64 (Steele, Lea, Flood 2014): uniform(-1, 1) from (seed, counter)
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return double(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

__global__ void random_block_kernel(double* V, int64_t ldv, int64_t N, int b, uint64_t seed,
                                    uint64_t offset) {
    const int64_t total = N * b;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = e / N, r = e - c * N;
        V[c * ldv + r] = splitmix_uniform(seed, offset + uint64_t(e));
    }
}

// ---- small symmetric eigenproblem: parallel cyclic Jacobi (round-robin pair ordering) ----
constexpr int kEigThreads = 256;
constexpr int kEigMax = 160;

__device__ __forceinline__ void rr_pair(int i, int r, int mp, int* a, int* b) {
    // round r of the circle method for mp (even) players; pair i
    if (i == 0) {
        *a = 0;
        *b = ((mp - 2 + r) % (mp - 1)) + 1;
    } else {
        *a = ((i - 1 + r) % (mp - 1)) + 1;
        *b = ((mp - 2 - i + r) % (mp - 1)) + 1;
    }
}

__global__ void __launch_bounds__(kEigThreads)
sym_eig_kernel(const double* __restrict__ Tin, int ldt, int m, double* __restrict__ evals,
               double* __restrict__ Sout, int lds, double* __restrict__ W, int* sweeps_out,
               bool w_given) {
    extern __shared__ double sT[];          // m x m, row-major with stride m
    __shared__ double cs[kEigMax / 2 + 1][2];
    __shared__ int prs[kEigMax / 2 + 1][2];
    const int tid = threadIdx.x;
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e - i * m;
        sT[e] = 0.5 * (Tin[i + int64_t(j) * ldt] + Tin[j + int64_t(i) * ldt]);
        if (!w_given) W[i + int64_t(j) * m] = (i == j) ? 1.0 : 0.0;   // eigenvector accumulator, column-major
    }
    __syncthreads();
    const int mp = (m % 2 == 0) ? m : m + 1;
    const int npairs = mp / 2;
    int sweep = 0;
    for (; sweep < 40; ++sweep) {
        int rotated = 0;   // this thread applied a rotation in this sweep
        for (int r = 0; r < mp - 1; ++r) {
            for (int i = tid; i < npairs; i += blockDim.x) {
                int a, b;
                rr_pair(i, r, mp, &a, &b);
                if (a > b) { int t = a; a = b; b = t; }
                double c = 1.0, s = 0.0;
                if (b < m) {
                    const double apq = sT[a * m + b];
                    const double app = sT[a * m + a], aqq = sT[b * m + b];
                    if (fabs(apq) > 1e-17 * sqrt(fabs(app * aqq)) && apq != 0.0) {
                        const double theta = (aqq - app) / (2.0 * apq);
                        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                        rotated = 1;
                    }
                }
                prs[i][0] = a;
                prs[i][1] = b;
                cs[i][0] = c;
                cs[i][1] = s;
            }
            __syncthreads();
            // rows: T <- J^T T
            for (int e = tid; e < npairs * m; e += blockDim.x) {
                const int i = e / m, j = e - i * m;
                const int a = prs[i][0], b = prs[i][1];
                if (b >= m || cs[i][1] == 0.0) continue;
                const double c = cs[i][0], s = cs[i][1];
                const double ta = sT[a * m + j], tb = sT[b * m + j];
                sT[a * m + j] = c * ta - s * tb;
                sT[b * m + j] = s * ta + c * tb;
            }
            __syncthreads();
            // columns: T <- T J ; eigenvectors W <- W J
            for (int e = tid; e < npairs * m; e += blockDim.x) {
                const int i = e / m, j = e - i * m;
                const int a = prs[i][0], b = prs[i][1];
                if (b >= m || cs[i][1] == 0.0) continue;
                const double c = cs[i][0], s = cs[i][1];
                const double ta = sT[j * m + a], tb = sT[j * m + b];
                sT[j * m + a] = c * ta - s * tb;
                sT[j * m + b] = s * ta + c * tb;
                const double wa = W[j + int64_t(a) * m], wb = W[j + int64_t(b) * m];
                W[j + int64_t(a) * m] = c * wa - s * wb;
                W[j + int64_t(b) * m] = s * wa + c * wb;
            }
            __syncthreads();
            for (int i = tid; i < npairs; i += blockDim.x) {
                const int a = prs[i][0], b = prs[i][1];
                if (b < m && cs[i][1] != 0.0) {
                    sT[a * m + b] = 0.0;
                    sT[b * m + a] = 0.0;
                }
            }
            __syncthreads();
        }
        // every thread takes the same decision (a shared flag reset by one thread at the top of
        // the next sweep could be read after the reset by a slower thread)
        if (!__syncthreads_or(rotated)) break;
    }
    // sort descending: rank by (value desc, index asc)
    for (int i = tid; i < m; i += blockDim.x) {
        const double di = sT[i * m + i];
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const double dj = sT[j * m + j];
            if (dj > di || (dj == di && j < i)) ++rank;
        }
        evals[rank] = di;
        for (int r = 0; r < m; ++r) Sout[r + int64_t(rank) * lds] = W[r + int64_t(i) * m];
    }
    if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// ---- the same parallel cyclic Jacobi in double-float arithmetic (float32 pipe) ----
// GB300's float64 pipe issues about 1.6 FMAs per clock per SM against ~113 float32 FMAs, so
// the rotations are applied to double-float (hi + lo) copies of T and of the eigenvector
// accumulator.  The rotation for a pair comes from a float32 tangent t (the textbook formula),
// with c = 1/sqrt(1 + t^2) and s = t c formed in double-float so that c^2 + s^2 = 1 to ~2^-48:
// every rotation is orthogonal to double-float accuracy, and an off-diagonal entry that a
// rotation leaves at ~2^-24 of its size is removed by the next sweep.  Sweeps stop when no
// off-diagonal entry exceeds off_tol sqrt(|T_aa T_bb|) (1e-14 by default).
constexpr int kEigDfThreads = 1024;
constexpr int kEigDfMax = 112;

__device__ __forceinline__ df::F2 df_from_double(double x) {
    const float h = float(x);
    return df::F2{h, float(x - double(h))};
}

// (c x - s y, s x + c y) for double-float c, s, x, y
__device__ __forceinline__ void df_rotate(df::F2 c, df::F2 sn, float& xh, float& xl, float& yh, float& yl) {
    const df::F2 x{xh, xl}, y{yh, yl};
    const df::F2 nx = df::sub(df::mul(c, x), df::mul(sn, y));
    const df::F2 ny = df::add(df::mul(sn, x), df::mul(c, y));
    xh = nx.h;
    xl = nx.l;
    yh = ny.h;
    yl = ny.l;
}

__global__ void __launch_bounds__(kEigDfThreads)
sym_eig_df_kernel(const double* __restrict__ Tin, int ldt, int m, double* __restrict__ evals,
                  double* __restrict__ Sout, int lds, int* sweeps_out, float off_tol) {
    extern __shared__ float sdf[];
    const int ld = m | 1;                       // odd stride: column accesses spread over banks
    float* Th = sdf;                            // T, row-major [m][ld]
    float* Tl = Th + m * ld;
    float* Wh = Tl + m * ld;                    // eigenvectors, column-major [m][ld]
    float* Wl = Wh + m * ld;
    __shared__ df::F2 cs[kEigDfMax / 2 + 1][2];
    __shared__ int prs[kEigDfMax / 2 + 1][2];
    const int tid = threadIdx.x;
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e - i * m;
        const df::F2 v = df_from_double(0.5 * (Tin[i + int64_t(j) * ldt] + Tin[j + int64_t(i) * ldt]));
        Th[i * ld + j] = v.h;
        Tl[i * ld + j] = v.l;
        Wh[j * ld + i] = (i == j) ? 1.f : 0.f;
        Wl[j * ld + i] = 0.f;
    }
    __syncthreads();
    const int mp = (m % 2 == 0) ? m : m + 1;
    const int npairs = mp / 2;
    int sweep = 0;
    for (; sweep < 40; ++sweep) {
        int rotated = 0;   // this thread applied a rotation in this sweep
        for (int r = 0; r < mp - 1; ++r) {
            for (int i = tid; i < npairs; i += blockDim.x) {
                int a, b;
                rr_pair(i, r, mp, &a, &b);
                if (a > b) { int t = a; a = b; b = t; }
                df::F2 c{1.f, 0.f}, sn{0.f, 0.f};
                if (b < m) {
                    const float apq = Th[a * ld + b];
                    const float app = Th[a * ld + a], aqq = Th[b * ld + b];
                    if (apq != 0.f && fabsf(apq) > off_tol * sqrtf(fabsf(app)) * sqrtf(fabsf(aqq))) {
                        const df::F2 d = df::sub(df::F2{Th[b * ld + b], Tl[b * ld + b]},
                                                 df::F2{Th[a * ld + a], Tl[a * ld + a]});
                        const float theta = d.h / (2.f * apq);
                        float t;
                        if (fabsf(theta) > 1e18f) {
                            t = 0.5f / theta;
                        } else {
                            t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
                        }
                        // u = 1 + t^2 (|t| <= 1) in double-float; c = 1/sqrt(u); s = t c
                        const df::F2 t2 = df::two_prod(t, t);
                        df::F2 u = df::fast_two_sum(1.f, t2.h);
                        u = df::fast_two_sum(u.h, df::add(u.l, t2.l));
                        float seed;
                        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(seed) : "f"(u.h));
                        const df::F2 su = df::sqrt(u, seed);
                        const float r0 = 1.f / su.h;
                        const df::F2 p = df::mul(su, df::F2{r0, 0.f});
                        const df::F2 e1 = df::sub(df::F2{1.f, 0.f}, p);
                        c = df::fast_two_sum(r0, r0 * e1.h);
                        sn = df::mul(df::F2{t, 0.f}, c);
                        rotated = 1;
                    }
                }
                prs[i][0] = a;
                prs[i][1] = b;
                cs[i][0] = c;
                cs[i][1] = sn;
            }
            __syncthreads();
            // T <- J^T T J in one pass: each 2 x 2 block (rows of pair I, columns of pair J) is
            // rotated by I's rotation on its rows, then by J's on its columns (the same operations,
            // in the same order, as a row pass over all of T followed by a column pass); a pair
            // whose partner is the padding index m has one row, and its rotation is the identity
            for (int e = tid; e < npairs * npairs; e += blockDim.x) {
                const int I = e / npairs, J = e - I * npairs;
                const bool rI = prs[I][1] < m && cs[I][1].h != 0.f, rJ = prs[J][1] < m && cs[J][1].h != 0.f;
                if (!rI && !rJ) continue;
                const int a = prs[I][0], b = prs[I][1], c = prs[J][0], d = prs[J][1];
                const bool hb = b < m, hd = d < m;
                float ach = Th[a * ld + c], acl = Tl[a * ld + c];
                float adh = hd ? Th[a * ld + d] : 0.f, adl = hd ? Tl[a * ld + d] : 0.f;
                float bch = hb ? Th[b * ld + c] : 0.f, bcl = hb ? Tl[b * ld + c] : 0.f;
                float bdh = (hb && hd) ? Th[b * ld + d] : 0.f, bdl = (hb && hd) ? Tl[b * ld + d] : 0.f;
                if (rI) {
                    df_rotate(cs[I][0], cs[I][1], ach, acl, bch, bcl);
                    df_rotate(cs[I][0], cs[I][1], adh, adl, bdh, bdl);
                }
                if (rJ) {
                    df_rotate(cs[J][0], cs[J][1], ach, acl, adh, adl);
                    df_rotate(cs[J][0], cs[J][1], bch, bcl, bdh, bdl);
                }
                Th[a * ld + c] = ach;
                Tl[a * ld + c] = acl;
                if (hd) {
                    Th[a * ld + d] = adh;
                    Tl[a * ld + d] = adl;
                }
                if (hb) {
                    Th[b * ld + c] = bch;
                    Tl[b * ld + c] = bcl;
                }
                if (hb && hd) {
                    Th[b * ld + d] = bdh;
                    Tl[b * ld + d] = bdl;
                }
            }
            // eigenvectors W <- W J
            for (int e = tid; e < npairs * m; e += blockDim.x) {
                const int i = e / m, j = e - i * m;
                const int a = prs[i][0], b = prs[i][1];
                if (b >= m || cs[i][1].h == 0.f) continue;
                df_rotate(cs[i][0], cs[i][1], Wh[a * ld + j], Wl[a * ld + j], Wh[b * ld + j], Wl[b * ld + j]);
            }
            __syncthreads();
        }
        // every thread takes the same decision (a shared flag reset by one thread at the top of
        // the next sweep could be read after the reset by a slower thread)
        if (!__syncthreads_or(rotated)) break;
    }
    // sort descending: rank by (value desc, index asc)
    for (int i = tid; i < m; i += blockDim.x) {
        const double di = double(Th[i * ld + i]) + double(Tl[i * ld + i]);
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const double dj = double(Th[j * ld + j]) + double(Tl[j * ld + j]);
            if (dj > di || (dj == di && j < i)) ++rank;
        }
        evals[rank] = di;
        for (int r = 0; r < m; ++r) Sout[r + int64_t(rank) * lds] = double(Wh[i * ld + r]) + double(Wl[i * ld + r]);
    }
    if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// out[i] = sqrt(s_i^T G s_i), s_i = S[srow0 : srow0 + b, i]
__global__ void residual_norms_kernel(const double* __restrict__ G, int ldg, const double* __restrict__ S,
                                      int lds, int srow0, int b, int ncols, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncols; i += gridDim.x * blockDim.x) {
        const double* s = S + int64_t(i) * lds + srow0;
        double acc = 0.0;
        for (int a = 0; a < b; ++a) {
            double t = 0.0;
            for (int c = 0; c < b; ++c) t = fma(G[a + int64_t(c) * ldg], s[c], t);
            acc = fma(s[a], t, acc);
        }
        out[i] = sqrt(fmax(acc, 0.0));
    }
}

// part[g][i] = sum over this CTA's rows of (AY[r,i] - theta_i Y[r,i])^2
__global__ void ritz_resid_partial(const double* __restrict__ AY, const double* __restrict__ Y, int64_t ld,
                                   int64_t N, int k, const double* __restrict__ theta,
                                   int64_t rows_per_part, double* __restrict__ part) {
    __shared__ double red[256];
    const int64_t r_begin = int64_t(blockIdx.x) * rows_per_part;
    int64_t r_end = r_begin + rows_per_part;
    if (r_end > N) r_end = N;
    for (int i = 0; i < k; ++i) {
        const double th = theta[i];
        double s = 0.0;
        for (int64_t r = r_begin + threadIdx.x; r < r_end; r += blockDim.x) {
            const double d = AY[i * ld + r] - th * Y[i * ld + r];
            s = fma(d, d, s);
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[int64_t(blockIdx.x) * k + i] = red[0];
        __syncthreads();
    }
}

__global__ void ritz_resid_final(const double* __restrict__ part, int parts, int k,
                                 const double* __restrict__ theta, double* __restrict__ out) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < parts; ++g) s += part[int64_t(g) * k + i];
        out[i] = sqrt(s) / fabs(theta[i]);
    }
}

// T = 0 except T[i][i] = theta_i (i < p) and the coupling rows/columns p..p+b-1:
// T[p + a][i] = T[i][p + a] = sum_c R[a][c] S[srow0 + c][i]
__global__ void set_restart_T_kernel(double* __restrict__ T, int ldt, int m, const double* __restrict__ theta,
                                     int p, const double* __restrict__ R, int ldr,
                                     const double* __restrict__ S, int lds, int srow0, int b) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
        const int i = e % m, j = e / m;
        double v = 0.0;
        if (i == j && i < p) v = theta[i];
        int a = -1, col = -1;
        if (i >= p && i < p + b && j < p) { a = i - p; col = j; }
        if (j >= p && j < p + b && i < p) { a = j - p; col = i; }
        if (a >= 0) {
            double s = 0.0;
            for (int c = a; c < b; ++c) s = fma(R[a + c * ldr], S[(srow0 + c) + int64_t(col) * lds], s);
            v = s;
        }
        T[i + int64_t(j) * ldt] = v;
    }
}

__global__ void to_float_kernel(const double* __restrict__ src, int64_t lds, float* __restrict__ dst,
                                int64_t ldd, int64_t rows, int cols) {
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = e / rows, r = e - c * rows;
        dst[c * ldd + r] = float(src[c * lds + r]);
    }
}

// T[r0 + i][c0 + j] = H[i][j]; if symmetric also T[c0 + j][r0 + i] = H[i][j]
// (an overlapping diagonal block is symmetrised).
__global__ void fill_T_block_kernel(double* __restrict__ T, int ldt, int r0, int c0,
                                    const double* __restrict__ H, int ldh, int rows, int cols,
                                    bool symmetric) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x) {
        const int i = e % rows, j = e / rows;
        const int gi = r0 + i, gj = c0 + j;
        double v = H[i + int64_t(j) * ldh];
        const bool diag_block = symmetric && gi >= c0 && gi < c0 + cols && gj >= r0 && gj < r0 + rows;
        if (diag_block) v = 0.5 * (v + H[(gj - r0) + int64_t(gi - c0) * ldh]);
        T[gi + int64_t(gj) * ldt] = v;
        if (symmetric) T[gj + int64_t(gi) * ldt] = v;
    }
}

__global__ void add_inplace_kernel(double* __restrict__ H, const double* __restrict__ H2, int n) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) H[e] += H2[e];
}

// W[:, c] = AX[:, c] - theta[c] X[:, c]  (block of Ritz residuals)
__global__ void ritz_residual_block_kernel(const double* __restrict__ AX, const double* __restrict__ X, int64_t ld,
                                           int64_t N, int nc, const double* __restrict__ theta,
                                           double* __restrict__ W, int64_t ldw) {
    const int64_t total = N * nc;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = e / N, i = e - c * N;
        W[c * ldw + i] = fma(-theta[c], X[c * ld + i], AX[c * ld + i]);
    }
}

int grid_for(int64_t work, int threads, int cap) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return int(b);
}

}  // namespace

// the largest dynamic shared memory of gemm_tall_kernel: p <= kGramMaxP rows of B, 32 columns
constexpr int kGemmMaxSmem = kGramMaxP * 32 * int(sizeof(double));

int num_sms() {
    static int cached = 0;
    if (cached == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) ==
                                                       cudaSuccess && n > 0)
            cached = n;
        else
            return 152;
    }
    return cached;
}

// two CTAs per SM (all resident at once), at least 64 rows each
int gram_parts(int64_t N) {
    int64_t parts = (N + 63) / 64;
    const int64_t cap = int64_t(num_sms()) * 2;
    if (parts > cap) parts = cap;
    if (parts < 1) parts = 1;
    return int(parts);
}

template <bool DF>
cudaError_t gram_impl(const double* A, int64_t lda, int p, const double* B, int64_t ldb, int q,
                      int64_t N, double* out, int ldo, double* part, int maxparts, cudaStream_t s) {
    if (p > kGramMaxP) return cudaErrorInvalidValue;
    if (p == 0 || q == 0) return cudaSuccess;
    int parts = gram_parts(N);
    if (parts > maxparts) parts = maxparts;
    int64_t rpp = (N + parts - 1) / parts;
    rpp = (rpp + kGramRows - 1) / kGramRows * kGramRows;
    parts = int((N + rpp - 1) / rpp);
    if (parts < 1) parts = 1;
    for (int j0 = 0; j0 < q; j0 += kGramMaxQ) {
        const int qq = (q - j0 < kGramMaxQ) ? q - j0 : kGramMaxQ;
        const size_t smem = size_t(kGramRows) * (gram_ld(p) + gram_ld(qq)) * sizeof(double);   // = float2 too
        auto kern = DF ? gram_partial_df : gram_partial;
        if (smem > 48 * 1024) {
            // the largest request ever (set, never lowered: launches of other threads stay valid)
            const int smax = int(size_t(kGramRows) * (gram_ld(kGramMaxP) + gram_ld(kGramMaxQ)) * sizeof(double));
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
            if (e != cudaSuccess) return e;
        }
        count_launches(2);
        kern<<<parts, kGramThreads, smem, s>>>(A, lda, p, B + int64_t(j0) * ldb, ldb, qq, N, rpp, part);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        gram_reduce<<<(p * qq + 31) / 32, 256, 0, s>>>(part, parts, p, qq, out + int64_t(j0) * ldo, ldo);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <bool DF>
cudaError_t gemm_tall_impl(double alpha, const double* A, int64_t lda, int64_t N, int p,
                           const double* B, int ldb, int q, double beta, double* C, int64_t ldc,
                           cudaStream_t s) {
    if (N == 0 || q == 0) return cudaSuccess;
    if (p == 0) {
        // C = beta * C
        return (beta == 1.0) ? cudaSuccess : cudaErrorInvalidValue;
    }
    if (p > kGramMaxP) return cudaErrorInvalidValue;
    for (int j0 = 0; j0 < q; j0 += 32) {
        const int qq = (q - j0 < 32) ? q - j0 : 32;
        const int QB = qq == 1 ? 1 : 4;
        const int ng = (qq + QB - 1) / QB;
        const size_t smem = size_t(p) * ng * QB * sizeof(double);
        const int blocks = grid_for(N * ng, 128, num_sms() * 16);
        const double* Bj = B + int64_t(j0) * ldb;
        count_launches(1);
        double* Cj = C + int64_t(j0) * ldc;
        cudaError_t e = cudaSuccess;
        auto kern = (QB == 1) ? (DF ? gemm_tall_df_kernel<1> : gemm_tall_kernel<1>)
                              : (DF ? gemm_tall_df_kernel<4> : gemm_tall_kernel<4>);
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmMaxSmem);
        if (e != cudaSuccess) return e;
        kern<<<blocks, 128, smem, s>>>(alpha, A, lda, N, p, Bj, ldb, qq, beta, Cj, ldc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_gram(const double* A, int64_t lda, int p, const double* B, int64_t ldb, int q,
                        int64_t N, double* out, int ldo, double* part, int maxparts, cudaStream_t s) {
    return gram_impl<false>(A, lda, p, B, ldb, q, N, out, ldo, part, maxparts, s);
}

cudaError_t launch_gram_df(const double* A, int64_t lda, int p, const double* B, int64_t ldb, int q,
                           int64_t N, double* out, int ldo, double* part, int maxparts, cudaStream_t s) {
    return gram_impl<true>(A, lda, p, B, ldb, q, N, out, ldo, part, maxparts, s);
}

cudaError_t launch_gemm_tall(double alpha, const double* A, int64_t lda, int64_t N, int p,
                             const double* B, int ldb, int q, double beta, double* C, int64_t ldc,
                             cudaStream_t s) {
    return gemm_tall_impl<false>(alpha, A, lda, N, p, B, ldb, q, beta, C, ldc, s);
}

cudaError_t launch_gemm_tall_df(double alpha, const double* A, int64_t lda, int64_t N, int p,
                                const double* B, int ldb, int q, double beta, double* C, int64_t ldc,
                                cudaStream_t s) {
    return gemm_tall_impl<true>(alpha, A, lda, N, p, B, ldb, q, beta, C, ldc, s);
}

cudaError_t launch_chol_inv(double* G, int ldg, int b, double* Rinv, double* R, int* flag,
                            cudaStream_t s) {
    chol_inv_kernel<<<1, 64, size_t(b) * b * sizeof(double), s>>>(G, ldg, b, Rinv, R, flag);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_random_block(double* V, int64_t ldv, int64_t N, int b, uint64_t seed,
                                uint64_t offset, cudaStream_t s) {
    random_block_kernel<<<grid_for(N * b, 256, num_sms() * 4), 256, 0, s>>>(V, ldv, N, b, seed, offset);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sym_eig_ws(const double* T, int ldt, int m, double* evals, double* S, int lds,
                              double* work, int* sweeps_out, cudaStream_t s, float off_tol) {
    if (m > kEigMax || m < 1) return cudaErrorInvalidValue;
    if (m <= kEigDfMax) {
        const size_t smem = size_t(4) * m * (m | 1) * sizeof(float);
        cudaError_t e = cudaFuncSetAttribute(sym_eig_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(size_t(4) * kEigDfMax * (kEigDfMax | 1) * sizeof(float)));
        if (e != cudaSuccess) return e;
        sym_eig_df_kernel<<<1, kEigDfThreads, smem, s>>>(T, ldt, m, evals, S, lds, sweeps_out, off_tol);
        count_launches(1);
        return cudaGetLastError();
    }
    const size_t smem = size_t(m) * m * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(sym_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(size_t(kEigMax) * kEigMax * sizeof(double)));
    if (e != cudaSuccess) return e;
    sym_eig_kernel<<<1, kEigThreads, smem, s>>>(T, ldt, m, evals, S, lds, work, sweeps_out, false);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_residual_norms(const double* G, int ldg, const double* S, int lds, int srow0,
                                  int b, int ncols, double* out, cudaStream_t s) {
    residual_norms_kernel<<<grid_for(ncols, 64, 64), 64, 0, s>>>(G, ldg, S, lds, srow0, b, ncols, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ritz_resid(const double* AY, const double* Y, int64_t ld, int64_t N, int k,
                              const double* theta, double* part, int maxparts, double* out,
                              cudaStream_t s) {
    int parts = gram_parts(N);
    if (parts > maxparts) parts = maxparts;
    const int64_t rpp = (N + parts - 1) / parts;
    ritz_resid_partial<<<parts, 256, 0, s>>>(AY, Y, ld, N, k, theta, rpp, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launches(2);
    ritz_resid_final<<<1, 64, 0, s>>>(part, parts, k, theta, out);
    return cudaGetLastError();
}

cudaError_t launch_set_restart_T(double* T, int ldt, int m, const double* theta, int p,
                                 const double* R, int ldr, const double* S, int lds, int srow0,
                                 int b, cudaStream_t s) {
    set_restart_T_kernel<<<grid_for(int64_t(m) * m, 256, 128), 256, 0, s>>>(T, ldt, m, theta, p, R, ldr, S,
                                                                           lds, srow0, b);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_copy_block(const double* src, int64_t lds, double* dst, int64_t ldd,
                              int64_t rows, int cols, cudaStream_t s) {
    return cudaMemcpy2DAsync(dst, size_t(ldd) * sizeof(double), src, size_t(lds) * sizeof(double),
                             size_t(rows) * sizeof(double), size_t(cols), cudaMemcpyDeviceToDevice, s);
}

cudaError_t launch_to_float(const double* src, int64_t lds, float* dst, int64_t ldd, int64_t rows,
                            int cols, cudaStream_t s) {
    to_float_kernel<<<grid_for(rows * cols, 256, num_sms() * 8), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill_T_block(double* T, int ldt, int r0, int c0, const double* H, int ldh,
                                int rows, int cols, bool symmetric, cudaStream_t s) {
    fill_T_block_kernel<<<grid_for(int64_t(rows) * cols, 256, 64), 256, 0, s>>>(T, ldt, r0, c0, H, ldh, rows,
                                                                               cols, symmetric);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_add_inplace(double* H, const double* H2, int n, cudaStream_t s) {
    add_inplace_kernel<<<grid_for(n, 256, 64), 256, 0, s>>>(H, H2, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ritz_residual_block(const double* AX, const double* X, int64_t ld, int64_t N, int nc,
                                      const double* theta, double* W, int64_t ldw, cudaStream_t s) {
    if (N == 0 || nc == 0) return cudaSuccess;
    ritz_residual_block_kernel<<<grid_for(N * nc, 256, num_sms() * 8), 256, 0, s>>>(AX, X, ld, N, nc, theta, W, ldw);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace kl
