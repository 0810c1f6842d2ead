// Stage 5 of Algorithm 1 on the tensor cores (tcgen05, sm_103a) by exact fixed-point slicing,
// for groups of up to 32 right-hand sides: z = Gamma u.  Two classes share one kernel:
//   * float64 class (KL_P_TC64): kernel values in double-float (~48 bits), six 8-bit digits;
//   * float32 class (KL_P_TC32): float32 kernel values (MUFU ex2/rsqrt), three 8-bit digits.
//
// Exact slicing.  Each kernel value g (scaled so |g| <= 1) is written as
// g = sum_{s<S} a_s 2^(-8(s+1)) with integer digits (|a_0| <= 256, |a_s| <= 128 after by
// round-to-nearest digit extraction, except |a_3| <= 256 where the double-float tail joins the
// remainder; every step exact), and each u value, after division by a
// per-vector power of two sigma >= max|u|, as u/sigma = sum_{t<S} b_t 2^(-8(t+1)).  The digits
// are stored as bfloat16 "slices" a_s 2^(-8(s+1)) and b_t 2^(-8t), which bfloat16 holds exactly.
// The tensor core forms the slice products exactly and adds them in float32, one accumulator per
// level d = s + t:
//   float64 class: levels 0-3 (1, 2, 3, 4 products) are multiples of 2^-8(d+1) and, summed over
//     128 columns, at most 2^24 of that unit, hence exact in float32 whatever the tensor core's
//     rounding; levels 4-5
//     (11 products, relative size <= 2^-32) share a fifth accumulator whose rounding stays
//     below ~2^-49 of the sum; products of levels >= 6 (relative size < 2^-48) are dropped;
//   float32 class: levels 0-2 (1, 2, 3 products) are exact the same way; levels >= 3
//     (relative size < 2^-24) are dropped.
// Every 128 columns the accumulators are drained into double-float sums.  The result carries a
// relative error of ~1e-14 (float64 class) or ~1e-7 (float32 class: the float32 kernel values
// and the 24-bit fixed point), independent of the number of points, because no float32 sum
// ever spans more than 128 columns.
//
// Pipeline and schedule (persistent tile ranges over (128-row block, 32-column chunk) tiles,
// loader / producers / MMA issuer synchronised by mbarriers):
//   * loader (one thread): bulk copy per 32-column chunk of a pre-staged image holding the
//     column coordinates and the u slices (tcx_image_kernel);
//   * producers (float64 class: 16 warps, four threads per row, 8 columns each; float32 class:
//     8 warps, two threads per row, 16 columns each, two CTAs per SM): kernel values, S slices
//     each, written K-major;
//   * MMA issuer (one thread): one MMA per slice product and 16 columns into the level
//     accumulators in tensor memory, double-buffered per 128-column drain block.
// Every wait is bounded (~2 s), after which the CTA records KL_ERR_TIMEOUT, drains its own
// asynchronous operations and returns.
#include "df2.cuh"
#include "df64.cuh"
#include "kernel32.cuh"
#include "tc_slices.cuh"
#include "tc_common.cuh"

namespace kl {
namespace {

using namespace tc;
using df::F2;

constexpr int kRows = 128;                        // MMA M
constexpr int kK = 16;                            // MMA K (16-bit inputs)
constexpr int kChunk = 32;                        // columns per stage
constexpr int kStages = 3;
constexpr int kNB = 32;                           // MMA N: vectors per group
constexpr int kDrainChunks = 4;                   // level accumulators drained every 128 columns
constexpr int kASub = kRows * kK * 2;             // 128 x 16 bf16: 4 KB
constexpr int kASlice = kASub * (kChunk / kK);    // 8 KB
constexpr int kBSub = kNB * kK * 2;               // 32 x 16 bf16: 1 KB
constexpr int kBSlice = kBSub * (kChunk / kK);    // 2 KB
constexpr uint32_t kIdesc = idesc_bf16(kRows, kNB);

// per class: slices, products, accumulators, coordinate floats per column, shared-memory layout
template <int CLS>
struct Tx {
    // producers: float64 class 16 warps (four threads per row, 8 columns and 8 vectors each),
    // float32 class 8 warps (two threads per row, 16 each), then the loader warp and the MMA warp
    static constexpr int kProducers = CLS == 64 ? 512 : 256;
    static constexpr int kThreads = kProducers + 64;
    static constexpr int kLoaderWarp = kProducers / 32;
    static constexpr int kMmaWarp = kLoaderWarp + 1;
    static constexpr int kVpt = 32 / (kProducers / 128);      // columns (and vectors) per thread
    // tensor memory: accumulator a of drain-block parity dp at dp * kTmemBuf + a * 32; the float32
    // class needs 192 columns, so two of its CTAs share an SM
    static constexpr int kTmemCols = CLS == 64 ? 512 : 256;
    static constexpr int kTmemBuf = kTmemCols / 2;
    static constexpr int kCtasPerSm = CLS == 64 ? 1 : 2;
    static constexpr int kSlices = CLS == 64 ? 6 : 3;
    static constexpr int kProducts = CLS == 64 ? 21 : 6;
    static constexpr int kAccs = CLS == 64 ? 5 : 3;
    static constexpr int kCoords = CLS == 64 ? 6 : 3;         // double-float heads/tails, or float
    static constexpr int kAStage = kASlice * kSlices;
    static constexpr int kCoordBytes = kCoords * kChunk * 4;
    static constexpr int kImg = kCoordBytes + kBSlice * kSlices;
    static constexpr int kOffA = 0;
    static constexpr int kOffImg = kOffA + kStages * kAStage;
    static constexpr int kOffTab = kOffImg + kStages * kImg;  // 2^(-j/64) heads and tails
    static constexpr int kOffBar = kOffTab + 128 * 4;
    static constexpr int kBarLoaded = 0, kBarFull = kStages, kBarEmpty = 2 * kStages;
    static constexpr int kBarBlkDone = 3 * kStages, kBarBlkFree = kBarBlkDone + 2;
    static constexpr int kNumBars = kBarBlkFree + 2;
    static constexpr int kOffTmem = kOffBar + 8 * kNumBars;
    static constexpr int kSmemBytes = kOffTmem + 16;
    static_assert(kImg % 16 == 0 && kOffImg % 16 == 0 && kOffBar % 8 == 0, "bulk-copy and mbarrier alignment");
    static_assert(kSmemBytes <= 227 * 1024, "shared memory");
};

// the slice products (a_s, b_t) grouped by accumulator.  Float64 class: s + t <= 5, levels 0,
// 1, 2, 3, then 4-5 together.  Float32 class: s + t <= 2, levels 0, 1, 2.
template <int CLS>
__device__ __forceinline__ void product(int q, int* s, int* t, int* acc, bool* first) {
    constexpr int S[21] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5};
    constexpr int T[21] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0};
    *s = S[q];
    *t = T[q];
    *acc = q == 0 ? 0 : q < 3 ? 1 : q < 6 ? 2 : q < 10 ? 3 : 4;
    *first = (q == 0 || q == 1 || q == 3 || q == 6 || q == 10);
}

using tcs::slices3;
using tcs::slices6;

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

using tcs::df_acc;

// sigma[v] = 2^e with 2^(e-1) <= max_c |u[v][c]| < 2^e (1 when the column is zero)
template <typename TU>
__global__ void tcx_scale_kernel(const TU* __restrict__ U, int64_t ldu, int64_t Nt, double* __restrict__ sigma) {
    __shared__ double red[256];
    const int v = blockIdx.x;
    double m = 0.0;
    for (int64_t c = threadIdx.x; c < Nt; c += blockDim.x) m = fmax(m, fabs(double(U[v * ldu + c])));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int e = 0;
        const double mx = red[0];
        if (mx > 0.0 && isfinite(mx)) {
            frexp(mx, &e);
            sigma[v] = ldexp(1.0, e);
        } else {
            sigma[v] = 1.0;
        }
    }
}

// Image of column chunk ch: coordinates (float64 class: double-float heads then tails from Pdf;
// float32 class: the float32 coordinates P32; zero past Ntilde) and the u slices of the group in
// the K-major operand layout (rows = vectors, zero past nv and Ntilde).
template <int CLS, typename TU>
__global__ void tcx_image_kernel(const float* __restrict__ P, int64_t ldp, int64_t Nt, const TU* __restrict__ U,
                                 int64_t ldu, int nv, const double* __restrict__ sigma,
                                 unsigned char* __restrict__ img, int64_t nchunks) {
    using X = Tx<CLS>;
    const int t = threadIdx.x;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        unsigned char* base = img + ch * X::kImg;
        const int64_t c0 = ch * kChunk;
        if (t < X::kCoords * kChunk) {
            const int64_t c = c0 + (t % kChunk);
            reinterpret_cast<float*>(base)[t] = c < Nt ? P[int64_t(t / kChunk) * ldp + c] : 0.f;
        }
        if (t < kNB * (kChunk / 8)) {
            const int v = t / (kChunk / 8), g8 = t % (kChunk / 8);
            const double inv = (v < nv) ? 1.0 / sigma[v] : 0.0;   // a power of two: exact
            float sl[X::kSlices][8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t c = c0 + g8 * 8 + e;
                const double x = (v < nv && c < Nt) ? double(U[v * ldu + c]) * inv : 0.0;
                float one[X::kSlices];
                tcs::u_slices<X::kSlices>(x, one);
#pragma unroll
                for (int q = 0; q < X::kSlices; ++q) sl[q][e] = one[q];
            }
#pragma unroll
            for (int q = 0; q < X::kSlices; ++q)
                *reinterpret_cast<uint4*>(base + X::kCoordBytes + q * kBSlice + kmajor_offset(v, g8 * 8, kBSub)) =
                    make_uint4(pack_bf16(sl[q][0], sl[q][1]), pack_bf16(sl[q][2], sl[q][3]),
                               pack_bf16(sl[q][4], sl[q][5]), pack_bf16(sl[q][6], sl[q][7]));
        }
    }
}

// part slot (b, seg) holds [kNB][kRows] doubles: sigma_v 2^-8 / gscale times the row sums
template <int CLS, int KIND>
__global__ void __launch_bounds__(Tx<CLS>::kThreads, Tx<CLS>::kCtasPerSm)
covmv_tcx_kernel(CovParams cp, const unsigned char* __restrict__ img, int nv, const double* __restrict__ sigma,
                 double* __restrict__ part, int64_t len, int64_t T, int maxseg, int* __restrict__ status) {
    using X = Tx<CLS>;
    constexpr int kSlices = X::kSlices, kAccs = X::kAccs, kAStage = X::kAStage, kImg = X::kImg;
    constexpr int kOffA = X::kOffA, kOffImg = X::kOffImg, kOffTab = X::kOffTab, kOffBar = X::kOffBar;
    constexpr int kOffTmem = X::kOffTmem, kCoordBytes = X::kCoordBytes;
    constexpr int kBarLoaded = X::kBarLoaded, kBarFull = X::kBarFull, kBarEmpty = X::kBarEmpty;
    constexpr int kBarBlkDone = X::kBarBlkDone, kBarBlkFree = X::kBarBlkFree;
    constexpr int kProducers = X::kProducers, kLoaderWarp = X::kLoaderWarp, kMmaWarp = X::kMmaWarp;
    constexpr int kVpt = X::kVpt, kTmemCols = X::kTmemCols, kTmemBuf = X::kTmemBuf;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + kOffBar;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffTmem);
    float* stab = reinterpret_cast<float*>(smem + kOffTab);

    if (tid < 128) stab[tid] = cp.tabdf[tid];
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(bar0 + 8 * (kBarLoaded + st), 1);
            mbar_init(bar0 + 8 * (kBarFull + st), kProducers);
            mbar_init(bar0 + 8 * (kBarEmpty + st), 1);
        }
        for (int p = 0; p < 2; ++p) {
            mbar_init(bar0 + 8 * (kBarBlkDone + p), 1);
            mbar_init(bar0 + 8 * (kBarBlkFree + p), kProducers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int64_t G = gridDim.x;
    const int64_t t0 = tile_begin(blockIdx.x, T, G);
    const int ntiles = int(tile_begin(int64_t(blockIdx.x) + 1, T, G) - t0);
    const int64_t Nt = cp.Nt;
    const float gscale = cp.gscale;
    bool ok = true;

    if (warp < kLoaderWarp) {
        // ------------------------------ producers ------------------------------
        const int r = tid & (kRows - 1), qd = tid / kRows;   // row in block; columns and vectors qd*kVpt..
        const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
        int seg = 0, nb = 0, qseg = 0;   // segment, drain block, chunk within the segment
        int64_t rb = -1;
        float rc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const float* rsrc = CLS == 64 ? cp.Pdf : cp.P32;
        // the row's double-float sums, two vectors to a packed pair (vectors 2w and 2w + 1)
        df2::P acc2[kVpt / 2];
#pragma unroll
        for (int w = 0; w < kVpt / 2; ++w) acc2[w] = df2::P{df2::dup(0.f), df2::dup(0.f)};
        bool pend = false, pend_seg_end = false;
        int pend_nb = 0, pend_seg = 0;
        int64_t pend_rb = 0;
        // add drain block nb's level accumulators into the double-float sums; at a segment end
        // write the row's sums to the segment's partial slot.  False if the wait gave up.
        auto drain = [&](int dnb, bool dseg_end, int64_t drb, int dseg) -> bool {
            const int dp = dnb & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(bar0 + 8 * (kBarBlkDone + dp), uint32_t((dnb >> 1) & 1))))
                return false;
            fence_after_sync();
#pragma unroll
            for (int g8 = 0; g8 < kVpt / 8; ++g8) {
                float L[kAccs][8];
#pragma unroll
                for (int a = 0; a < kAccs; ++a)
                    tmem_ld8(tmem + lane_base + uint32_t(dp * kTmemBuf + a * 32 + qd * kVpt + g8 * 8), L[a]);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    df2::P& A = acc2[g8 * 4 + w];
#pragma unroll
                    for (int a = 0; a < kAccs; ++a) df2::acc_add(A, df2::mk(L[a][2 * w], L[a][2 * w + 1]));
                    A = df2::fast_two_sum(A.h, A.l);
                }
            }
            fence_before_sync();
            mbar_arrive(bar0 + 8 * (kBarBlkFree + dp));
            if (dseg_end) {
                if (drb * kRows + r < Nt) {
                    double* slot = part + (int64_t(blockIdx.x) * maxseg + dseg) * (int64_t(kNB) * kRows) + r;
#pragma unroll
                    for (int v = 0; v < kVpt; ++v) {
                        const int vv = qd * kVpt + v;
                        const df2::P& A = acc2[v / 2];
                        const float h = (v & 1) ? df2::hi(A.h) : df2::lo(A.h);
                        const float l = (v & 1) ? df2::hi(A.l) : df2::lo(A.l);
                        if (vv < nv) slot[vv * kRows] = (double(h) + double(l)) * (sigma[vv] * 0.00390625 / double(gscale));
                    }
                }
#pragma unroll
                for (int w = 0; w < kVpt / 2; ++w) acc2[w] = df2::P{df2::dup(0.f), df2::dup(0.f)};
            }
            return true;
        };
        for (int i = 0; i < ntiles; ++i) {
            const int64_t t = t0 + i;
            if (t / len != rb) {
                rb = t / len;
                const int64_t row = rb * kRows + r;
#pragma unroll
                for (int k = 0; k < X::kCoords; ++k) rc[k] = row < Nt ? rsrc[k * cp.ldp + row] : 0.f;
            }
            if (i == 0 || t % len == 0) qseg = 0;
            const int st = i % kStages;
            ok = __all_sync(0xffffffffu, mbar_wait(bar0 + 8 * (kBarLoaded + st), uint32_t((i / kStages) & 1)));
            if (!ok) break;
            const float* img_c = reinterpret_cast<const float*>(smem + kOffImg + st * kImg);
#pragma unroll
            for (int g8 = 0; g8 < kVpt / 8; ++g8) {
                // the 8 columns qd*kVpt + g8*8 .. +7; the float32 class reads their coordinates as
                // float4 pairs, the float64 class as float2 pairs per two columns (fewer live registers)
                const int c0 = qd * kVpt + g8 * 8;
                float cv[3][8];
                if constexpr (CLS == 32) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float4 a = *reinterpret_cast<const float4*>(img_c + k * kChunk + c0);
                        const float4 b = *reinterpret_cast<const float4*>(img_c + k * kChunk + c0 + 4);
                        cv[k][0] = a.x; cv[k][1] = a.y; cv[k][2] = a.z; cv[k][3] = a.w;
                        cv[k][4] = b.x; cv[k][5] = b.y; cv[k][6] = b.z; cv[k][7] = b.w;
                    }
                }
                uint32_t w[kSlices][4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    if constexpr (CLS == 64 && KIND != KL_K_POLY_TEST) {
                        // the two columns e, e + 1 in the two lanes of packed pairs (bit-identical
                        // to evaluating them one after the other)
                        df2::V r6[6], c6[6];
#pragma unroll
                        for (int k = 0; k < 6; ++k) {
                            r6[k] = df2::dup(rc[k]);
                            c6[k] = df2::V{*reinterpret_cast<const unsigned long long*>(img_c + k * kChunk + c0 + e)};
                        }
                        const df2::P g = df2::kernel_df<KIND>(r6, c6, stab, stab + 64);
                        df2::V o2[6];
                        df2::slices6(g, o2);
#pragma unroll
                        for (int q = 0; q < kSlices; ++q) w[q][e / 2] = pack_bf16(df2::lo(o2[q]), df2::hi(o2[q]));
                    } else if constexpr (CLS == 32 && KIND != KL_K_POLY_TEST) {
                        // float32 class: the two columns e, e + 1 in packed pairs (bit-identical)
                        const df2::V dx = df2::sub(df2::dup(rc[0]), df2::mk(cv[0][e], cv[0][e + 1]));
                        const df2::V dy = df2::sub(df2::dup(rc[1]), df2::mk(cv[1][e], cv[1][e + 1]));
                        const df2::V dz = df2::sub(df2::dup(rc[2]), df2::mk(cv[2][e], cv[2][e + 1]));
                        df2::V o2[3];
                        df2::slices3(df2::kernel32<KIND>(dx, dy, dz), o2);
#pragma unroll
                        for (int q = 0; q < kSlices; ++q) w[q][e / 2] = pack_bf16(df2::lo(o2[q]), df2::hi(o2[q]));
                    } else {
                        float o[2][kSlices];
                        float2 cp2[CLS == 64 ? 6 : 1];
                        if constexpr (CLS == 64) {
#pragma unroll
                            for (int k = 0; k < 6; ++k)
                                cp2[k] = *reinterpret_cast<const float2*>(img_c + k * kChunk + c0 + e);
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            if constexpr (CLS == 64) {
                                float c6[6];
#pragma unroll
                                for (int k = 0; k < 6; ++k) c6[k] = h ? cp2[k].y : cp2[k].x;
                                F2 g = df::kernel_df<KIND>(rc, c6, cp.poly_m, stab, stab + 64);
                                if (KIND == KL_K_POLY_TEST) {   // the other kernels have gscale = 1
                                    g.h = __fmul_rn(g.h, gscale);
                                    g.l = __fmul_rn(g.l, gscale);
                                }
                                slices6(g, o[h]);
                            } else {
                                const float x1 = cv[0][e + h], y1 = cv[1][e + h], z1 = cv[2][e + h];
                                const float g = kernel32<KIND>(rc[0] - x1, rc[1] - y1, rc[2] - z1, rc[0], rc[1],
                                                               rc[2], x1, y1, z1, cp.poly_m);
                                slices3(KIND == KL_K_POLY_TEST ? __fmul_rn(g, gscale) : g, o[h]);
                            }
                        }
#pragma unroll
                        for (int q = 0; q < kSlices; ++q) w[q][e / 2] = pack_bf16(o[0][q], o[1][q]);
                    }
                }
                unsigned char* As = smem + kOffA + st * kAStage + kmajor_offset(r, c0, kASub);
#pragma unroll
                for (int q = 0; q < kSlices; ++q)
                    *reinterpret_cast<uint4*>(As + q * kASlice) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
            }
            fence_proxy_async();
            mbar_arrive(bar0 + 8 * (kBarFull + st));

            // drain the block that ended one tile ago (its MMAs have had this tile's evaluation
            // time to finish; the accumulators are double-buffered, so the tensor core is already
            // filling the other buffer)
            if (pend) {
                ok = drain(pend_nb, pend_seg_end, pend_rb, pend_seg);
                if (!ok) break;
                pend = false;
            }
            const bool seg_end = (i == ntiles - 1) || ((t + 1) % len == 0);
            const bool blk_end = seg_end || (qseg % kDrainChunks == kDrainChunks - 1);
            ++qseg;
            if (blk_end) {
                pend = true;
                pend_nb = nb++;
                pend_seg_end = seg_end;
                pend_rb = rb;
                pend_seg = seg;
                if (seg_end) ++seg;
            }
        }
        if (ok && pend) ok = drain(pend_nb, pend_seg_end, pend_rb, pend_seg);
    } else if (warp == kLoaderWarp) {
        // ------------------------------ loader ------------------------------
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < ntiles; ++i) {
                const int st = i % kStages;
                if (i >= kStages) {
                    ok = mbar_wait(bar0 + 8 * (kBarEmpty + st), uint32_t(((i / kStages) - 1) & 1));
                    if (!ok) break;
                }
                const int64_t ch = (t0 + i) % len;
                bulk_load(sbase + kOffImg + st * kImg, img + ch * kImg, kImg, bar0 + 8 * (kBarLoaded + st));
                issued = i + 1;
            }
            if (!ok) {
                for (int i = issued - kStages; i < issued; ++i)
                    if (i >= 0) mbar_wait(bar0 + 8 * (kBarLoaded + i % kStages), uint32_t((i / kStages) & 1));
            }
        }
        __syncwarp();
    } else {
        // ------------------------------ MMA issuer ------------------------------
        if (lane == 0) {
            int nb = 0, qseg = 0, committed = 0;
            for (int i = 0; i < ntiles; ++i) {
                const int64_t t = t0 + i;
                const int st = i % kStages;
                const uint32_t ph = uint32_t((i / kStages) & 1);
                const bool seg_begin = (i == 0) || (t % len == 0);
                if (seg_begin) qseg = 0;
                const bool blk_begin = seg_begin || (qseg % kDrainChunks == 0);
                const bool seg_end = (i == ntiles - 1) || ((t + 1) % len == 0);
                const bool blk_end = seg_end || (qseg % kDrainChunks == kDrainChunks - 1);
                const int dp = nb & 1;
                if (blk_begin && nb >= 2) {
                    ok = mbar_wait(bar0 + 8 * (kBarBlkFree + dp), uint32_t(((nb >> 1) - 1) & 1));
                    if (!ok) break;
                }
                ok = mbar_wait(bar0 + 8 * (kBarFull + st), ph);
                if (!ok) break;
                ok = mbar_wait(bar0 + 8 * (kBarLoaded + st), ph);
                if (!ok) break;
                fence_after_sync();
                const uint32_t a0 = sbase + kOffA + st * kAStage;
                const uint32_t b0 = sbase + kOffImg + st * kImg + kCoordBytes;
#pragma unroll
                for (int ks = 0; ks < kChunk / kK; ++ks) {
#pragma unroll
                    for (int q = 0; q < X::kProducts; ++q) {
                        int s, u, a;
                        bool first;
                        product<CLS>(q, &s, &u, &a, &first);
                        const uint32_t d = tmem + uint32_t(dp * kTmemBuf + a * 32);
                        const bool fresh = first && ks == 0 && blk_begin;
                        mma_bf16(d, make_desc(a0 + s * kASlice + ks * kASub, 128, 256),
                                 make_desc(b0 + u * kBSlice + ks * kBSub, 128, 256), kIdesc, fresh ? 0u : 1u);
                    }
                }
                mma_commit(bar0 + 8 * (kBarEmpty + st));
                committed = i + 1;
                if (blk_end) {
                    mma_commit(bar0 + 8 * (kBarBlkDone + dp));
                    ++nb;
                }
                ++qseg;
            }
            if (!ok && committed > 0) {
                const int last = committed - 1;
                mbar_wait(bar0 + 8 * (kBarEmpty + last % kStages), uint32_t((last / kStages) & 1));
            }
        }
        __syncwarp();
    }
    fence_before_sync();
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    fence_after_sync();
    if (!ok && tid == 0) atomicExch(status, int(KL_ERR_TIMEOUT));
    if (warp == kMmaWarp) tmem_dealloc(tmem, kTmemCols);
}

template <int CLS, int KIND>
cudaError_t launch_kind(const CovParams& cp, const unsigned char* im, int g, const double* sigma, double* part,
                        const Schedule& sc, int* status, cudaStream_t s) {
    // the attribute is only ever set to this kernel's one value (safe from concurrent callers)
    cudaError_t e = cudaFuncSetAttribute(covmv_tcx_kernel<CLS, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Tx<CLS>::kSmemBytes);
    if (e != cudaSuccess) return e;
    covmv_tcx_kernel<CLS, KIND><<<unsigned(sc.G), Tx<CLS>::kThreads, Tx<CLS>::kSmemBytes, s>>>(
        cp, im, g, sigma, part, sc.len, sc.T, sc.maxseg, status);
    return cudaGetLastError();
}

template <int CLS, typename TU>
cudaError_t launch_tcx(const CovParams& cp, const TU* U, int64_t ldu, int nvec, double* Z, int64_t ldz, double scale2,
                       const double* J, double* part, void* img, int* status, cudaStream_t s) {
    using X = Tx<CLS>;
    const int64_t Nt = cp.Nt;
    if (Nt == 0 || nvec == 0) return cudaSuccess;
    Schedule sc;
    cudaError_t e = make_schedule(Nt, kRows, kChunk, X::kCtasPerSm, &sc);
    if (e != cudaSuccess) return e;
    unsigned char* im = static_cast<unsigned char*>(img);
    const int64_t nchunks = sc.len;
    double* sigma = reinterpret_cast<double*>(im + nchunks * X::kImg);
    const int img_blocks = int(nchunks < int64_t(num_sms()) * 8 ? nchunks : int64_t(num_sms()) * 8);
    const float* P = CLS == 64 ? cp.Pdf : cp.P32;
    for (int v0 = 0; v0 < nvec; v0 += kNB) {
        const int g = (nvec - v0) < kNB ? (nvec - v0) : kNB;
        const TU* Ug = U + int64_t(v0) * ldu;
        tcx_scale_kernel<TU><<<g, 256, 0, s>>>(Ug, ldu, Nt, sigma);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        tcx_image_kernel<CLS, TU><<<img_blocks, 6 * kChunk, 0, s>>>(P, cp.ldp, Nt, Ug, ldu, g, sigma, im, nchunks);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        switch (cp.kind) {
            case KL_K_EXP: e = launch_kind<CLS, KL_K_EXP>(cp, im, g, sigma, part, sc, status, s); break;
            case KL_K_GAUSS: e = launch_kind<CLS, KL_K_GAUSS>(cp, im, g, sigma, part, sc, status, s); break;
            case KL_K_EXP_SEPARABLE:
                e = launch_kind<CLS, KL_K_EXP_SEPARABLE>(cp, im, g, sigma, part, sc, status, s);
                break;
            default: e = launch_kind<CLS, KL_K_POLY_TEST>(cp, im, g, sigma, part, sc, status, s);
        }
        if (e != cudaSuccess) return e;
        const int64_t tot = Nt * g;
        int blocks = int((tot + 255) / 256);
        if (blocks > num_sms() * 8) blocks = num_sms() * 8;
        slot_reduce<kRows, kNB><<<blocks, 256, 0, s>>>(part, Nt, g, sc.len, sc.T, sc.G, sc.maxseg,
                                                       Z + int64_t(v0) * ldz, ldz, scale2, J);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        count_launches(4);
    }
    return cudaSuccess;
}

template <int CLS>
size_t part_doubles(int64_t Nt) {
    Schedule sc;
    if (Nt <= 0 || make_schedule(Nt, kRows, kChunk, Tx<CLS>::kCtasPerSm, &sc) != cudaSuccess) return 0;
    return size_t(sc.G) * size_t(sc.maxseg) * kNB * kRows;
}

// ------------------------------------------------------------------------------------------
// Symmetric float64-class kernel: each kernel value serves the pairs (k, l) and (l, k)
// ------------------------------------------------------------------------------------------
// Row block I (128 rows) is paired with the column chunks c >= 4I only: the four chunks of its
// own 128 x 128 diagonal block (row side only: it holds both (k, l) and (l, k)) and every chunk
// of the column blocks J > I.  For an off-diagonal chunk the kernel values are used twice:
//   * row side, as in covmv_tcx_kernel: D1[row][v] += Gamma[row][col] (u/sigma)[col][v];
//   * column side: D2[v][col] += (u/sigma)[row][v]^T Gamma[row][col] over the block's 128 rows,
//     with A = the row block's u slices (K-major, vectors on M, rows on K; M = 128 with lanes
//     32..127 unused) and B = the same kernel-value slices read MN-major (columns on N, rows
//     on K: the 16-byte rows of the values' core matrices are 8 consecutive columns).
// The value slices are stored with a uniform core-matrix grid (8-row groups 512 bytes apart,
// 8-column groups 128 bytes apart) so that both descriptors address them: K-major for the row
// side (leading byte offset 128, stride byte offset 512), MN-major for the column side (leading
// byte offset 512 between the K groups of rows, stride byte offset 128 between the N groups of
// columns).  The column side's level sums over the 128 rows are exact like the row side's over
// 128 columns; they are drained after every chunk by the four warps that own tensor-memory
// lanes 0..31 (one per vector), combined in double-float and added into a float64 column-sum
// array with atomic additions (the only step whose summation order is not fixed), which the
// final reduction adds to the row sums.
constexpr int kSymStages = 2;
constexpr int kRowU = 4 * kBSlice * 6;            // the row block's u slices: 4 chunks x 6 slices x 2 KB
constexpr int kRowUPad = 4096;                    // lanes 32..127 of the column-side A operand read past the end
struct Ts {
    using X = Tx<64>;
    static constexpr int kOffA = 0;
    static constexpr int kOffImg = kOffA + kSymStages * X::kAStage;
    static constexpr int kOffRowU = kOffImg + kSymStages * X::kImg;
    static constexpr int kOffTab = kOffRowU + kRowU + kRowUPad;
    static constexpr int kOffBar = kOffTab + 128 * 4;
    static constexpr int kBarLoaded = 0, kBarFull = kSymStages, kBarEmpty = 2 * kSymStages;
    static constexpr int kBarBlkDone = 3 * kSymStages, kBarBlkFree = kBarBlkDone + 2;
    static constexpr int kBarRowU = kBarBlkFree + 2, kBarRowUFree = kBarRowU + 1;
    static constexpr int kBarD2Done = kBarRowUFree + 1, kBarD2Free = kBarD2Done + 1;
    static constexpr int kNumBars = kBarD2Free + 1;
    static constexpr int kOffTmem = kOffBar + 8 * kNumBars;
    static constexpr int kSmemBytes = kOffTmem + 16;
    static constexpr int kD2Col = 320;            // column-side accumulators after the row side's 2 x 5 x 32
    // producers, loader, row-side and column-side MMA issuers
    static constexpr int kThreads = Tx<64>::kProducers + 96;
    static_assert(kOffRowU % 16 == 0 && kOffBar % 8 == 0, "bulk-copy and mbarrier alignment");
    static_assert(kSmemBytes <= 227 * 1024, "shared memory");
};

// tiles before row block I: sum over I' < I of (len - 4 I')
__host__ __device__ __forceinline__ int64_t sym_tiles_before(int64_t I, int64_t len) { return I * len - 2 * I * (I - 1); }

// row block and chunk of tile t
__host__ __device__ __forceinline__ void sym_tile(int64_t t, int64_t len, int64_t* I, int64_t* c) {
    const double a = double(len) + 2.0;
    int64_t i = int64_t((a - sqrt(fmax(a * a - 8.0 * double(t), 0.0))) * 0.25);
    if (i < 0) i = 0;
    while (i > 0 && sym_tiles_before(i, len) > t) --i;
    while (sym_tiles_before(i + 1, len) <= t && len - 4 * (i + 1) > 0) ++i;
    *I = i;
    *c = 4 * i + (t - sym_tiles_before(i, len));
}

struct SymSchedule {
    int64_t len = 0, rb = 0, T = 0, G = 0;
};

inline cudaError_t make_sym_schedule(int64_t Nt, SymSchedule* sc) {
    sc->len = (Nt + kChunk - 1) / kChunk;
    sc->rb = (Nt + kRows - 1) / kRows;
    sc->T = sym_tiles_before(sc->rb, sc->len);
    sc->G = int64_t(num_sms());
    if (sc->G > sc->T) sc->G = sc->T;
    if (sc->G < 1) sc->G = 1;
    return cudaSuccess;
}

// Symmetric float64-class kernel.  part slot b + I (kNB x kRows doubles) holds CTA b's row sums
// of row block I; zcol[v * Nt + col] receives the column sums (scaled like the row sums).
template <int KIND>
__global__ void __launch_bounds__(Ts::kThreads, 1)
covmv_tcs_kernel(CovParams cp, const unsigned char* __restrict__ img, int nv, const double* __restrict__ sigma,
                 double* __restrict__ part, double* __restrict__ zcol, int64_t len, int64_t T,
                 int* __restrict__ status) {
    using X = Tx<64>;
    constexpr int kSlices = X::kSlices, kAccs = X::kAccs, kAStage = X::kAStage, kImg = X::kImg;
    constexpr int kCoordBytes = X::kCoordBytes, kProducers = X::kProducers;
    constexpr int kVpt = X::kVpt;
    // warps 0..15 producers (warps 0, 4, 8, 12 also drain the column side: tensor-memory lanes
    // 0..31), 16 loader, 17 row-side MMA issuer (allocates tensor memory), 18 column-side MMA issuer
    constexpr int kLoaderWarp = 16, kMmaWarp = 17, kMma2Warp = 18;
    constexpr int kTmemCols = X::kTmemCols, kTmemBuf = 160;   // row side: 2 buffers x 5 x 32 columns
    constexpr int kOffA = Ts::kOffA, kOffImg = Ts::kOffImg, kOffRowU = Ts::kOffRowU, kOffTab = Ts::kOffTab;
    constexpr int kOffBar = Ts::kOffBar, kOffTmem = Ts::kOffTmem;
    constexpr int kBarLoaded = Ts::kBarLoaded, kBarFull = Ts::kBarFull, kBarEmpty = Ts::kBarEmpty;
    constexpr int kBarBlkDone = Ts::kBarBlkDone, kBarBlkFree = Ts::kBarBlkFree;
    constexpr int kBarRowU = Ts::kBarRowU, kBarRowUFree = Ts::kBarRowUFree;
    constexpr int kBarD2Done = Ts::kBarD2Done, kBarD2Free = Ts::kBarD2Free;
    constexpr uint32_t kIdesc2 = idesc_bf16(kRows, kNB) | (1u << 16);   // B read MN-major
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + kOffBar;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffTmem);
    float* stab = reinterpret_cast<float*>(smem + kOffTab);

    if (tid < 128) stab[tid] = cp.tabdf[tid];
    // the pad read by the unused lanes of the column-side A operand: finite (zero) values
    for (int e = tid; e < kRowUPad / 16; e += blockDim.x)
        reinterpret_cast<uint4*>(smem + kOffRowU + kRowU)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int st = 0; st < kSymStages; ++st) {
            mbar_init(bar0 + 8 * (kBarLoaded + st), 1);
            mbar_init(bar0 + 8 * (kBarFull + st), kProducers);
            mbar_init(bar0 + 8 * (kBarEmpty + st), 2);   // both MMA issuers commit
        }
        for (int p = 0; p < 2; ++p) {
            mbar_init(bar0 + 8 * (kBarBlkDone + p), 1);
            mbar_init(bar0 + 8 * (kBarBlkFree + p), kProducers);
        }
        mbar_init(bar0 + 8 * kBarRowU, 1);
        mbar_init(bar0 + 8 * kBarRowUFree, 1);
        mbar_init(bar0 + 8 * kBarD2Done, 1);
        mbar_init(bar0 + 8 * kBarD2Free, 4);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const int64_t G = gridDim.x;
    const int64_t t0 = tile_begin(blockIdx.x, T, G);
    const int ntiles = int(tile_begin(int64_t(blockIdx.x) + 1, T, G) - t0);
    int I0, c0;
    {
        int64_t Iw, cw;
        sym_tile(t0, len, &Iw, &cw);
        I0 = int(Iw);
        c0 = int(cw);
    }
    const int lenc = int(len);
    const int64_t Nt = cp.Nt;
    bool ok = true;

    if (warp < kLoaderWarp) {
        // ------------------------------ producers ------------------------------
        const int r = tid & (kRows - 1), qd = tid / kRows;   // row in block; columns and vectors qd*kVpt..
        const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
        const bool d2_warp = (warp & 3) == 0;                 // owns tensor-memory lanes 0..31 (the vectors)
        int nb = 0, qseg = 0;
        int I = I0, c = c0, rb = -1;
        float rc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        F2 acc[kVpt];
#pragma unroll
        for (int v = 0; v < kVpt; ++v) acc[v] = F2{0.f, 0.f};
        bool pend = false, pend_seg_end = false;
        int pend_nb = 0;
        int pend_rb = 0;
        bool pend2 = false;                                   // column-side sums of the previous tile
        int n2p = 0;                                          // column-side uses produced so far
        int pend2_c = 0;
        const double cscale = 0.00390625 / double(cp.gscale);
        // row side: add drain block dnb's level accumulators into the double-float sums; at a
        // segment end write the row's sums to the segment's partial slot.  False if the wait gave up.
        auto drain = [&](int dnb, bool dseg_end, int drb) -> bool {
            const int dp = dnb & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(bar0 + 8 * (kBarBlkDone + dp), uint32_t((dnb >> 1) & 1))))
                return false;
            fence_after_sync();
            float L[kAccs][8];
#pragma unroll
            for (int a = 0; a < kAccs; ++a)
                tmem_ld8(tmem + lane_base + uint32_t(dp * kTmemBuf + a * 32 + qd * kVpt), L[a]);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
#pragma unroll
                for (int a = 0; a < kAccs; ++a) df_acc(acc[v], L[a][v]);
                acc[v] = df::fast_two_sum(acc[v].h, acc[v].l);
            }
            fence_before_sync();
            mbar_arrive(bar0 + 8 * (kBarBlkFree + dp));
            if (dseg_end) {
                if (int64_t(drb) * kRows + r < Nt) {
                    // slot b + I of row block I: a CTA's segments take consecutive slots and the next
                    // CTA starts at or after its last row block, so slots never collide
                    double* slot = part + (int64_t(blockIdx.x) + drb) * (int64_t(kNB) * kRows) + r;
#pragma unroll
                    for (int v = 0; v < kVpt; ++v) {
                        const int vv = qd * kVpt + v;
                        if (vv < nv) slot[vv * kRows] = (double(acc[v].h) + double(acc[v].l)) * (sigma[vv] * cscale);
                    }
                }
#pragma unroll
                for (int v = 0; v < kVpt; ++v) acc[v] = F2{0.f, 0.f};
            }
            return true;
        };
        // column side (warps 0, 4, 8, 12): the level sums of chunk dc for vector = lane and columns
        // 8 (warp / 4) .. + 7, added in float64 (the level sums are exact float32 values, and the
        // float64 pipe is otherwise idle) into the column-sum array
        auto drain2 = [&](int dn2, int dc) -> bool {
            if (!__all_sync(0xffffffffu, mbar_wait(bar0 + 8 * kBarD2Done, uint32_t(dn2 & 1)))) return false;
            fence_after_sync();
            const int jq = warp >> 2;
            uint32_t L[kAccs][8];
#pragma unroll
            for (int a = 0; a < kAccs; ++a) tmem_ld8_nowait(tmem + uint32_t(Ts::kD2Col + a * 32 + 8 * jq), L[a]);
            tmem_ld_wait();
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar0 + 8 * kBarD2Free);
            if (lane < nv) {
                const double sc = sigma[lane] * cscale;
                double* zc = zcol + int64_t(lane) * Nt + int64_t(dc) * kChunk + 8 * jq;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    double x = double(__uint_as_float(L[0][j]));
#pragma unroll
                    for (int a = 1; a < kAccs; ++a) x += double(__uint_as_float(L[a][j]));
                    if (int64_t(dc) * kChunk + 8 * jq + j < Nt) atomicAdd(zc + j, x * sc);
                }
            }
            return true;
        };
        for (int i = 0; i < ntiles; ++i) {
            if (I != rb) {
                rb = I;
                const int64_t row = int64_t(rb) * kRows + r;
#pragma unroll
                for (int k = 0; k < 6; ++k) rc[k] = row < Nt ? cp.Pdf[k * cp.ldp + row] : 0.f;
            }
            if (i == 0 || c == 4 * I) qseg = 0;
            const int st = i % kSymStages;
            ok = __all_sync(0xffffffffu, mbar_wait(bar0 + 8 * (kBarLoaded + st), uint32_t((i / kSymStages) & 1)));
            if (!ok) break;
            const float* img_c = reinterpret_cast<const float*>(smem + kOffImg + st * kImg);
            {
                // the 8 columns qd*8 .. +7, coordinates read as float2 pairs per two columns
                const int cc = qd * kVpt;
                uint32_t w[kSlices][4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    float o[2][kSlices];
                    float2 cp2[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) cp2[k] = *reinterpret_cast<const float2*>(img_c + k * kChunk + cc + e);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float c6[6];
#pragma unroll
                        for (int k = 0; k < 6; ++k) c6[k] = h ? cp2[k].y : cp2[k].x;
                        F2 g = df::kernel_df<KIND>(rc, c6, cp.poly_m, stab, stab + 64);
                        if (KIND == KL_K_POLY_TEST) {   // the other kernels have gscale = 1
                            g.h = __fmul_rn(g.h, cp.gscale);
                            g.l = __fmul_rn(g.l, cp.gscale);
                        }
                        slices6(g, o[h]);
                    }
#pragma unroll
                    for (int q = 0; q < kSlices; ++q) w[q][e / 2] = pack_bf16(o[0][q], o[1][q]);
                }
                // uniform core-matrix grid: 8-row groups 512 bytes apart, 8-column groups 128
                unsigned char* As = smem + kOffA + st * kAStage + (r >> 3) * 512 + (cc >> 3) * 128 + (r & 7) * 16;
#pragma unroll
                for (int q = 0; q < kSlices; ++q)
                    *reinterpret_cast<uint4*>(As + q * kASlice) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
            }
            fence_proxy_async();
            mbar_arrive(bar0 + 8 * (kBarFull + st));

            // deferred drains of the previous tile's accumulators (the tensor core has had this
            // tile's evaluation time to finish them)
            if (pend) {
                ok = drain(pend_nb, pend_seg_end, pend_rb);
                if (!ok) break;
                pend = false;
            }
            if (pend2) {
                if (d2_warp) {
                    ok = drain2(n2p - 1, pend2_c);
                    if (!ok) break;
                }
                pend2 = false;
            }
            const bool seg_end = (i == ntiles - 1) || (c == lenc - 1);
            const bool blk_end = seg_end || (qseg % kDrainChunks == kDrainChunks - 1);
            ++qseg;
            if (blk_end) {
                pend = true;
                pend_nb = nb++;
                pend_seg_end = seg_end;
                pend_rb = rb;
            }
            if (c >= 4 * I + 4) {   // off the diagonal block: the column side follows
                pend2 = true;
                pend2_c = c;
                ++n2p;
            }
            if (++c == lenc) {
                ++I;
                c = 4 * I;
            }
        }
        if (ok && pend) ok = drain(pend_nb, pend_seg_end, pend_rb);
        if (ok && pend2 && d2_warp) ok = drain2(n2p - 1, pend2_c);
    } else if (warp == kLoaderWarp) {
        // ------------------------------ loader ------------------------------
        if (lane == 0) {
            int issued = 0, krow = 0;
            int I = I0, c = c0, prevI = -1;
            for (int i = 0; i < ntiles; ++i) {
                const int st = i % kSymStages;
                if (i >= kSymStages) {
                    ok = mbar_wait(bar0 + 8 * (kBarEmpty + st), uint32_t(((i / kSymStages) - 1) & 1));
                    if (!ok) break;
                }
                if (I != prevI) {
                    // the row block's u slices (chunks 4I .. 4I+3 of the image; the image holds
                    // zero chunks up to 4 x row blocks) once the previous row block's MMAs are done
                    if (krow >= 1) {
                        ok = mbar_wait(bar0 + 8 * kBarRowUFree, uint32_t((krow - 1) & 1));
                        if (!ok) break;
                    }
                    const uint32_t rbar = bar0 + 8 * kBarRowU;
                    mbar_expect_tx(rbar, uint32_t(kRowU));
                    for (int q = 0; q < 4; ++q)
                        bulk_copy_tx(sbase + kOffRowU + q * (kRowU / 4), img + int64_t(4 * I + q) * kImg + kCoordBytes,
                                     uint32_t(kRowU / 4), rbar);
                    ++krow;
                    prevI = I;
                }
                bulk_load(sbase + kOffImg + st * kImg, img + int64_t(c) * kImg, kImg, bar0 + 8 * (kBarLoaded + st));
                issued = i + 1;
                if (++c == lenc) {
                    ++I;
                    c = 4 * I;
                }
            }
            if (!ok) {
                for (int i = issued - kSymStages; i < issued; ++i)
                    if (i >= 0) mbar_wait(bar0 + 8 * (kBarLoaded + i % kSymStages), uint32_t((i / kSymStages) & 1));
                if (krow >= 1) mbar_wait(bar0 + 8 * kBarRowU, uint32_t((krow - 1) & 1));
            }
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ------------------------------ row-side MMA issuer ------------------------------
        if (lane == 0) {
            int nb = 0, qseg = 0, committed = 0;
            int I = I0, c = c0;
            // descriptor low words: start address >> 4 in bits 0..13 (addresses stay below 256 KB,
            // so constant offsets never carry out of the field); high words are constant
            const uint32_t dA = uint32_t(make_desc(sbase + kOffA, 128, 512));
            const uint32_t dB = uint32_t(make_desc(sbase + kOffImg + kCoordBytes, 128, 256));
            const uint32_t hA = uint32_t(make_desc(0, 128, 512) >> 32), hB = uint32_t(make_desc(0, 128, 256) >> 32);
            for (int i = 0; i < ntiles; ++i) {
                const int st = i % kSymStages;
                const uint32_t ph = uint32_t((i / kSymStages) & 1);
                const bool seg_begin = (i == 0) || (c == 4 * I);
                if (seg_begin) qseg = 0;
                const bool blk_begin = seg_begin || (qseg % kDrainChunks == 0);
                const bool seg_end = (i == ntiles - 1) || (c == lenc - 1);
                const bool blk_end = seg_end || (qseg % kDrainChunks == kDrainChunks - 1);
                const int dp = nb & 1;
                if (blk_begin && nb >= 2) {
                    ok = mbar_wait(bar0 + 8 * (kBarBlkFree + dp), uint32_t(((nb >> 1) - 1) & 1));
                    if (!ok) break;
                }
                ok = mbar_wait(bar0 + 8 * (kBarFull + st), ph);
                if (!ok) break;
                ok = mbar_wait(bar0 + 8 * (kBarLoaded + st), ph);
                if (!ok) break;
                fence_after_sync();
                const uint32_t a0 = dA + uint32_t((st * kAStage) >> 4), b0 = dB + uint32_t((st * kImg) >> 4);
                const uint32_t d0 = tmem + uint32_t(dp * kTmemBuf);
                // row side: values K-major (columns on K), u slices of the chunk's columns
#pragma unroll
                for (int ks = 0; ks < kChunk / kK; ++ks) {
#pragma unroll
                    for (int q = 0; q < X::kProducts; ++q) {
                        int sl, ul, a;
                        bool first;
                        product<64>(q, &sl, &ul, &a, &first);
                        const bool fresh = first && ks == 0 && blk_begin;
                        mma_bf16_lo(d0 + uint32_t(a * 32), a0 + uint32_t((sl * kASlice + ks * 256) >> 4), hA,
                                    b0 + uint32_t((ul * kBSlice + ks * kBSub) >> 4), hB, kIdesc, fresh ? 0u : 1u);
                    }
                }
                mma_commit(bar0 + 8 * (kBarEmpty + st));
                committed = i + 1;
                if (blk_end) {
                    mma_commit(bar0 + 8 * (kBarBlkDone + dp));
                    ++nb;
                }
                ++qseg;
                if (++c == lenc) {
                    ++I;
                    c = 4 * I;
                }
            }
            if (!ok && committed > 0) {
                const int last = committed - 1;
                mbar_wait(bar0 + 8 * (kBarEmpty + last % kSymStages), uint32_t((last / kSymStages) & 1));
            }
        }
        __syncwarp();
    } else if (warp == kMma2Warp) {
        // ------------------------------ column-side MMA issuer ------------------------------
        if (lane == 0) {
            int committed = 0, krow = 0, n2 = 0;
            int I = I0, c = c0, curI = -1;
            const uint32_t dU = uint32_t(make_desc(sbase + kOffRowU, 128, 256));
            const uint32_t dV = uint32_t(make_desc(sbase + kOffA, 512, 128));
            const uint32_t hU = uint32_t(make_desc(0, 128, 256) >> 32), hV = uint32_t(make_desc(0, 512, 128) >> 32);
            for (int i = 0; i < ntiles; ++i) {
                const int st = i % kSymStages;
                const uint32_t ph = uint32_t((i / kSymStages) & 1);
                const bool seg_end = (i == ntiles - 1) || (c == lenc - 1);
                const bool offdiag = c >= 4 * I + 4;
                if (I != curI) {
                    ok = mbar_wait(bar0 + 8 * kBarRowU, uint32_t(krow & 1));
                    if (!ok) break;
                    ++krow;
                    curI = I;
                }
                // every tile, also on the diagonal: this issuer's Empty commit for tile i must not
                // come before the stage holds tile i (it would complete an earlier use's phase)
                ok = mbar_wait(bar0 + 8 * (kBarFull + st), ph);
                if (!ok) break;
                ok = mbar_wait(bar0 + 8 * (kBarLoaded + st), ph);
                if (!ok) break;
                if (offdiag) {
                    if (n2 >= 1) {
                        ok = mbar_wait(bar0 + 8 * kBarD2Free, uint32_t((n2 - 1) & 1));
                        if (!ok) break;
                    }
                    fence_after_sync();
                    // u slices of the row block (vectors on M, rows on K) times the values read
                    // MN-major (rows on K, columns on N)
                    const uint32_t v0 = dV + uint32_t((st * kAStage) >> 4);
                    const uint32_t d0 = tmem + uint32_t(Ts::kD2Col);
#pragma unroll
                    for (int kk = 0; kk < kRows / kK; ++kk) {
#pragma unroll
                        for (int q = 0; q < X::kProducts; ++q) {
                            int sl, ul, a;
                            bool first;
                            product<64>(q, &sl, &ul, &a, &first);
                            mma_bf16_lo(d0 + uint32_t(a * 32),
                                        dU + uint32_t(((kk >> 1) * (kRowU / 4) + ul * kBSlice + (kk & 1) * kBSub) >> 4), hU,
                                        v0 + uint32_t((sl * kASlice + kk * 1024) >> 4), hV, kIdesc2,
                                        (first && kk == 0) ? 0u : 1u);
                        }
                    }
                    mma_commit(bar0 + 8 * kBarD2Done);
                    ++n2;
                }
                // every tile: the stage is free of this issuer's reads (at once on the diagonal)
                mma_commit(bar0 + 8 * (kBarEmpty + st));
                committed = i + 1;
                if (seg_end) mma_commit(bar0 + 8 * kBarRowUFree);
                if (++c == lenc) {
                    ++I;
                    c = 4 * I;
                }
            }
            if (!ok && committed > 0) {
                const int last = committed - 1;
                mbar_wait(bar0 + 8 * (kBarEmpty + last % kSymStages), uint32_t((last / kSymStages) & 1));
            }
        }
        __syncwarp();
    }
    fence_before_sync();
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    fence_after_sync();
    if (!ok && tid == 0) atomicExch(status, int(KL_ERR_TIMEOUT));
    if (warp == kMmaWarp) tmem_dealloc(tmem, kTmemCols);
}
// z[v][r] = scale2 J[r] (row sums from the partial slots of r's row block, CTAs in increasing order,
// + the column sums)
__global__ void tcs_reduce(const double* __restrict__ part, const double* __restrict__ zcol, int64_t Nt, int nv,
                           int64_t len, int64_t T, int64_t G, double* __restrict__ Z, int64_t ldz, double scale2,
                           const double* __restrict__ J) {
    const int64_t total = Nt * nv;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t v = idx / Nt, r = idx - v * Nt;
        const int64_t rb = r / kRows, rl = r - rb * kRows;
        const int64_t tlo = sym_tiles_before(rb, len), thi = sym_tiles_before(rb + 1, len) - 1;
        const int64_t blo = ((tlo + 1) * G - 1) / T, bhi = ((thi + 1) * G - 1) / T;
        double acc = 0.0;
        for (int64_t b = blo; b <= bhi; ++b) acc += part[((b + rb) * kNB + v) * kRows + rl];
        acc += zcol[v * Nt + r];
        acc *= scale2;
        if (J) acc *= J[r];
        Z[v * ldz + r] = acc;
    }
}

template <int KIND>
cudaError_t launch_tcs_kind(const CovParams& cp, const unsigned char* im, int g, const double* sigma, double* slots,
                            double* zcol, const SymSchedule& sc, int* status, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(covmv_tcs_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Ts::kSmemBytes);
    if (e != cudaSuccess) return e;
    covmv_tcs_kernel<KIND><<<unsigned(sc.G), Ts::kThreads, Ts::kSmemBytes, s>>>(cp, im, g, sigma, slots, zcol,
                                                                                      sc.len, sc.T, status);
    return cudaGetLastError();
}

bool g_tc_symmetric = false;

}  // namespace

void set_tc_symmetric(bool on) { g_tc_symmetric = on; }
bool tc_symmetric_used(int64_t Nt) { return g_tc_symmetric && Nt >= 2 * kRows; }

// workspace of the symmetric float64-class kernel: G + row blocks partial slots, then the column
// sums (32 x Ntilde doubles); the image holds 4 chunks per row block
size_t covmv_tcs64_part_doubles(int64_t Nt) {
    SymSchedule sc;
    if (Nt <= 0 || make_sym_schedule(Nt, &sc) != cudaSuccess) return 0;
    return size_t(sc.G + sc.rb) * kNB * kRows + size_t(Nt) * kNB;
}
size_t covmv_tcs64_image_bytes(int64_t Nt) {
    return size_t(4 * ((Nt + kRows - 1) / kRows)) * Tx<64>::kImg + kNB * sizeof(double);
}

cudaError_t launch_covmv_tcs64(const CovParams& cp, const double* U, int64_t ldu, int nvec, double* Z, int64_t ldz,
                               double scale2, const double* J, double* part, void* img, int* status, cudaStream_t s) {
    using X = Tx<64>;
    const int64_t Nt = cp.Nt;
    if (Nt == 0 || nvec == 0) return cudaSuccess;
    SymSchedule sc;
    cudaError_t e = make_sym_schedule(Nt, &sc);
    if (e != cudaSuccess) return e;
    unsigned char* im = static_cast<unsigned char*>(img);
    const int64_t nchunks = 4 * sc.rb;
    double* sigma = reinterpret_cast<double*>(im + nchunks * X::kImg);
    double* slots = part;
    double* zcol = part + (sc.G + sc.rb) * kNB * kRows;
    const int img_blocks = int(nchunks < int64_t(num_sms()) * 8 ? nchunks : int64_t(num_sms()) * 8);
    for (int v0 = 0; v0 < nvec; v0 += kNB) {
        const int g = (nvec - v0) < kNB ? (nvec - v0) : kNB;
        const double* Ug = U + int64_t(v0) * ldu;
        tcx_scale_kernel<double><<<g, 256, 0, s>>>(Ug, ldu, Nt, sigma);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        tcx_image_kernel<64, double><<<img_blocks, 6 * kChunk, 0, s>>>(cp.Pdf, cp.ldp, Nt, Ug, ldu, g, sigma, im,
                                                                      nchunks);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(zcol, 0, size_t(Nt) * g * sizeof(double), s);
        if (e != cudaSuccess) return e;
        switch (cp.kind) {
            case KL_K_EXP: e = launch_tcs_kind<KL_K_EXP>(cp, im, g, sigma, slots, zcol, sc, status, s); break;
            case KL_K_GAUSS: e = launch_tcs_kind<KL_K_GAUSS>(cp, im, g, sigma, slots, zcol, sc, status, s); break;
            case KL_K_EXP_SEPARABLE:
                e = launch_tcs_kind<KL_K_EXP_SEPARABLE>(cp, im, g, sigma, slots, zcol, sc, status, s);
                break;
            default: e = launch_tcs_kind<KL_K_POLY_TEST>(cp, im, g, sigma, slots, zcol, sc, status, s);
        }
        if (e != cudaSuccess) return e;
        const int64_t tot = Nt * g;
        int blocks = int((tot + 255) / 256);
        if (blocks > num_sms() * 8) blocks = num_sms() * 8;
        tcs_reduce<<<blocks, 256, 0, s>>>(slots, zcol, Nt, g, sc.len, sc.T, sc.G, Z + int64_t(v0) * ldz, ldz,
                                          scale2, J);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        count_launches(4);
    }
    return cudaSuccess;
}

size_t covmv_tc64_part_doubles(int64_t Nt) { return part_doubles<64>(Nt); }
size_t covmv_tc_part_doubles(int64_t Nt) { return part_doubles<32>(Nt); }

// image bytes followed by the 32 per-vector scales
size_t covmv_tc64_image_bytes(int64_t Nt) {
    return size_t((Nt + kChunk - 1) / kChunk) * Tx<64>::kImg + kNB * sizeof(double);
}
size_t covmv_tc_image_bytes(int64_t Nt) {
    return size_t((Nt + kChunk - 1) / kChunk) * Tx<32>::kImg + kNB * sizeof(double);
}

cudaError_t launch_covmv_tc64(const CovParams& cp, const double* U, int64_t ldu, int nvec, double* Z, int64_t ldz,
                              double scale2, const double* J, double* part, void* img, int* status, cudaStream_t s) {
    return launch_tcx<64, double>(cp, U, ldu, nvec, Z, ldz, scale2, J, part, img, status, s);
}

cudaError_t launch_covmv_tc(const CovParams& cp, const float* U, int64_t ldu, int nvec, double* Z, int64_t ldz,
                            double scale2, const double* J, double* part, void* img, int* status, cudaStream_t s) {
    return launch_tcx<32, float>(cp, U, ldu, nvec, Z, ldz, scale2, J, part, img, status, s);
}

}  // namespace kl
