// Stage 5 of Algorithm 1 with float64-level accuracy on the tensor cores (tcgen05, sm_103a),
// for groups of up to 32 right-hand sides: z = Gamma u.
//
// Exact slicing.  Each kernel value g (double-float, ~48 bits, scaled so |g| <= 1) is written
// as g = sum_{s<6} a_s 2^(-8(s+1)) with integer digits |a_s| <= 256 (round-to-nearest digit
// extraction, every step exact), and each u value, after division by a per-vector power of two
// sigma >= max|u|, as u/sigma = sum_{t<6} b_t 2^(-8(t+1)).  The digits are stored as bfloat16
// "slices" a_s 2^(-8s) and b_t 2^(-8t), which bfloat16 holds exactly (at most 8 significant
// bits).  The tensor core forms the slice products exactly and adds them in float32:
//   levels 0-3 (1, 2, 3 and 4 products): partial sums over 128 columns are multiples of
//     2^-8d below 2^(24-8d), hence exact in float32 whatever the tensor core's rounding;
//   levels 4-5 (11 products, relative size <= 2^-32) share a fifth accumulator, whose float32
//     rounding (truncating or not) stays below ~2^-49 of the sum;
// all five are drained every 128 columns into double-float accumulators.
// Products of levels >= 6 are dropped (relative size < 2^-48).  The result carries a relative
// error of ~1e-14 like the double-float kernel, with every multiply-add on the tensor cores.
//
// Pipeline and schedule as in the float32 tensor-core kernel (persistent tile ranges,
// loader / producers / MMA issuer synchronised by mbarriers), one CTA per SM:
//   * loader (one thread): bulk copy per 32-column chunk of a pre-staged image holding the
//     column coordinates (double-float) and the u slices (tc64_image_kernel);
//   * producers (16 warps, four threads per row, 8 columns each): kernel values in double-float
//     (the evaluation of the double-float kernel), six slices each, written K-major;
//   * MMA issuer (one thread): 21 MMAs per 16 columns into five tensor-memory accumulators,
//     double-buffered per 128-column drain block.
// Every wait is bounded (~2 s), after which the CTA records KL_ERR_TIMEOUT, drains its own
// asynchronous operations and returns.
#include "df64.cuh"
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
constexpr int kSlices = 6;
constexpr int kDrainChunks = 4;                   // exact accumulators drained every 128 columns
constexpr int kProducers = 512;                   // warps 0-15
constexpr int kThreads = kProducers + 64;         // + loader warp 16 + MMA warp 17
constexpr int kLoaderWarp = kProducers / 32;
constexpr int kMmaWarp = kLoaderWarp + 1;
// tensor memory (512 columns): accumulator a (level 0, 1, 2, 3, levels 4-5) of drain block
// parity dp at dp*256 + a*32
constexpr int kTmemCols = 512;
constexpr int kTmemBuf = 256;
constexpr int kAccs = 5;

constexpr int kASub = kRows * kK * 2;             // 128 x 16 bf16: 4 KB
constexpr int kASlice = kASub * (kChunk / kK);    // 8 KB
constexpr int kAStage = kASlice * kSlices;        // 48 KB
constexpr int kBSub = kNB * kK * 2;               // 32 x 16 bf16: 1 KB
constexpr int kBSlice = kBSub * (kChunk / kK);    // 2 KB
constexpr int kCoordBytes = 6 * kChunk * 4;       // heads x, y, z then tails x, y, z
constexpr int kImg = kCoordBytes + kBSlice * kSlices;   // 13056 B
constexpr int kOffA = 0;
constexpr int kOffImg = kOffA + kStages * kAStage;
constexpr int kOffTab = kOffImg + kStages * kImg;       // 2^(-j/64) heads and tails
constexpr int kOffBar = kOffTab + 128 * 4;
constexpr int kBarLoaded = 0, kBarFull = kStages, kBarEmpty = 2 * kStages;
constexpr int kBarBlkDone = 3 * kStages, kBarBlkFree = kBarBlkDone + 2;
constexpr int kNumBars = kBarBlkFree + 2;
constexpr int kOffTmem = kOffBar + 8 * kNumBars;
constexpr int kSmemBytes = kOffTmem + 16;
constexpr uint32_t kIdesc = idesc_bf16(kRows, kNB);
static_assert(kImg % 16 == 0 && kOffImg % 16 == 0 && kOffBar % 8 == 0, "bulk-copy and mbarrier alignment");
static_assert(kSmemBytes <= 227 * 1024, "shared memory");

// the 21 slice products (a_s, b_t) with s + t <= 5, grouped by accumulator: level 0, 1, 2, 3,
// then levels 4-5 together
constexpr int kNumProducts = 21;
__device__ __forceinline__ void product(int q, int* s, int* t, int* acc, bool* first) {
    constexpr int S[kNumProducts] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5};
    constexpr int T[kNumProducts] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0};
    *s = S[q];
    *t = T[q];
    *acc = q == 0 ? 0 : q < 3 ? 1 : q < 6 ? 2 : q < 10 ? 3 : 4;
    *first = (q == 0 || q == 1 || q == 3 || q == 6 || q == 10);
}

// integer digit of x * scale by round-to-nearest (|x * scale| < 2^22), and the exact remainder
__device__ __forceinline__ float digit(float& x, float scale) {
    const float magic = 12582912.0f;   // 1.5 * 2^23
    const float p = __fsub_rn(__fmaf_rn(x, scale, magic), magic);
    x = __fmaf_rn(x, scale, -p);
    return p;
}

// six slices a_s 2^(-8s) of a double-float g with |g| <= 1 (see the file comment); the tail
// joins the remainder after the three head digits
__device__ __forceinline__ void slices6(F2 g, float* out) {
    float x = g.h;
    out[0] = digit(x, 256.f);
    out[1] = __fmul_rn(digit(x, 256.f), 0.00390625f);
    out[2] = __fmul_rn(digit(x, 256.f), 1.52587890625e-05f);
    x = __fmaf_rn(g.l, 16777216.f, x);   // remainder is in units of 2^-24
    out[3] = __fmul_rn(digit(x, 256.f), 5.9604644775390625e-08f);
    out[4] = __fmul_rn(digit(x, 256.f), 2.3283064365386963e-10f);
    out[5] = __fmul_rn(digit(x, 256.f), 9.0949470177292824e-13f);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// acc += x for a float x (exact two-sum into the head, tail accumulated)
__device__ __forceinline__ void df_acc(F2& acc, float x) {
    const F2 s = df::two_sum(acc.h, x);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, s.l);
}

// sigma[v] = 2^e with 2^(e-1) <= max_c |u[v][c]| < 2^e (1 when the column is zero)
__global__ void tc64_scale_kernel(const double* __restrict__ U, int64_t ldu, int64_t Nt, double* __restrict__ sigma) {
    __shared__ double red[256];
    const int v = blockIdx.x;
    double m = 0.0;
    for (int64_t c = threadIdx.x; c < Nt; c += blockDim.x) m = fmax(m, fabs(U[v * ldu + c]));
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

// Image of column chunk ch: double-float coordinates (zero past Ntilde) and the six u slices
// of the group in the K-major operand layout (rows = vectors, zero past nv and Ntilde).
__global__ void tc64_image_kernel(const float* __restrict__ Pdf, int64_t ldp, int64_t Nt, const double* __restrict__ U,
                                  int64_t ldu, int nv, const double* __restrict__ sigma,
                                  unsigned char* __restrict__ img, int64_t nchunks) {
    const int t = threadIdx.x;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        unsigned char* base = img + ch * kImg;
        const int64_t c0 = ch * kChunk;
        if (t < 6 * kChunk) {
            const int64_t c = c0 + (t % kChunk);
            reinterpret_cast<float*>(base)[t] = c < Nt ? Pdf[int64_t(t / kChunk) * ldp + c] : 0.f;
        }
        if (t < kNB * (kChunk / 8)) {
            const int v = t / (kChunk / 8), g8 = t % (kChunk / 8);
            const double inv = (v < nv) ? 1.0 / sigma[v] : 0.0;   // a power of two: exact
            float sl[kSlices][8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t c = c0 + g8 * 8 + e;
                double x = (v < nv && c < Nt) ? U[v * ldu + c] * inv : 0.0;
                double w = 1.0;
#pragma unroll
                for (int q = 0; q < kSlices; ++q) {
                    const double p = rint(x * 256.0);
                    x = fma(x, 256.0, -p);   // exact
                    sl[q][e] = float(p * w);  // |p| <= 256: exact in bfloat16 after scaling
                    w *= 0.00390625;
                }
            }
#pragma unroll
            for (int q = 0; q < kSlices; ++q)
                *reinterpret_cast<uint4*>(base + kCoordBytes + q * kBSlice + kmajor_offset(v, g8 * 8, kBSub)) =
                    make_uint4(pack_bf16(sl[q][0], sl[q][1]), pack_bf16(sl[q][2], sl[q][3]),
                               pack_bf16(sl[q][4], sl[q][5]), pack_bf16(sl[q][6], sl[q][7]));
        }
    }
}

// part slot (b, seg) holds [kNB][kRows] doubles: sigma_v 2^-16 / gscale times the row sums
template <int KIND>
__global__ void __launch_bounds__(kThreads, 1)
covmv_tc64_kernel(CovParams cp, const unsigned char* __restrict__ img, int nv, const double* __restrict__ sigma,
                  double* __restrict__ part, int64_t len, int64_t T, int maxseg, int* __restrict__ status) {
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
        const int r = tid & (kRows - 1), qd = tid / kRows;   // row in block; columns and vectors qd*8..qd*8+7
        const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
        int seg = 0, nb = 0, qseg = 0;
        int64_t rb = -1;
        float rc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        F2 acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = F2{0.f, 0.f};
        for (int i = 0; i < ntiles; ++i) {
            const int64_t t = t0 + i;
            if (t / len != rb) {
                rb = t / len;
                const int64_t row = rb * kRows + r;
#pragma unroll
                for (int k = 0; k < 6; ++k) rc[k] = row < Nt ? cp.Pdf[k * cp.ldp + row] : 0.f;
            }
            if (i == 0 || t % len == 0) qseg = 0;
            const int st = i % kStages;
            ok = __all_sync(0xffffffffu, mbar_wait(bar0 + 8 * (kBarLoaded + st), uint32_t((i / kStages) & 1)));
            if (!ok) break;
            const float* cc = reinterpret_cast<const float*>(smem + kOffImg + st * kImg) + qd * 8;
            uint32_t w[kSlices][4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float o[2][kSlices];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float c6[6] = {cc[e + h], cc[kChunk + e + h], cc[2 * kChunk + e + h],
                                         cc[3 * kChunk + e + h], cc[4 * kChunk + e + h], cc[5 * kChunk + e + h]};
                    F2 g = df::kernel_df<KIND>(rc, c6, cp.poly_m, stab, stab + 64);
                    g.h = __fmul_rn(g.h, gscale);
                    g.l = __fmul_rn(g.l, gscale);
                    slices6(g, o[h]);
                }
#pragma unroll
                for (int q = 0; q < kSlices; ++q) w[q][e / 2] = pack_bf16(o[0][q], o[1][q]);
            }
            unsigned char* As = smem + kOffA + st * kAStage + kmajor_offset(r, qd * 8, kASub);
#pragma unroll
            for (int q = 0; q < kSlices; ++q)
                *reinterpret_cast<uint4*>(As + q * kASlice) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
            fence_proxy_async();
            mbar_arrive(bar0 + 8 * (kBarFull + st));

            const bool seg_end = (i == ntiles - 1) || ((t + 1) % len == 0);
            const bool blk_end = seg_end || (qseg % kDrainChunks == kDrainChunks - 1);
            ++qseg;
            if (blk_end) {
                // drain the five accumulators into the double-float sums
                const int dp = nb & 1;
                ok = __all_sync(0xffffffffu, mbar_wait(bar0 + 8 * (kBarBlkDone + dp), uint32_t((nb >> 1) & 1)));
                if (!ok) break;
                fence_after_sync();
                float L[kAccs][8];
#pragma unroll
                for (int a = 0; a < kAccs; ++a)
                    tmem_ld8(tmem + lane_base + uint32_t(dp * kTmemBuf + a * 32 + qd * 8), L[a]);
                fence_before_sync();
                mbar_arrive(bar0 + 8 * (kBarBlkFree + dp));
#pragma unroll
                for (int v = 0; v < 8; ++v) {
#pragma unroll
                    for (int a = 0; a < kAccs; ++a) df_acc(acc[v], L[a][v]);
                    acc[v] = df::fast_two_sum(acc[v].h, acc[v].l);
                }
                ++nb;
                if (seg_end) {
                    if (rb * kRows + r < Nt) {
                        double* slot = part + (int64_t(blockIdx.x) * maxseg + seg) * (int64_t(kNB) * kRows) + r;
#pragma unroll
                        for (int v = 0; v < 8; ++v) {
                            const int vv = qd * 8 + v;
                            if (vv < nv)
                                slot[vv * kRows] = (double(acc[v].h) + double(acc[v].l)) *
                                                   (sigma[vv] * 1.52587890625e-05 / double(gscale));
                        }
                    }
#pragma unroll
                    for (int v = 0; v < 8; ++v) acc[v] = F2{0.f, 0.f};
                    ++seg;
                }
            }
        }
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
                    for (int q = 0; q < kNumProducts; ++q) {
                        int s, u, a;
                        bool first;
                        product(q, &s, &u, &a, &first);
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

cudaError_t set_smem_attr(int kind) {
    switch (kind) {
        case KL_K_EXP:
            return cudaFuncSetAttribute(covmv_tc64_kernel<KL_K_EXP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kSmemBytes);
        case KL_K_GAUSS:
            return cudaFuncSetAttribute(covmv_tc64_kernel<KL_K_GAUSS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kSmemBytes);
        case KL_K_EXP_SEPARABLE:
            return cudaFuncSetAttribute(covmv_tc64_kernel<KL_K_EXP_SEPARABLE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        default:
            return cudaFuncSetAttribute(covmv_tc64_kernel<KL_K_POLY_TEST>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    }
}

}  // namespace

size_t covmv_tc64_part_doubles(int64_t Nt) {
    Schedule sc;
    if (Nt <= 0 || make_schedule(Nt, kRows, kChunk, 1, &sc) != cudaSuccess) return 0;
    return size_t(sc.G) * size_t(sc.maxseg) * kNB * kRows;
}

// image bytes followed by the 32 per-vector scales
size_t covmv_tc64_image_bytes(int64_t Nt) { return size_t((Nt + kChunk - 1) / kChunk) * kImg + kNB * sizeof(double); }

cudaError_t launch_covmv_tc64(const CovParams& cp, const double* U, int64_t ldu, int nvec, double* Z, int64_t ldz,
                              double scale2, const double* J, double* part, void* img, int* status, cudaStream_t s) {
    const int64_t Nt = cp.Nt;
    if (Nt == 0 || nvec == 0) return cudaSuccess;
    Schedule sc;
    cudaError_t e = make_schedule(Nt, kRows, kChunk, 1, &sc);
    if (e != cudaSuccess) return e;
    e = set_smem_attr(cp.kind);
    if (e != cudaSuccess) return e;
    unsigned char* im = static_cast<unsigned char*>(img);
    const int64_t nchunks = sc.len;
    double* sigma = reinterpret_cast<double*>(im + nchunks * kImg);
    const int img_blocks = int(nchunks < 152 * 8 ? nchunks : 152 * 8);
    for (int v0 = 0; v0 < nvec; v0 += kNB) {
        const int g = (nvec - v0) < kNB ? (nvec - v0) : kNB;
        const double* Ug = U + int64_t(v0) * ldu;
        tc64_scale_kernel<<<g, 256, 0, s>>>(Ug, ldu, Nt, sigma);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        tc64_image_kernel<<<img_blocks, 6 * kChunk, 0, s>>>(cp.Pdf, cp.ldp, Nt, Ug, ldu, g, sigma, im, nchunks);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const dim3 grid(unsigned(sc.G));
        switch (cp.kind) {
            case KL_K_EXP:
                covmv_tc64_kernel<KL_K_EXP><<<grid, kThreads, kSmemBytes, s>>>(cp, im, g, sigma, part, sc.len, sc.T,
                                                                               sc.maxseg, status);
                break;
            case KL_K_GAUSS:
                covmv_tc64_kernel<KL_K_GAUSS><<<grid, kThreads, kSmemBytes, s>>>(cp, im, g, sigma, part, sc.len,
                                                                                 sc.T, sc.maxseg, status);
                break;
            case KL_K_EXP_SEPARABLE:
                covmv_tc64_kernel<KL_K_EXP_SEPARABLE><<<grid, kThreads, kSmemBytes, s>>>(cp, im, g, sigma, part,
                                                                                         sc.len, sc.T, sc.maxseg,
                                                                                         status);
                break;
            default:
                covmv_tc64_kernel<KL_K_POLY_TEST><<<grid, kThreads, kSmemBytes, s>>>(cp, im, g, sigma, part, sc.len,
                                                                                     sc.T, sc.maxseg, status);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t tot = Nt * g;
        int blocks = int((tot + 255) / 256);
        if (blocks > 152 * 8) blocks = 152 * 8;
        slot_reduce<kRows, kNB><<<blocks, 256, 0, s>>>(part, Nt, g, sc.len, sc.T, sc.G, sc.maxseg,
                                                       Z + int64_t(v0) * ldz, ldz, scale2, J);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        count_launches(4);
    }
    return cudaSuccess;
}

}  // namespace kl
