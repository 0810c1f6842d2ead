// Stage 5 of Algorithm 1 as a tensor-core block contraction (tcgen05, sm_103a), for blocks of
// 16 right-hand sides: z = Gamma u with Gamma generated tile by tile in registers and never
// stored in global memory.
//
// A CTA owns 128 rows (the MMA M dimension) and a contiguous range of columns.  For every
// 32-column chunk each thread evaluates the float32 kernel values of its row (MUFU rsqrt/ex2,
// same arithmetic as the scalar float32 kernel) and writes them to shared memory split into
// three bfloat16 terms g = g1 + g2 + g3 (8 significant bits each, 24 together); the u block is
// split the same way.  One elected thread then issues tcgen05.mma (kind::f16, bf16 inputs,
// float32 accumulation in tensor memory) for the six products g_a u_b with a + b <= 4, which
// reproduce float32 products to ~2^-24.  Two shared-memory stages alternate so the kernel
// values of chunk i+1 are computed while the tensor core consumes chunk i; completion is
// tracked with tcgen05.commit on an mbarrier per stage.  At the end each warp reads its 32
// accumulator lanes with tcgen05.ld and writes float64 split partials (combined by
// covmv_reduce as for the other stage-5 kernels).
//
// Every wait is bounded: after ~2 s of spinning a CTA records an error in a device status word,
// waits (again bounded) for its own MMAs, releases its tensor memory and returns; the launcher
// reports KL_ERR_TIMEOUT.
#include <cuda_bf16.h>

#include "kernel32.cuh"
#include "tc_common.cuh"

// Stage 5 of Algorithm 1 as a tensor-core block contraction (tcgen05, sm_103a) for groups of up
// to 32 right-hand sides: z = Gamma u, with Gamma generated tile by tile in registers and never
// stored in global memory.
//
// Work decomposition.  Rows come in blocks of 128 (the MMA M dimension), columns in chunks of 32;
// a (row block, column chunk) pair is a tile.  The tiles, ordered row block by row block, are cut
// into one contiguous range per CTA (persistent grid of resident CTAs), so every CTA does the same
// number of tiles; a range covers at most a few row blocks ("segments").  Each segment's sums go
// to a partial slot, and a fixed-order reduction adds the slots of a row block.
//
// Per CTA, three roles run as a pipeline over shared-memory stages, synchronised by mbarriers:
//   * loader (one thread): one bulk copy per chunk of a pre-staged image holding the 32 column
//     coordinates and the u chunk already split into bfloat16 terms (written by tc_image_kernel);
//   * producers (eight warps, two threads per row, 16 columns each): evaluate float32 kernel
//     values (MUFU rsqrt/ex2, as in the scalar float32 kernel), split each into three bfloat16
//     terms by truncation (g = g1 + g2 + g3 exactly), and write them K-major to shared memory;
//   * MMA issuer (one thread): six tcgen05.mma per 16 columns (kind::f16, bf16 x bf16, float32
//     accumulation in tensor memory) for the term products g_a u_b with a + b <= 4 (1-based),
//     which reproduce float32 products to ~2^-24, then tcgen05.commit to free the stage.
// At a segment end the producers read their accumulator lanes with tcgen05.ld; tensor memory holds
// four accumulator buffers so the next segment starts without waiting for that read.
//
// Every wait is bounded: after ~2 s of spinning a role records an error in a device status word,
// drains the asynchronous operations it started (again bounded), and the CTA releases its tensor
// memory and returns; the launcher's caller reports KL_ERR_TIMEOUT.
#include "kl_internal.h"

namespace kl {
namespace {

using namespace tc;

constexpr int kTcRows = 128;                      // MMA M (rows per block)
constexpr int kTcK = 16;                          // MMA K for 16-bit inputs
constexpr int kTcChunk = 32;                      // columns per pipeline stage (2 K-steps)
constexpr int kTcStages = 3;                      // shared-memory stages
constexpr int kTcNB = 32;                         // MMA N: vectors per group
constexpr int kTcNBuf = 4;                        // accumulator buffers in tensor memory
constexpr int kTcTmemCols = kTcNB * kTcNBuf;      // 128 columns (power of two >= 32)
constexpr int kTcProducers = 256;                 // warps 0-7: two threads per row, 16 columns each
constexpr int kTcThreads = kTcProducers + 64;     // + loader warp 8 + MMA warp 9
constexpr int kTcLoaderWarp = kTcProducers / 32;
constexpr int kTcMmaWarp = kTcLoaderWarp + 1;
constexpr int kTcPieces = 3;                      // bfloat16 terms per float32 value

// shared-memory layout (bytes); operand tiles are canonical K-major without swizzle: core
// matrices of 8 rows x 16 bytes, 256 bytes between 8-row groups, 128 bytes between 8-column halves
constexpr int kASub = kTcRows * kTcK * 2;                  // 128 x 16 bf16: 4 KB
constexpr int kAPiece = kASub * (kTcChunk / kTcK);         // 8 KB
constexpr int kAStage = kAPiece * kTcPieces;               // 24 KB
constexpr int kBSub = kTcNB * kTcK * 2;                    // 32 x 16 bf16: 1 KB
constexpr int kBPiece = kBSub * (kTcChunk / kTcK);         // 2 KB
constexpr int kCoordBytes = 3 * kTcChunk * 4;              // x[32], y[32], z[32] floats
constexpr int kImg = kCoordBytes + kBPiece * kTcPieces;    // one chunk image: 6528 B
constexpr int kOffA = 0;
constexpr int kOffImg = kOffA + kTcStages * kAStage;
constexpr int kOffBar = kOffImg + kTcStages * kImg;
constexpr int kBarLoaded = 0;                              // per stage: image copy landed (tx count)
constexpr int kBarFull = kTcStages;                        // per stage: one arrival per producer
constexpr int kBarEmpty = 2 * kTcStages;                   // per stage: MMAs done reading (commit)
constexpr int kBarSegDone = 3 * kTcStages;                 // per buffer: segment accumulated (commit)
constexpr int kBarTmemFree = 3 * kTcStages + kTcNBuf;      // per buffer: every producer read it
constexpr int kNumBars = 3 * kTcStages + 2 * kTcNBuf;
constexpr int kOffTmem = kOffBar + 8 * kNumBars;
constexpr int kSmemBytes = kOffTmem + 16;
constexpr uint32_t kIdesc = idesc_bf16(kTcRows, kTcNB);
static_assert(kImg % 16 == 0 && kOffImg % 16 == 0 && kOffBar % 8 == 0, "bulk-copy and mbarrier alignment");

// g = hi + mid + lo exactly, each term a bfloat16 (the upper 16 bits of the returned words):
// truncation keeps the leading 8 significant bits, and both subtractions are exact
__device__ __forceinline__ void split3(float g, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
    w0 = __float_as_uint(g) & 0xFFFF0000u;
    const float r1 = g - __uint_as_float(w0);
    w1 = __float_as_uint(r1) & 0xFFFF0000u;
    w2 = __float_as_uint(r1 - __uint_as_float(w1));
}

// two bfloat16 (upper halves of a and b) packed as elements (k, k+1)
__device__ __forceinline__ uint32_t pack_bf16(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x7632); }

// The image of column chunk ch: the chunk's coordinates (x[32], y[32], z[32], zero past Ntilde)
// and the group's u values split into three bfloat16 terms, in the K-major operand layout the
// MMA reads (rows = vectors, zero past nv and past Ntilde).  128 threads per chunk.
__global__ void tc_image_kernel(const float* __restrict__ P, int64_t ldp, int64_t Nt, const float* __restrict__ U,
                                int64_t ldu, int nv, unsigned char* __restrict__ img, int64_t nchunks) {
    const int t = threadIdx.x;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        unsigned char* base = img + ch * kImg;
        const int64_t c0 = ch * kTcChunk;
        if (t < 3 * kTcChunk) {
            const int64_t c = c0 + (t % kTcChunk);
            reinterpret_cast<float*>(base)[t] = c < Nt ? P[int64_t(t / kTcChunk) * ldp + c] : 0.f;
        }
        const int v = t / (kTcChunk / 8), g8 = t % (kTcChunk / 8);
        uint32_t w[kTcPieces][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const int64_t ca = c0 + g8 * 8 + e, cb = ca + 1;
            const float ua = (v < nv && ca < Nt) ? U[v * ldu + ca] : 0.f;
            const float ub = (v < nv && cb < Nt) ? U[v * ldu + cb] : 0.f;
            uint32_t a0, a1, a2, b0, b1, b2;
            split3(ua, a0, a1, a2);
            split3(ub, b0, b1, b2);
            w[0][e / 2] = pack_bf16(a0, b0);
            w[1][e / 2] = pack_bf16(a1, b1);
            w[2][e / 2] = pack_bf16(a2, b2);
        }
#pragma unroll
        for (int q = 0; q < kTcPieces; ++q)
            *reinterpret_cast<uint4*>(base + kCoordBytes + q * kBPiece + kmajor_offset(v, g8 * 8, kBSub)) =
                make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
}

// Persistent tile-range kernel (see the file comment).  len = column chunks per row block,
// T = row blocks x len; the partial sums of segment `seg` of CTA b go to slot b * maxseg + seg as
// [kTcNB][128] doubles (only v < nv and rows < Ntilde written).
template <int KIND>
__global__ void __launch_bounds__(kTcThreads)
covmv_tc_kernel(CovParams cp, const unsigned char* __restrict__ img, int nv, double* __restrict__ part, int64_t len,
                int64_t T, int maxseg, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + kOffBar;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffTmem);

    if (tid == 0) {
        for (int st = 0; st < kTcStages; ++st) {
            mbar_init(bar0 + 8 * (kBarLoaded + st), 1);
            mbar_init(bar0 + 8 * (kBarFull + st), kTcProducers);
            mbar_init(bar0 + 8 * (kBarEmpty + st), 1);
        }
        for (int bf = 0; bf < kTcNBuf; ++bf) {
            mbar_init(bar0 + 8 * (kBarSegDone + bf), 1);
            mbar_init(bar0 + 8 * (kBarTmemFree + bf), kTcProducers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == kTcMmaWarp) {
        tmem_alloc(smem_u32(tmem_slot), kTcTmemCols);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const int64_t G = gridDim.x;
    const int64_t t0 = tile_begin(blockIdx.x, T, G);
    const int ntiles = int(tile_begin(int64_t(blockIdx.x) + 1, T, G) - t0);
    const int64_t Nt = cp.Nt;
    bool ok = true;

    if (warp < kTcLoaderWarp) {
        // ------------------------------ producers ------------------------------
        const int r = tid & (kTcRows - 1), half = tid / kTcRows;   // row in block, column half
        int seg = 0;
        int64_t rb = -1;
        float x0 = 0.f, y0 = 0.f, z0 = 0.f;
        for (int i = 0; i < ntiles; ++i) {
            const int64_t t = t0 + i;
            if (t / len != rb) {
                rb = t / len;
                const int64_t row = rb * kTcRows + r;
                const bool rv = row < Nt;
                x0 = rv ? cp.P32[row] : 0.f;
                y0 = rv ? cp.P32[cp.ldp + row] : 0.f;
                z0 = rv ? cp.P32[2 * cp.ldp + row] : 0.f;
            }
            const int st = i % kTcStages;
            ok = __all_sync(0xffffffffu, mbar_wait(bar0 + 8 * (kBarLoaded + st), uint32_t((i / kTcStages) & 1)));
            if (!ok) break;
            const float* cx = reinterpret_cast<const float*>(smem + kOffImg + st * kImg);
            unsigned char* As = smem + kOffA + st * kAStage;
#pragma unroll
            for (int gg = 0; gg < 2; ++gg) {
                const int g8 = half * 2 + gg;
                const float4 xa = *reinterpret_cast<const float4*>(cx + g8 * 8);
                const float4 xb = *reinterpret_cast<const float4*>(cx + g8 * 8 + 4);
                const float4 ya = *reinterpret_cast<const float4*>(cx + kTcChunk + g8 * 8);
                const float4 yb = *reinterpret_cast<const float4*>(cx + kTcChunk + g8 * 8 + 4);
                const float4 za = *reinterpret_cast<const float4*>(cx + 2 * kTcChunk + g8 * 8);
                const float4 zb = *reinterpret_cast<const float4*>(cx + 2 * kTcChunk + g8 * 8 + 4);
                const float xs[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
                const float ys[8] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
                const float zs[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
                uint32_t w[kTcPieces][4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    const float ga = kernel32<KIND>(x0 - xs[e], y0 - ys[e], z0 - zs[e], x0, y0, z0, xs[e], ys[e],
                                                     zs[e], cp.poly_m);
                    const float gb = kernel32<KIND>(x0 - xs[e + 1], y0 - ys[e + 1], z0 - zs[e + 1], x0, y0, z0,
                                                     xs[e + 1], ys[e + 1], zs[e + 1], cp.poly_m);
                    uint32_t a0, a1, a2, b0, b1, b2;
                    split3(ga, a0, a1, a2);
                    split3(gb, b0, b1, b2);
                    w[0][e / 2] = pack_bf16(a0, b0);
                    w[1][e / 2] = pack_bf16(a1, b1);
                    w[2][e / 2] = pack_bf16(a2, b2);
                }
#pragma unroll
                for (int q = 0; q < kTcPieces; ++q)
                    *reinterpret_cast<uint4*>(As + q * kAPiece + kmajor_offset(r, g8 * 8, kASub)) =
                        make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(bar0 + 8 * (kBarFull + st));
            if (i == ntiles - 1 || (t + 1) % len == 0) {
                // segment end: read this row's accumulators (vectors half*16 .. half*16+15)
                const int bf = seg % kTcNBuf;
                ok = __all_sync(0xffffffffu,
                                mbar_wait(bar0 + 8 * (kBarSegDone + bf), uint32_t((seg / kTcNBuf) & 1)));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                uint32_t d[16];
                const uint32_t taddr =
                    tmem + (uint32_t((warp & 3) * 32) << 16) + uint32_t(bf * kTcNB + half * 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];\n"
                    : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
                      "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]),
                      "=r"(d[15])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                mbar_arrive(bar0 + 8 * (kBarTmemFree + bf));
                if (rb * kTcRows + r < Nt) {
                    double* slot = part + (int64_t(blockIdx.x) * maxseg + seg) * (int64_t(kTcNB) * kTcRows) + r;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (half * 16 + j < nv) slot[(half * 16 + j) * kTcRows] = double(__uint_as_float(d[j]));
                }
                ++seg;
            }
        }
    } else if (warp == kTcLoaderWarp) {
        // ------------------------------ loader ------------------------------
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < ntiles; ++i) {
                const int st = i % kTcStages;
                if (i >= kTcStages) {
                    ok = mbar_wait(bar0 + 8 * (kBarEmpty + st), uint32_t(((i / kTcStages) - 1) & 1));
                    if (!ok) break;
                }
                const int64_t ch = (t0 + i) % len;
                bulk_load(sbase + kOffImg + st * kImg, img + ch * kImg, kImg, bar0 + 8 * (kBarLoaded + st));
                issued = i + 1;
            }
            if (!ok) {
                // drain: the last copy issued into each stage must land before the CTA exits
                for (int i = issued - kTcStages; i < issued; ++i)
                    if (i >= 0) mbar_wait(bar0 + 8 * (kBarLoaded + i % kTcStages), uint32_t((i / kTcStages) & 1));
            }
        }
        __syncwarp();
    } else {
        // ------------------------------ MMA issuer ------------------------------
        if (lane == 0) {
            int seg = 0, committed = 0;
            for (int i = 0; i < ntiles; ++i) {
                const int64_t t = t0 + i;
                const int st = i % kTcStages;
                const uint32_t ph = uint32_t((i / kTcStages) & 1);
                const bool seg_begin = (i == 0) || (t % len == 0);
                const bool seg_end = (i == ntiles - 1) || ((t + 1) % len == 0);
                const int bf = seg % kTcNBuf;
                if (seg_begin && seg >= kTcNBuf) {
                    ok = mbar_wait(bar0 + 8 * (kBarTmemFree + bf), uint32_t(((seg / kTcNBuf) - 1) & 1));
                    if (!ok) break;
                }
                ok = mbar_wait(bar0 + 8 * (kBarFull + st), ph);
                if (!ok) break;
                ok = mbar_wait(bar0 + 8 * (kBarLoaded + st), ph);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a0 = sbase + kOffA + st * kAStage;
                const uint32_t b0 = sbase + kOffImg + st * kImg + kCoordBytes;
                const uint32_t dcol = tmem + uint32_t(bf * kTcNB);
                // term products (a, b), 0-based, with a + b <= 2
                const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
                for (int ks = 0; ks < kTcChunk / kTcK; ++ks) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const uint64_t ad = make_desc(a0 + pa[q] * kAPiece + ks * kASub, 128, 256);
                        const uint64_t bd = make_desc(b0 + pb[q] * kBPiece + ks * kBSub, 128, 256);
                        mma_bf16(dcol, ad, bd, kIdesc, (seg_begin && ks == 0 && q == 0) ? 0u : 1u);
                    }
                }
                mma_commit(bar0 + 8 * (kBarEmpty + st));
                committed = i + 1;
                if (seg_end) {
                    mma_commit(bar0 + 8 * (kBarSegDone + bf));
                    ++seg;
                }
            }
            if (!ok && committed > 0) {
                // drain: a commit tracks every earlier MMA of this thread
                const int last = committed - 1;
                mbar_wait(bar0 + 8 * (kBarEmpty + last % kTcStages), uint32_t((last / kTcStages) & 1));
            }
        }
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok && tid == 0) atomicExch(status, int(KL_ERR_TIMEOUT));
    if (warp == kTcMmaWarp)
        tmem_dealloc(tmem, kTcTmemCols);
}

cudaError_t set_smem_attr(int kind) {
    switch (kind) {
        case KL_K_EXP:
            return cudaFuncSetAttribute(covmv_tc_kernel<KL_K_EXP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kSmemBytes);
        case KL_K_GAUSS:
            return cudaFuncSetAttribute(covmv_tc_kernel<KL_K_GAUSS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kSmemBytes);
        case KL_K_EXP_SEPARABLE:
            return cudaFuncSetAttribute(covmv_tc_kernel<KL_K_EXP_SEPARABLE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        default:
            return cudaFuncSetAttribute(covmv_tc_kernel<KL_K_POLY_TEST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kSmemBytes);
    }
}

}  // namespace

size_t covmv_tc_part_doubles(int64_t Nt) {
    Schedule sc;
    if (Nt <= 0 || make_schedule(Nt, kTcRows, kTcChunk, 2, &sc) != cudaSuccess) return 0;
    return size_t(sc.G) * size_t(sc.maxseg) * kTcNB * kTcRows;
}

size_t covmv_tc_image_bytes(int64_t Nt) { return size_t((Nt + kTcChunk - 1) / kTcChunk) * kImg; }

cudaError_t launch_covmv_tc(const CovParams& cp, const float* U, int64_t ldu, int nvec, double* Z, int64_t ldz,
                            double scale2, const double* J, double* part, void* img, int* status, cudaStream_t s) {
    const int64_t Nt = cp.Nt;
    if (Nt == 0 || nvec == 0) return cudaSuccess;
    Schedule sc;
    cudaError_t e = make_schedule(Nt, kTcRows, kTcChunk, 2, &sc);
    if (e != cudaSuccess) return e;
    e = set_smem_attr(cp.kind);
    if (e != cudaSuccess) return e;
    unsigned char* im = static_cast<unsigned char*>(img);
    const int64_t nchunks = sc.len;
    const int img_blocks = int(nchunks < 152 * 8 ? nchunks : 152 * 8);
    for (int v0 = 0; v0 < nvec; v0 += kTcNB) {
        const int g = (nvec - v0) < kTcNB ? (nvec - v0) : kTcNB;
        tc_image_kernel<<<img_blocks, 128, 0, s>>>(cp.P32, cp.ldp, Nt, U + int64_t(v0) * ldu, ldu, g, im, nchunks);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const dim3 grid(unsigned(sc.G));
        switch (cp.kind) {
            case KL_K_EXP:
                covmv_tc_kernel<KL_K_EXP><<<grid, kTcThreads, kSmemBytes, s>>>(cp, im, g, part, sc.len, sc.T,
                                                                               sc.maxseg, status);
                break;
            case KL_K_GAUSS:
                covmv_tc_kernel<KL_K_GAUSS><<<grid, kTcThreads, kSmemBytes, s>>>(cp, im, g, part, sc.len, sc.T,
                                                                                 sc.maxseg, status);
                break;
            case KL_K_EXP_SEPARABLE:
                covmv_tc_kernel<KL_K_EXP_SEPARABLE><<<grid, kTcThreads, kSmemBytes, s>>>(cp, im, g, part, sc.len,
                                                                                         sc.T, sc.maxseg, status);
                break;
            default:
                covmv_tc_kernel<KL_K_POLY_TEST><<<grid, kTcThreads, kSmemBytes, s>>>(cp, im, g, part, sc.len, sc.T,
                                                                                     sc.maxseg, status);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t tot = Nt * g;
        int blocks = int((tot + 255) / 256);
        if (blocks > 152 * 8) blocks = 152 * 8;
        slot_reduce<kTcRows, kTcNB><<<blocks, 256, 0, s>>>(part, Nt, g, sc.len, sc.T, sc.G, sc.maxseg,
                                                           Z + int64_t(v0) * ldz, ldz,
                                         scale2, J);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        count_launches(3);
    }
    return cudaSuccess;
}

}  // namespace kl
