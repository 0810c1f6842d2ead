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

#include "kl_internal.h"

namespace kl {
namespace {

constexpr int kTcRows = 128;     // MMA M
constexpr int kTcN = 16;         // MMA N: vectors per launch group
constexpr int kTcK = 16;         // MMA K for 16-bit inputs
constexpr int kTcChunk = 32;     // columns per pipeline stage (2 MMA K-steps)
constexpr int kTcThreads = 128;
constexpr int kTcPieces = 3;     // bfloat16 terms per float32 value
constexpr int kTcTmemCols = 32;  // allocation granule (>= N)

// shared-memory layout (bytes), canonical K-major, no swizzle: core matrices of 8 rows x 16 bytes
constexpr int kASub = kTcRows * kTcK * 2;                 // one 128 x 16 bf16 sub-tile: 4 KB
constexpr int kAPiece = kASub * (kTcChunk / kTcK);        // one piece of a chunk: 8 KB
constexpr int kAStage = kAPiece * kTcPieces;              // 24 KB
constexpr int kBSub = kTcN * kTcK * 2;                    // 16 x 16 bf16: 512 B
constexpr int kBPiece = kBSub * (kTcChunk / kTcK);        // 1 KB
constexpr int kBStage = kBPiece * kTcPieces;              // 3 KB
constexpr int kOffA = 0;
constexpr int kOffB = 2 * kAStage;                        // 48 KB
constexpr int kOffC = kOffB + 2 * kBStage;                // column points: 2 stages x 32 float4
constexpr int kOffBar = kOffC + 2 * kTcChunk * 16;        // 2 mbarriers
constexpr int kOffTmem = kOffBar + 16;
constexpr int kSmemBytes = kOffTmem + 16;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row r, k) inside a K-major no-swizzle tile of 16-column sub-tiles
__device__ __forceinline__ int kmajor_offset(int r, int k, int sub_bytes) {
    const int t = k / kTcK, kk = k % kTcK;
    return t * sub_bytes + (r >> 3) * 256 + (kk >> 3) * 128 + (r & 7) * 16 + (kk & 7) * 2;
}

// tcgen05 shared-memory matrix descriptor: start address, leading (K-direction) and stride
// (M/N-direction) byte offsets between core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((saddr >> 4) & 0x3FFF);
    d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// instruction descriptor, kind::f16: D float32, A and B bfloat16, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kTcN >> 3) << 17) |
                            (uint32_t(kTcRows >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity; false on timeout (~2 s at 2 GHz)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 4000000000ll) return false;
    }
    return true;
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16* p) {
    const __nv_bfloat16 a = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(a);
    const __nv_bfloat16 b = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b);
    p[0] = a;
    p[1] = b;
    p[2] = __float2bfloat16_rn(r2);
}

template <int KIND>
__device__ __forceinline__ float kernel_tc(float dx, float dy, float dz, float x0, float y0, float z0, float x1,
                                           float y1, float z1, int pm) {
    if (KIND == KL_K_EXP) {
        float s = fmaxf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), 1e-30f);
        float rs, g;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(s));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(-s * rs));
        return g;
    } else if (KIND == KL_K_GAUSS) {
        float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx)), g;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(-s));
        return g;
    } else if (KIND == KL_K_EXP_SEPARABLE) {
        float g;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(-(fabsf(dx) + fabsf(dy) + fabsf(dz))));
        return g;
    } else {
        float f = fmaf(x0, x1, 1.f) * fmaf(y0, y1, 1.f) * fmaf(z0, z1, 1.f), r = 1.f;
        for (int i = 0; i < pm; ++i) r *= f;
        return r;
    }
}

template <int KIND>
__global__ void __launch_bounds__(kTcThreads)
covmv_tc_kernel(CovParams cp, const float* __restrict__ U, int64_t ldu, int nv, double* __restrict__ part,
                int64_t cols_per_split, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + kOffBar, bar1 = sbase + kOffBar + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffTmem);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const int64_t Nt = cp.Nt;
    const float* P = cp.P32;
    const int64_t row = int64_t(blockIdx.x) * kTcRows + tid;
    const bool rvalid = row < Nt;
    const float x0 = rvalid ? P[row] : 0.f, y0 = rvalid ? P[cp.ldp + row] : 0.f, z0 = rvalid ? P[2 * cp.ldp + row] : 0.f;

    const int64_t c_begin = int64_t(blockIdx.y) * cols_per_split;
    int64_t c_end = c_begin + cols_per_split;
    if (c_end > Nt) c_end = Nt;
    const int nchunks = int((c_end - c_begin + kTcChunk - 1) / kTcChunk);

    bool ok = true;
    for (int it = 0; it < nchunks; ++it) {
        const int s = it & 1;
        const uint32_t bar = s ? bar1 : bar0;
        if (it >= 2 && ok) ok = mbar_wait(bar, uint32_t(((it - 2) >> 1) & 1));
        const int64_t c0 = c_begin + int64_t(it) * kTcChunk;
        float4* cst = reinterpret_cast<float4*>(smem + kOffC) + s * kTcChunk;
        if (tid < kTcChunk) {
            const int64_t c = c0 + tid;
            cst[tid] = (c < c_end) ? make_float4(P[c], P[cp.ldp + c], P[2 * cp.ldp + c], 0.f)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // u chunk -> B pieces: thread t handles vector v = t / 8 and the 8-column group t % 8 ... but
        // the chunk has 32 columns = 4 groups of 8 for each of 16 vectors = 64 items for 128 threads
        unsigned char* Bst = smem + kOffB + s * kBStage;
        if (tid < kTcN * (kTcChunk / 8)) {
            const int v = tid / (kTcChunk / 8), g8 = tid % (kTcChunk / 8);
            __align__(16) __nv_bfloat16 pc[kTcPieces][8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t c = c0 + g8 * 8 + e;
                const float u = (v < nv && c < c_end) ? U[v * ldu + c] : 0.f;
                __nv_bfloat16 t3[3];
                split3(u, t3);
                pc[0][e] = t3[0];
                pc[1][e] = t3[1];
                pc[2][e] = t3[2];
            }
#pragma unroll
            for (int q = 0; q < kTcPieces; ++q)
                *reinterpret_cast<uint4*>(Bst + q * kBPiece + kmajor_offset(v, g8 * 8, kBSub)) =
                    *reinterpret_cast<const uint4*>(pc[q]);
        }
        __syncthreads();
        // kernel values of this thread's row for the 32 columns -> A pieces
        unsigned char* Ast = smem + kOffA + s * kAStage;
#pragma unroll 1
        for (int g8 = 0; g8 < kTcChunk / 8; ++g8) {
            __align__(16) __nv_bfloat16 pc[kTcPieces][8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float4 q = cst[g8 * 8 + e];
                const float g = kernel_tc<KIND>(x0 - q.x, y0 - q.y, z0 - q.z, x0, y0, z0, q.x, q.y, q.z, cp.poly_m);
                __nv_bfloat16 t3[3];
                split3(g, t3);
                pc[0][e] = t3[0];
                pc[1][e] = t3[1];
                pc[2][e] = t3[2];
            }
#pragma unroll
            for (int q = 0; q < kTcPieces; ++q)
                *reinterpret_cast<uint4*>(Ast + q * kAPiece + kmajor_offset(tid, g8 * 8, kASub)) =
                    *reinterpret_cast<const uint4*>(pc[q]);
        }
        // make the generic-proxy shared-memory writes visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a0 = sbase + kOffA + s * kAStage, b0 = sbase + kOffB + s * kBStage;
            // products of pieces (a, b) with a + b <= 2 (0-based): g1u1, g1u2, g2u1, g1u3, g2u2, g3u1
            const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
            for (int ks = 0; ks < kTcChunk / kTcK; ++ks) {
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint64_t ad = make_desc(a0 + pa[p] * kAPiece + ks * kASub, 128, 256);
                    const uint64_t bd = make_desc(b0 + pb[p] * kBPiece + ks * kBSub, 128, 256);
                    mma_bf16(tmem, ad, bd, (it > 0 || ks > 0 || p > 0) ? 1u : 0u);
                }
            }
            mma_commit(bar);
        }
    }
    // wait for the last chunk's MMAs (a commit covers every earlier MMA of the issuing thread)
    if (nchunks > 0) {
        const int last = nchunks - 1;
        const bool done = mbar_wait((last & 1) ? bar1 : bar0, uint32_t((last >> 1) & 1));
        ok = ok && done;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok) {
        if (lane == 0) atomicExch(status, int(KL_ERR_TIMEOUT));
    } else if (nchunks > 0) {
        uint32_t d[16];
        const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
            : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
              "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (rvalid) {
#pragma unroll
            for (int v = 0; v < kTcN; ++v)
                if (v < nv) part[(int64_t(blockIdx.y) * nv + v) * Nt + row] = double(__uint_as_float(d[v]));
        }
    } else if (rvalid) {
        for (int v = 0; v < nv; ++v) part[(int64_t(blockIdx.y) * nv + v) * Nt + row] = 0.0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
}

__global__ void tc_reduce(const double* __restrict__ part, int splits, int64_t Nt, int nv, double* __restrict__ Z,
                          int64_t ldz, double scale2, const double* __restrict__ J) {
    const int64_t total = Nt * nv;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t v = idx / Nt, r = idx - v * Nt;
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp) s += part[(int64_t(sp) * nv + v) * Nt + r];
        s *= scale2;
        if (J) s *= J[r];
        Z[v * ldz + r] = s;
    }
}

}  // namespace

int covmv_tc_splits(int64_t Nt) {
    const int64_t rowblocks = (Nt + kTcRows - 1) / kTcRows;
    int64_t splits = (152 * 3 * 2 + rowblocks - 1) / rowblocks;
    int64_t maxs = Nt / (8 * kTcChunk);
    if (maxs < 1) maxs = 1;
    if (splits > maxs) splits = maxs;
    if (splits > 64) splits = 64;
    if (splits < 1) splits = 1;
    return int(splits);
}

cudaError_t launch_covmv_tc(const CovParams& cp, const float* U, int64_t ldu, int nvec, double* Z, int64_t ldz,
                            double scale2, const double* J, double* part, int splits, int* status,
                            cudaStream_t s) {
    const int64_t Nt = cp.Nt;
    if (Nt == 0 || nvec == 0) return cudaSuccess;
    int64_t cps = (Nt + splits - 1) / splits;
    cps = (cps + kTcChunk - 1) / kTcChunk * kTcChunk;
    const int used = int((Nt + cps - 1) / cps);
    dim3 grid(unsigned((Nt + kTcRows - 1) / kTcRows), unsigned(used));
    static bool attr_done[4] = {false, false, false, false};
    for (int v0 = 0; v0 < nvec; v0 += kTcN) {
        const int g = (nvec - v0) < kTcN ? (nvec - v0) : kTcN;
        const float* Ug = U + int64_t(v0) * ldu;
        cudaError_t e = cudaSuccess;
#define KL_TC_CASE(K)                                                                                         \
    case K:                                                                                                   \
        if (!attr_done[K]) {                                                                                  \
            e = cudaFuncSetAttribute(covmv_tc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes); \
            if (e != cudaSuccess) return e;                                                                   \
            attr_done[K] = true;                                                                              \
        }                                                                                                     \
        covmv_tc_kernel<K><<<grid, kTcThreads, kSmemBytes, s>>>(cp, Ug, ldu, g, part, cps, status);           \
        break;
        switch (cp.kind) {
            KL_TC_CASE(KL_K_EXP)
            KL_TC_CASE(KL_K_GAUSS)
            KL_TC_CASE(KL_K_EXP_SEPARABLE)
            default:
                KL_TC_CASE(KL_K_POLY_TEST)
        }
#undef KL_TC_CASE
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        count_launches(2);
        int64_t tot = Nt * g;
        int blocks = int((tot + 255) / 256);
        if (blocks > 152 * 8) blocks = 152 * 8;
        tc_reduce<<<blocks, 256, 0, s>>>(part, used, Nt, g, Z + int64_t(v0) * ldz, ldz, scale2, J);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace kl
