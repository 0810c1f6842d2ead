// Learned warm start: a multilayer perceptron (bfloat16 weights and layer inputs, float32
// sums, tanh hidden layers, linear output) that maps problem parameters to the coefficients
// of k standard-form vectors on a coarse mesh, trained on eigenpairs the solver generates with
// a loss on orthogonal projectors, ||Y Y^T - V V^T||_F^2 / k (rotation and sign invariant):
//   loss = ||Y^T Y||_F^2 - 2 ||V^T Y||_F^2 + ||V^T V||_F^2,   dL/dY = 4 Y (Y^T Y) - 4 V (V^T Y).
//
// The three products of a training step run on the tensor cores (tcgen05, bfloat16 operands,
// float32 accumulators in tensor memory), each written as C[m][n] = sum_k A[m][k] B[n][k] with
// both operands K-contiguous, so that the large dimension (the output width) is the M side:
//   forward   Z^T = W^T H^T        A = W^T (dout x din), B = H (batch x din)
//   dW        dW^T = dZ^T H        A = dZ^T (dout x batch), B = H^T (din x batch)
//   dH        dH^T = W dZ^T        A = W (din x dout), B = dZ (batch x dout), split over dout
// Operands are staged by cp.async (16 bytes per thread) straight into the canonical no-swizzle
// K-major layout, four stages deep; one thread issues the MMAs; four warps read the
// accumulators back and store C transposed (coalesced along m).  Shapes the tensor-core kernel
// cannot take (an inner dimension that is not a multiple of 8, e.g. the 4 network inputs) go
// through a tiled float32-FMA GEMM.  The loss Gram matrices are split over row chunks and
// reduced in a fixed order; Adam (Kingma and Ba 2015, Algorithm 1) keeps float32 master
// weights and refreshes both bfloat16 copies (W and W^T) in one tiled pass per layer.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kl_internal.h"
#include "tc_common.cuh"

struct kl_mlp_s {
    int n_in = 0, width = 0, depth = 0, n_out = 0;
    int layers = 0;
    std::vector<int> din, dout;                 // per layer
    std::vector<size_t> woff, boff;             // offsets into the flat parameter array
    std::vector<size_t> wtoff;                  // offsets of W^T (dout x din) in Wt, multiples of 8
    size_t nparam = 0, nwt = 0;
    float* P = nullptr;                         // float32 master parameters (weights then biases per layer)
    float* G = nullptr;                         // gradients
    float* M = nullptr;                         // Adam first moments
    float* V = nullptr;                         // Adam second moments
    __nv_bfloat16* Wb = nullptr;                // bfloat16 copy of the parameters (parameter layout)
    __nv_bfloat16* Wt = nullptr;                // bfloat16 W^T per layer
    int t = 0;                                  // Adam step
    int cap = 0;                                // batch the activation buffers hold
    std::vector<size_t> aoff;                   // per level 0..layers: offset of [batch][d] activations
    kl::DevBuf hf, hb, ht, dzf, dzb, dzt, dh, part, gpart, gram, status;
};

namespace kl {
namespace {

using bf16 = __nv_bfloat16;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------------------
// tensor-core GEMM: C[m][n] = sum_{k in split z} A[m*lda + k] B[n*ldb + k]
// ---------------------------------------------------------------------------------------
constexpr int kTcM = 128, kTcK = 64, kTcMaxStages = 4, kTcThreads = 160;
constexpr int kTcAStage = kTcM * kTcK * 2;                    // 16 KB
constexpr int kTcMaxSmem = kTcMaxStages * (kTcAStage + 256 * kTcK * 2) + 256;
constexpr int kSmemPerSm = 233472;                            // 228 KB, of which 1 KB per CTA is reserved

struct TcArgs {
    int M, N, K;
    const bf16* A;
    int64_t lda;
    const bf16* B;
    int64_t ldb;
    int NT;               // N tile (multiple of 16, at most 256)
    int tmem_cols;        // power of two >= max(32, NT)
    int kchunk;           // K range per split (multiple of kTcK)
    int stages;           // 1..4 shared-memory stages of kTcK columns
    const float* bias;    // per m (forward), or null
    int act;              // 1: tanh
    float* out;           // out[(z * N + n) * ldo + m]
    bf16* outb;           // optional bfloat16 copy (same indexing)
    int64_t ldo;
    int* status;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

// wait until at most n of this thread's cp.async groups are pending (n = 0..3)
__device__ __forceinline__ void cp_async_wait(int n) {
    switch (n) {
        case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    }
}

// one stage of rows [r0, r0 + rows) x K columns [kb, kb + 64) of a K-contiguous operand into the
// no-swizzle K-major layout (16-column sub-tiles of rows * 32 bytes); rows beyond `valid_rows`
// and columns beyond k1 are zero-filled
__device__ __forceinline__ void stage_rows(uint32_t dst, const bf16* __restrict__ X, int64_t ld, int r0, int rows,
                                           int valid_rows, int kb, int k1, int tid) {
    const int sub = rows * 32;
    for (int c = tid; c < rows * 8; c += 128) {
        const int r = c >> 3, kc = c & 7;
        const int k = kb + kc * 8;
        const int row = r0 + r;
        const bool v = (row < valid_rows) && (k < k1);
        const bf16* src = v ? X + int64_t(row) * ld + k : X;
        cp_async16(dst + (kc >> 1) * sub + (r >> 3) * 256 + (kc & 1) * 128 + (r & 7) * 16, src, v ? 16u : 0u);
    }
}

__global__ void __launch_bounds__(kTcThreads) tc_gemm_kernel(TcArgs a) {
    using namespace kl::tc;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NT = a.NT, S = a.stages, lag = a.stages - 1;
    const int stage_bytes = kTcAStage + NT * kTcK * 2;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + S * stage_bytes;              // full[4], empty[4], done
    const uint32_t bar_full = bar0, bar_empty = bar0 + 8 * kTcMaxStages, bar_done = bar0 + 16 * kTcMaxStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S * stage_bytes + 16 * kTcMaxStages + 8);
    int* s_fail = reinterpret_cast<int*>(smem + S * stage_bytes + 16 * kTcMaxStages + 16);

    const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * NT, z = blockIdx.z;
    const int k0 = z * a.kchunk;
    const int k1 = min(a.K, k0 + a.kchunk);
    const int nk = (k1 - k0 + kTcK - 1) / kTcK;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(bar_full + 8 * s, 128);
            mbar_init(bar_empty + 8 * s, 1);
        }
        mbar_init(bar_done, 1);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 4) tmem_alloc(smem_u32(tmem_slot), uint32_t(a.tmem_cols));
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        // ---------------- producers, then epilogue ----------------
        bool ok = true;
        int arrived = 0;
        for (int i = 0; i < nk; ++i) {
            const int st = i % S;
            if (i >= S) {
                ok = __all_sync(0xffffffffu, mbar_wait(bar_empty + 8 * st, uint32_t(((i / S) - 1) & 1)));
                if (!ok) break;
            }
            const int kb = k0 + i * kTcK;
            const uint32_t sa = sbase + st * stage_bytes;
            stage_rows(sa, a.A, a.lda, m0, kTcM, a.M, kb, k1, tid);
            stage_rows(sa + kTcAStage, a.B, a.ldb, n0, NT, a.N, kb, k1, tid);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            if (i >= lag) {
                cp_async_wait(lag);
                fence_proxy_async();
                mbar_arrive(bar_full + 8 * ((i - lag) % S));
                arrived = i - lag + 1;
            }
        }
        // every copy of this thread has landed before the CTA can leave
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        fence_proxy_async();
        if (ok) {
            for (int j = arrived; j < nk; ++j) mbar_arrive(bar_full + 8 * (j % S));
            ok = __all_sync(0xffffffffu, mbar_wait(bar_done, 0));
        }
        if (ok) {
            fence_after_sync();
            const int m = m0 + warp * 32 + lane;
            for (int c0 = 0; c0 < NT; c0 += 16) {
                uint32_t d[16];
                const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];\n"
                    : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
                      "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]),
                      "=r"(d[15])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (m < a.M) {
                    const float bm = a.bias ? a.bias[m] : 0.f;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = n0 + c0 + j;
                        if (n < a.N) {
                            float v = __uint_as_float(d[j]) + bm;
                            if (a.act) v = tanhf(v);
                            const int64_t o = (int64_t(z) * a.N + n) * a.ldo + m;
                            a.out[o] = v;
                            if (a.outb) a.outb[o] = __float2bfloat16_rn(v);
                        }
                    }
                }
            }
        }
        if (!ok) atomicExch(s_fail, 1);
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = idesc_bf16(kTcM, NT);
        bool ok = true;
        for (int i = 0; i < nk; ++i) {
            const int st = i % S;
            ok = mbar_wait(bar_full + 8 * st, uint32_t((i / S) & 1));
            if (!ok) break;
            fence_after_sync();
            const uint32_t sa = sbase + st * stage_bytes, sb = sa + kTcAStage;
#pragma unroll
            for (int t = 0; t < kTcK / 16; ++t) {
                const uint64_t ad = make_desc(sa + t * (kTcM * 32), 128, 256);
                const uint64_t bd = make_desc(sb + t * (NT * 32), 128, 256);
                mma_bf16(tmem, ad, bd, idesc, (i > 0 || t > 0) ? 1u : 0u);
            }
            mma_commit(bar_empty + 8 * st);
        }
        // arrives once every MMA issued above has completed
        mma_commit(bar_done);
        if (!ok) atomicExch(s_fail, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 4) {
        // the accumulators may be released only after the MMAs have finished
        if (lane == 0 && *s_fail) mbar_wait(bar_done, 0);
        __syncwarp();
        fence_after_sync();
        tmem_dealloc(tmem, uint32_t(a.tmem_cols));
    }
    if (tid == 0 && *s_fail) atomicExch(a.status, int(KL_ERR_TIMEOUT));
}

bool tc_shape_ok(int K, const void* A, int64_t lda, const void* B, int64_t ldb) {
    return K > 0 && K % 8 == 0 && lda % 8 == 0 && ldb % 8 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(B) & 15) == 0;
}

// launches the tensor-core GEMM over `splits` K ranges of kchunk (a multiple of 64); split z
// writes to out + z * N * ldo
kl_status tc_gemm(int M, int N, int K, const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int kchunk,
                  const float* bias, int act, float* out, bf16* outb, int64_t ldo, int* status, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        KL_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcMaxSmem));
        attr = true;
    }
    if (M < 1 || N < 1 || K < 1 || kchunk < kTcK || kchunk % kTcK != 0)
        return fail(KL_ERR_INVALID_ARG, "tensor-core GEMM: bad shape");
    TcArgs a;
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = A;
    a.lda = lda;
    a.B = B;
    a.ldb = ldb;
    a.NT = int(std::min<size_t>(256, round_up(size_t(N), 16)));
    a.tmem_cols = 32;
    while (a.tmem_cols < a.NT) a.tmem_cols *= 2;
    a.kchunk = kchunk;
    a.bias = bias;
    a.act = act;
    a.out = out;
    a.outb = outb;
    a.ldo = ldo;
    a.status = status;
    const int splits = (K + kchunk - 1) / kchunk;
    // short contractions (<= 4 K blocks per CTA) are latency-bound: two stages and more CTAs per
    // SM; long ones get four stages.  Shared memory is padded so that the resident CTAs never ask
    // for more than the 512 tensor-memory columns of an SM.
    const int nk = kchunk / kTcK;
    a.stages = nk > 4 ? kTcMaxStages : std::min(nk, 2);
    size_t smem = size_t(a.stages) * (kTcAStage + size_t(a.NT) * kTcK * 2) + 256;
    const size_t occ_tmem = size_t(512 / a.tmem_cols);
    const size_t min_smem = (kSmemPerSm + occ_tmem) / (occ_tmem + 1) - 1024 + 16;
    if (smem < min_smem) smem = min_smem;
    dim3 grid((M + kTcM - 1) / kTcM, (N + a.NT - 1) / a.NT, splits);
    tc_gemm_kernel<<<grid, kTcThreads, smem, s>>>(a);
    KL_CUDA(cudaGetLastError());
    count_launches(1);
    return KL_OK;
}

// K range per split for a contraction of length K producing `tiles` output tiles: about two
// CTAs per SM, at least two K blocks per split
int tc_kchunk(int tiles, int K) {
    const int want = num_sms() * 2;
    int sp = 1;
    if (tiles < want && K > 4 * kTcK) {
        sp = (want + tiles - 1) / tiles;
        sp = std::min(sp, (K + 2 * kTcK - 1) / (2 * kTcK));
        sp = std::max(sp, 1);
    }
    return int(round_up(size_t((K + sp - 1) / sp), kTcK));
}

// ---------------------------------------------------------------------------------------
// float32-FMA GEMM for shapes the tensor-core kernel does not take
// ---------------------------------------------------------------------------------------
constexpr int kBM = 64, kBN = 64, kBK = 16, kGemmThreads = 256;

// C[m][n] (+)= sum_k A(m,k) B(k,n) over k in [k0, k1); A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn].
// Output of split z to out + z * M * N (row-major, float32).
__global__ void __launch_bounds__(kGemmThreads)
gemm_bf16_kernel(int M, int N, int K, const bf16* __restrict__ A, int64_t sam, int64_t sak,
                 const bf16* __restrict__ B, int64_t sbk, int64_t sbn, float* __restrict__ out, int kchunk) {
    __shared__ float sA[kBK][kBM + 1];
    __shared__ float sB[kBK][kBN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int k0 = blockIdx.z * kchunk;
    int k1 = k0 + kchunk;
    if (k1 > K) k1 = K;
    float acc[4][4] = {{0.f}};
    for (int kb = k0; kb < k1; kb += kBK) {
        for (int e = threadIdx.x; e < kBK * kBM; e += kGemmThreads) {
            const int kk = e / kBM, mm = e - kk * kBM;
            const int m = m0 + mm, k = kb + kk;
            sA[kk][mm] = (m < M && k < k1) ? __bfloat162float(A[int64_t(m) * sam + int64_t(k) * sak]) : 0.f;
        }
        for (int e = threadIdx.x; e < kBK * kBN; e += kGemmThreads) {
            const int kk = e / kBN, nn = e - kk * kBN;
            const int n = n0 + nn, k = kb + kk;
            sB[kk][nn] = (n < N && k < k1) ? __bfloat162float(B[int64_t(k) * sbk + int64_t(n) * sbn]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = sA[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = sB[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* o = out + size_t(blockIdx.z) * size_t(M) * size_t(N);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n < N) o[size_t(m) * N + n] = acc[i][j];
        }
    }
}

// out[m][n] = act(sum_z part[z][m][n] + bias[n]) (fixed split order); optional bfloat16 copy
__global__ void gemm_epilogue(const float* __restrict__ part, int splits, int M, int N, const float* __restrict__ bias,
                              int tanh_act, float* __restrict__ out, bf16* __restrict__ outb) {
    const size_t total = size_t(M) * N;
    for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[size_t(z) * total + idx];
        if (bias) s += bias[idx % N];
        if (tanh_act) s = tanhf(s);
        if (out) out[idx] = s;
        if (outb) outb[idx] = __float2bfloat16_rn(s);
    }
}

// dz[b][j] = (sum_z part[z][b][j]) * (1 - h[b][j]^2) (fixed split order); bfloat16 copy
__global__ void split_tanh_backward(const float* __restrict__ part, int splits, size_t total,
                                    const float* __restrict__ h, float* __restrict__ dz, bf16* __restrict__ dzb) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[size_t(z) * total + i];
        const float v = s * (1.f - h[i] * h[i]);
        dz[i] = v;
        dzb[i] = __float2bfloat16_rn(v);
    }
}

__global__ void to_bf16(const float* __restrict__ x, size_t n, bf16* __restrict__ y) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// dst[c][r] = src[r][c] for r < rows, 0 for rows <= r < ldd (32 x 32 tiles through shared memory)
__global__ void transpose_bf16(const bf16* __restrict__ src, int rows, int cols, int64_t lds, bf16* __restrict__ dst,
                               int64_t ldd) {
    __shared__ bf16 tile[32][34];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src[int64_t(r) * lds + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < ldd) dst[int64_t(c) * ldd + r] = tile[threadIdx.x][i];
    }
}

// db[n] = sum over rows m of dz[m][n] (fixed order)
__global__ void column_sums(const float* __restrict__ dz, int M, int N, float* __restrict__ db) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int m = 0; m < M; ++m) s += dz[size_t(m) * N + n];
        db[n] = s;
    }
}

// ---------------------------------------------------------------------------------------
// projector loss
// ---------------------------------------------------------------------------------------
// Gram matrix of X = [Y V] (the k predicted and the k target vectors of one sample, n rows):
// C = X^T X (2k x 2k, rows padded to R with zeros), of which Y^T Y, V^T Y and V^T V are used.
// CTA (c, s) accumulates row chunks c, c + gridDim.x, ... of sample s: each chunk of ch rows is
// staged in shared memory (X^T rows of ch + 4 floats) and every thread keeps an (R/16) x (R/16)
// tile C[tr + 16 i][tc + 16 j] in registers, reading four rows at a time as float4.
// Partial sums to gp[(s * gridDim.x + c) * R * R].
template <int R>
__global__ void __launch_bounds__(256) loss_gram_partial(const float* __restrict__ out, const float* __restrict__ tgt,
                                                         int n, int k, int ch, float* __restrict__ gp) {
    constexpr int T = R / 16;
    extern __shared__ __align__(16) float xs[];          // R rows of ld floats
    const int s = blockIdx.y, ld = ch + 4;
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
    const float* Y = out + size_t(s) * k * n;
    const float* V = tgt + size_t(s) * k * n;
    float acc[T][T];
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) acc[i][j] = 0.f;
    const int nch = (n + ch - 1) / ch;
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int i0 = c * ch;
        __syncthreads();
        for (int e = threadIdx.x; e < R * ch; e += blockDim.x) {
            const int a = e / ch, ii = e - a * ch;
            const int i = i0 + ii;
            float v = 0.f;
            if (i < n) {
                if (a < k)
                    v = Y[size_t(a) * n + i];
                else if (a < 2 * k)
                    v = V[size_t(a - k) * n + i];
            }
            xs[a * ld + ii] = v;
        }
        __syncthreads();
        for (int ii = 0; ii < ch; ii += 4) {
            float4 ra[T], rb[T];
#pragma unroll
            for (int i = 0; i < T; ++i) ra[i] = *reinterpret_cast<const float4*>(xs + (tr + 16 * i) * ld + ii);
#pragma unroll
            for (int j = 0; j < T; ++j) rb[j] = *reinterpret_cast<const float4*>(xs + (tc + 16 * j) * ld + ii);
#pragma unroll
            for (int i = 0; i < T; ++i)
#pragma unroll
                for (int j = 0; j < T; ++j) {
                    acc[i][j] = fmaf(ra[i].x, rb[j].x, acc[i][j]);
                    acc[i][j] = fmaf(ra[i].y, rb[j].y, acc[i][j]);
                    acc[i][j] = fmaf(ra[i].z, rb[j].z, acc[i][j]);
                    acc[i][j] = fmaf(ra[i].w, rb[j].w, acc[i][j]);
                }
        }
    }
    float* g = gp + (size_t(s) * gridDim.x + blockIdx.x) * R * R;
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) g[(tr + 16 * i) * R + tc + 16 * j] = acc[i][j];
}

// per sample (one CTA of 256 threads): partial Grams summed in order; gram[s] = (Y^T Y, V^T Y);
// loss[s] = (||Y^T Y||^2 - 2 ||V^T Y||^2 + ||V^T V||^2) / k (fixed-order tree)
__global__ void loss_gram_reduce(const float* __restrict__ gp, int parts, int R, int k, float* __restrict__ gram,
                                 float* __restrict__ loss) {
    __shared__ float red[256];
    const int s = blockIdx.x, kk = k * k;
    float l = 0.f;
    for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
        const int w = e / kk, ab = e - w * kk, a = ab / k, b = ab - a * k;
        // w = 0: Y^T Y = C[a][b]; w = 1: V^T Y = C[k + a][b]; w = 2: V^T V = C[k + a][k + b]
        const int row = (w == 0 ? a : k + a), col = (w == 2 ? k + b : b);
        float acc = 0.f;
        for (int c = 0; c < parts; ++c) acc += gp[(size_t(s) * parts + c) * R * R + row * R + col];
        if (w < 2) gram[size_t(s) * 2 * kk + e] = acc;
        l += (w == 1 ? -2.f : 1.f) * acc * acc;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[s] = red[0] / float(k);
}

// dY[s][b*n + i] = scale * (4 sum_a Y[i][a] YtY[a][b] - 4 sum_a V[i][a] VtY[a][b]);
// thread = row i, block.y = sample; the two k x k matrices of the sample in shared memory
// (rows of KMAX floats, read as broadcast float4)
template <int KMAX>
__global__ void __launch_bounds__(256) loss_grad(const float* __restrict__ out, const float* __restrict__ tgt,
                                                 const float* __restrict__ gram, int n, int k, float scale,
                                                 float* __restrict__ dy, bf16* __restrict__ dyb) {
    __shared__ __align__(16) float g1[KMAX * KMAX], g2[KMAX * KMAX];
    const int s = blockIdx.y, kk = k * k;
    const float* YtY = gram + size_t(s) * 2 * kk;
    for (int e = threadIdx.x; e < KMAX * KMAX; e += blockDim.x) {
        const int a = e / KMAX, b = e - a * KMAX;
        const bool v = a < k && b < k;
        g1[e] = v ? YtY[a * k + b] : 0.f;
        g2[e] = v ? -YtY[kk + a * k + b] : 0.f;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* Y = out + size_t(s) * k * n + i;
    const float* V = tgt + size_t(s) * k * n + i;
    float acc[KMAX];
#pragma unroll
    for (int b = 0; b < KMAX; ++b) acc[b] = 0.f;
    for (int a = 0; a < k; ++a) {
        const float ya = Y[size_t(a) * n], va = V[size_t(a) * n];
#pragma unroll
        for (int b = 0; b < KMAX; b += 4) {
            const float4 p = *reinterpret_cast<const float4*>(g1 + a * KMAX + b);
            const float4 q = *reinterpret_cast<const float4*>(g2 + a * KMAX + b);
            acc[b] = fmaf(ya, p.x, fmaf(va, q.x, acc[b]));
            acc[b + 1] = fmaf(ya, p.y, fmaf(va, q.y, acc[b + 1]));
            acc[b + 2] = fmaf(ya, p.z, fmaf(va, q.z, acc[b + 2]));
            acc[b + 3] = fmaf(ya, p.w, fmaf(va, q.w, acc[b + 3]));
        }
    }
    float* d = dy + size_t(s) * k * n + i;
    bf16* db = dyb + size_t(s) * k * n + i;
#pragma unroll
    for (int b = 0; b < KMAX; ++b)
        if (b < k) {
            const float g = 4.f * scale * acc[b];
            d[size_t(b) * n] = g;
            db[size_t(b) * n] = __float2bfloat16_rn(g);
        }
}

// ---------------------------------------------------------------------------------------
// Adam and the bfloat16 copies
// ---------------------------------------------------------------------------------------
// one layer's (din + 1) x dout block of the flat parameters (the bias is row din); update = 0
// only refreshes Wb and Wt from P.  32 x 32 tiles, W^T written through shared memory.
__global__ void adam_layer(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ Mo,
                           float* __restrict__ Vo, bf16* __restrict__ Wb, bf16* __restrict__ Wt, size_t woff, int din,
                           int dout, int update, float lr, float b1, float b2, float eps, float c1, float c2) {
    __shared__ bf16 tile[32][34];
    const int o0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int j = j0 + r, o = o0 + threadIdx.x;
        if (j <= din && o < dout) {
            const size_t idx = woff + size_t(j) * dout + o;
            float p = P[idx];
            if (update) {
                const float gi = G[idx];
                const float mi = b1 * Mo[idx] + (1.f - b1) * gi;
                const float vi = b2 * Vo[idx] + (1.f - b2) * gi * gi;
                Mo[idx] = mi;
                Vo[idx] = vi;
                p = p - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
                P[idx] = p;
            }
            const bf16 pb = __float2bfloat16_rn(p);
            Wb[idx] = pb;
            tile[r][threadIdx.x] = pb;
        }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int o = o0 + r, j = j0 + threadIdx.x;
        if (o < dout && j < din) Wt[size_t(o) * din + j] = tile[threadIdx.x][r];
    }
}

// The same update on 32 x 128 tiles, four consecutive outputs a thread (float4 loads and stores
// of P, G, M, V, four bfloat16 of Wb in one 8-byte store), for layers whose dout and offset are
// multiples of 4; W^T leaves shared memory two bfloat16 at a time.  Per element the same float
// operations as adam_layer.
__device__ __forceinline__ float adam_one(float& p, float g, float& m, float& v, float lr, float b1, float b2,
                                          float eps, float c1, float c2) {
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    p = p - lr * (m / c1) / (sqrtf(v / c2) + eps);
    return p;
}

__global__ void adam_layer4(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ Mo,
                            float* __restrict__ Vo, bf16* __restrict__ Wb, bf16* __restrict__ Wt, size_t woff, int din,
                            int dout, int update, float lr, float b1, float b2, float eps, float c1, float c2) {
    __shared__ bf16 tile[32][136];
    const int o0 = blockIdx.x * 128, j0 = blockIdx.y * 32;
    const int o = o0 + 4 * threadIdx.x;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int j = j0 + r;
        if (j <= din && o < dout) {
            const size_t idx = woff + size_t(j) * dout + o;
            float4 p = *reinterpret_cast<const float4*>(P + idx);
            if (update) {
                const float4 g = *reinterpret_cast<const float4*>(G + idx);
                float4 m = *reinterpret_cast<const float4*>(Mo + idx);
                float4 v = *reinterpret_cast<const float4*>(Vo + idx);
                adam_one(p.x, g.x, m.x, v.x, lr, b1, b2, eps, c1, c2);
                adam_one(p.y, g.y, m.y, v.y, lr, b1, b2, eps, c1, c2);
                adam_one(p.z, g.z, m.z, v.z, lr, b1, b2, eps, c1, c2);
                adam_one(p.w, g.w, m.w, v.w, lr, b1, b2, eps, c1, c2);
                *reinterpret_cast<float4*>(Mo + idx) = m;
                *reinterpret_cast<float4*>(Vo + idx) = v;
                *reinterpret_cast<float4*>(P + idx) = p;
            }
            const bf16 q0 = __float2bfloat16_rn(p.x), q1 = __float2bfloat16_rn(p.y);
            const bf16 q2 = __float2bfloat16_rn(p.z), q3 = __float2bfloat16_rn(p.w);
            __nv_bfloat162 lo, hi;
            lo.x = q0;
            lo.y = q1;
            hi.x = q2;
            hi.y = q3;
            uint2 pk;
            pk.x = *reinterpret_cast<const unsigned*>(&lo);
            pk.y = *reinterpret_cast<const unsigned*>(&hi);
            *reinterpret_cast<uint2*>(Wb + idx) = pk;
            tile[r][4 * threadIdx.x] = q0;
            tile[r][4 * threadIdx.x + 1] = q1;
            tile[r][4 * threadIdx.x + 2] = q2;
            tile[r][4 * threadIdx.x + 3] = q3;
        }
    }
    __syncthreads();
    // W^T rows o (din entries each): 16 threads write 32 j of one row, two at a time
    const int t = threadIdx.y * 32 + threadIdx.x;
    const int jj = 2 * (t & 15);
    for (int oo = t >> 4; oo < 128; oo += 16) {
        const int oc = o0 + oo, j = j0 + jj;
        if (oc >= dout || j >= din) continue;
        if (j + 1 < din) {
            __nv_bfloat162 w2;
            w2.x = tile[jj][oo];
            w2.y = tile[jj + 1][oo];
            if (((size_t(oc) * din + j) & 1) == 0) {
                *reinterpret_cast<__nv_bfloat162*>(Wt + size_t(oc) * din + j) = w2;
                continue;
            }
            Wt[size_t(oc) * din + j + 1] = tile[jj + 1][oo];
        }
        Wt[size_t(oc) * din + j] = tile[jj][oo];
    }
}

// grow a work buffer only after the stream's earlier work (which may read it) has finished
kl_status grow(DevBuf& b, size_t bytes, cudaStream_t s) {
    if (b.bytes >= bytes) return KL_OK;
    KL_CUDA(cudaStreamSynchronize(s));
    return ensure(b, bytes);
}

// rows idx[j] of src (rows of `width` floats) into dst row j
__global__ void gather_rows(const float* __restrict__ src, const int* __restrict__ idx, int rows, int64_t width,
                            float* __restrict__ dst) {
    const size_t total = size_t(rows) * size_t(width);
    for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < total; e += size_t(gridDim.x) * blockDim.x) {
        const size_t r = e / size_t(width), c = e - r * size_t(width);
        dst[e] = src[size_t(idx[r]) * size_t(width) + c];
    }
}

int blocks_for(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > size_t(num_sms()) * 8) b = size_t(num_sms()) * 8;
    return int(b < 1 ? 1 : b);
}

// float32-FMA product out (+ bias, act) = A x B with the strides described at gemm_bf16_kernel
kl_status gemm(kl_mlp m, int M, int N, int K, const bf16* A, int64_t sam, int64_t sak, const bf16* B, int64_t sbk,
               int64_t sbn, const float* bias, int act, float* out, bf16* outb, cudaStream_t s) {
    const int tiles = ((M + kBM - 1) / kBM) * ((N + kBN - 1) / kBN);
    int splits = 1;
    const int want = num_sms() * 4;
    if (tiles < want && K > 512) {
        splits = (want + tiles - 1) / tiles;
        const int maxs = (K + 255) / 256;
        if (splits > maxs) splits = maxs;
        if (splits > 64) splits = 64;
    }
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + kBK - 1) / kBK * kBK;
    splits = (K + kchunk - 1) / kchunk;
    if (splits < 1) splits = 1;
    KL_TRY(grow(m->part, size_t(splits) * M * N * sizeof(float), s));
    float* part = static_cast<float*>(m->part.ptr);
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, splits);
    gemm_bf16_kernel<<<grid, kGemmThreads, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, part, kchunk);
    KL_CUDA(cudaGetLastError());
    gemm_epilogue<<<blocks_for(size_t(M) * N), 256, 0, s>>>(part, splits, M, N, bias, act, out, outb);
    KL_CUDA(cudaGetLastError());
    count_launches(2);
    return KL_OK;
}

int level_dim(kl_mlp m, int l) { return l == 0 ? m->n_in : m->dout[size_t(l) - 1]; }

// activation buffers for `batch` rows: per level l, [batch][d_l] float32 and bfloat16
kl_status ensure_acts(kl_mlp m, int batch, cudaStream_t s) {
    if (batch <= m->cap) return KL_OK;
    KL_CUDA(cudaStreamSynchronize(s));
    m->aoff.assign(size_t(m->layers) + 2, 0);
    size_t o = 0, dmax = 0;
    for (int l = 0; l <= m->layers; ++l) {
        m->aoff[size_t(l)] = o;
        o += round_up(size_t(batch) * level_dim(m, l), 64);
        dmax = std::max(dmax, size_t(level_dim(m, l)));
    }
    m->aoff[size_t(m->layers) + 1] = o;
    const size_t ldb = round_up(size_t(batch), 8);
    KL_TRY(ensure(m->hf, o * sizeof(float)));
    KL_TRY(ensure(m->hb, o * sizeof(bf16)));
    KL_TRY(ensure(m->ht, dmax * ldb * sizeof(bf16)));
    KL_TRY(ensure(m->dzf, size_t(batch) * dmax * sizeof(float)));
    KL_TRY(ensure(m->dzb, size_t(batch) * dmax * sizeof(bf16)));
    KL_TRY(ensure(m->dzt, dmax * ldb * sizeof(bf16)));
    KL_TRY(ensure(m->dh, size_t(batch) * dmax * sizeof(float)));
    m->cap = batch;
    return KL_OK;
}

int* status_ptr(kl_mlp m) { return static_cast<int*>(m->status.ptr); }

kl_status check_status(kl_mlp m, cudaStream_t s) {
    int h = 0;
    KL_CUDA(cudaMemcpyAsync(&h, m->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    KL_CUDA(cudaStreamSynchronize(s));
    if (h != 0) {
        cudaMemsetAsync(m->status.ptr, 0, sizeof(int), s);
        return fail(KL_ERR_TIMEOUT, "warm-start network: a tensor-core wait gave up");
    }
    return KL_OK;
}

// forward for `batch` rows of x (float32, batch x n_in); activations kept for backward
kl_status forward_impl(kl_mlp m, const float* x, int batch, cudaStream_t s) {
    KL_TRY(ensure_acts(m, batch, s));
    float* hf = static_cast<float*>(m->hf.ptr);
    bf16* hb = static_cast<bf16*>(m->hb.ptr);
    KL_CUDA(cudaMemcpyAsync(hf, x, size_t(batch) * m->n_in * sizeof(float), cudaMemcpyDeviceToDevice, s));
    to_bf16<<<blocks_for(size_t(batch) * m->n_in), 256, 0, s>>>(hf, size_t(batch) * m->n_in, hb);
    KL_CUDA(cudaGetLastError());
    count_launches(1);
    for (int l = 0; l < m->layers; ++l) {
        const int di = m->din[size_t(l)], dout = m->dout[size_t(l)];
        const bool last = (l == m->layers - 1);
        const bf16* in = hb + m->aoff[size_t(l)];
        float* of = hf + m->aoff[size_t(l) + 1];
        bf16* ob = last ? nullptr : hb + m->aoff[size_t(l) + 1];
        const bf16* wt = m->Wt + m->wtoff[size_t(l)];
        if (tc_shape_ok(di, wt, di, in, di)) {
            // Z^T = W^T H^T: m = output feature, n = sample; stored as Z[n][m]
            KL_TRY(tc_gemm(dout, batch, di, wt, di, in, di, int(round_up(size_t(di), kTcK)), m->P + m->boff[size_t(l)],
                           last ? 0 : 1, of, ob, dout, status_ptr(m), s));
        } else {
            KL_TRY(gemm(m, batch, dout, di, in, di, 1, m->Wb + m->woff[size_t(l)], dout, 1, m->P + m->boff[size_t(l)],
                        last ? 0 : 1, of, ob, s));
        }
    }
    return KL_OK;
}

// loss of the current outputs against targets (float32, batch x k*n) and backward pass into m->G
kl_status backward_impl(kl_mlp m, const float* tgt, int batch, int k, int n, float* loss_dev, cudaStream_t s) {
    if (k > 64) return fail(KL_ERR_INVALID_ARG, "warm-start loss: at most 64 vectors per sample");
    if (batch > 65535) return fail(KL_ERR_INVALID_ARG, "warm-start loss: at most 65535 samples per batch");
    float* hf = static_cast<float*>(m->hf.ptr);
    bf16* hb = static_cast<bf16*>(m->hb.ptr);
    const float* out = hf + m->aoff[size_t(m->layers)];
    float* dzf = static_cast<float*>(m->dzf.ptr);
    bf16* dzb = static_cast<bf16*>(m->dzb.ptr);
    bf16* dzt = static_cast<bf16*>(m->dzt.ptr);
    bf16* ht = static_cast<bf16*>(m->ht.ptr);
    const int ldb = int(round_up(size_t(batch), 8));

    // Gram matrices of [Y V] in row chunks (shared memory: R rows of ch + 4 floats), at most 8
    // chunk groups per sample, reduced in order
    const int R = (2 * k <= 32) ? 32 : (2 * k <= 64 ? 64 : 128);
    const int ch = (R == 128) ? 88 : 160;
    const int parts = std::min(8, (n + ch - 1) / ch);
    KL_TRY(grow(m->gpart, size_t(batch) * parts * R * R * sizeof(float), s));
    KL_TRY(grow(m->gram, size_t(batch) * 2 * k * k * sizeof(float), s));
    float* gp = static_cast<float*>(m->gpart.ptr);
    float* gram = static_cast<float*>(m->gram.ptr);
    const size_t gsm = size_t(R) * (ch + 4) * sizeof(float);
    const dim3 gg(parts, batch);
    if (R == 32)
        loss_gram_partial<32><<<gg, 256, gsm, s>>>(out, tgt, n, k, ch, gp);
    else if (R == 64)
        loss_gram_partial<64><<<gg, 256, gsm, s>>>(out, tgt, n, k, ch, gp);
    else
        loss_gram_partial<128><<<gg, 256, gsm, s>>>(out, tgt, n, k, ch, gp);
    KL_CUDA(cudaGetLastError());
    loss_gram_reduce<<<batch, 256, 0, s>>>(gp, parts, R, k, gram, loss_dev);
    KL_CUDA(cudaGetLastError());
    const dim3 lg((n + 255) / 256, batch);
    const float scale = 1.f / float(k * batch);
    if (k <= 16)
        loss_grad<16><<<lg, 256, 0, s>>>(out, tgt, gram, n, k, scale, dzf, dzb);
    else if (k <= 32)
        loss_grad<32><<<lg, 256, 0, s>>>(out, tgt, gram, n, k, scale, dzf, dzb);
    else
        loss_grad<64><<<lg, 256, 0, s>>>(out, tgt, gram, n, k, scale, dzf, dzb);
    KL_CUDA(cudaGetLastError());
    count_launches(3);

    for (int l = m->layers - 1; l >= 0; --l) {
        const int di = m->din[size_t(l)], dout = m->dout[size_t(l)];
        const bf16* hin = hb + m->aoff[size_t(l)];
        // dW^T = dZ^T H: A = dZ^T (dout x ldb), B = H^T (di x ldb), zero columns beyond the batch
        transpose_bf16<<<dim3((dout + 31) / 32, (ldb + 31) / 32), dim3(32, 8), 0, s>>>(dzb, batch, dout, dout, dzt, ldb);
        transpose_bf16<<<dim3((di + 31) / 32, (ldb + 31) / 32), dim3(32, 8), 0, s>>>(hin, batch, di, di, ht, ldb);
        KL_CUDA(cudaGetLastError());
        count_launches(2);
        KL_TRY(tc_gemm(dout, di, ldb, dzt, ldb, ht, ldb, int(round_up(size_t(ldb), kTcK)), nullptr, 0,
                       m->G + m->woff[size_t(l)], nullptr, dout, status_ptr(m), s));
        column_sums<<<(dout + 255) / 256, 256, 0, s>>>(dzf, batch, dout, m->G + m->boff[size_t(l)]);
        KL_CUDA(cudaGetLastError());
        count_launches(1);
        if (l == 0) break;
        // dH^T = W dZ^T, then through tanh: dz_{l-1} = dH (1 - h^2)
        const float* hprev = hf + m->aoff[size_t(l)];
        const bf16* w = m->Wb + m->woff[size_t(l)];
        if (tc_shape_ok(dout, w, dout, dzb, dout)) {
            const int tiles = ((di + kTcM - 1) / kTcM) * ((batch + 255) / 256);
            const int kchunk = tc_kchunk(tiles, dout);
            const int splits = (dout + kchunk - 1) / kchunk;
            KL_TRY(grow(m->part, size_t(splits) * batch * di * sizeof(float), s));
            float* part = static_cast<float*>(m->part.ptr);
            KL_TRY(tc_gemm(di, batch, dout, w, dout, dzb, dout, kchunk, nullptr, 0, part, nullptr, di, status_ptr(m),
                           s));
            split_tanh_backward<<<blocks_for(size_t(batch) * di), 256, 0, s>>>(part, splits, size_t(batch) * di, hprev,
                                                                               dzf, dzb);
        } else {
            float* dh = static_cast<float*>(m->dh.ptr);
            KL_TRY(gemm(m, batch, di, dout, dzb, dout, 1, w, 1, dout, nullptr, 0, dh, nullptr, s));
            split_tanh_backward<<<blocks_for(size_t(batch) * di), 256, 0, s>>>(dh, 1, size_t(batch) * di, hprev, dzf,
                                                                               dzb);
        }
        KL_CUDA(cudaGetLastError());
        count_launches(1);
    }
    return KL_OK;
}

kl_status refresh_copies(kl_mlp m, int update, double lr, cudaStream_t s) {
    float c1 = 1.f, c2 = 1.f;
    if (update) {
        m->t += 1;
        c1 = float(1.0 - std::pow(0.9, m->t));
        c2 = float(1.0 - std::pow(0.999, m->t));
    }
    for (int l = 0; l < m->layers; ++l) {
        const int di = m->din[size_t(l)], dout = m->dout[size_t(l)];
        if (dout % 4 == 0 && m->woff[size_t(l)] % 4 == 0)
            adam_layer4<<<dim3((dout + 127) / 128, (di + 1 + 31) / 32), dim3(32, 8), 0, s>>>(
                m->P, m->G, m->M, m->V, m->Wb, m->Wt + m->wtoff[size_t(l)], m->woff[size_t(l)], di, dout, update,
                float(lr), 0.9f, 0.999f, 1e-8f, c1, c2);
        else
            adam_layer<<<dim3((dout + 31) / 32, (di + 1 + 31) / 32), dim3(32, 8), 0, s>>>(
                m->P, m->G, m->M, m->V, m->Wb, m->Wt + m->wtoff[size_t(l)], m->woff[size_t(l)], di, dout, update,
                float(lr), 0.9f, 0.999f, 1e-8f, c1, c2);
        KL_CUDA(cudaGetLastError());
    }
    count_launches(m->layers);
    return KL_OK;
}

}  // namespace
}  // namespace kl

using namespace kl;

extern "C" {

kl_status kl_mlp_create(int n_in, int width, int depth, int n_out, uint64_t seed, kl_mlp* out) {
    if (!out) return fail(KL_ERR_INVALID_ARG, "null output");
    *out = nullptr;
    if (n_in < 1 || width < 1 || depth < 1 || n_out < 1 || depth > 16)
        return fail(KL_ERR_INVALID_ARG, "network sizes must be positive (1..16 hidden layers)");
    kl_mlp m = new (std::nothrow) kl_mlp_s();
    if (!m) return fail(KL_ERR_OOM, "host allocation failed");
    m->n_in = n_in;
    m->width = width;
    m->depth = depth;
    m->n_out = n_out;
    m->layers = depth + 1;
    size_t off = 0, toff = 0;
    for (int l = 0; l < m->layers; ++l) {
        m->din.push_back(l == 0 ? n_in : width);
        m->dout.push_back(l == m->layers - 1 ? n_out : width);
        m->woff.push_back(off);
        off += size_t(m->din.back()) * m->dout.back();
        m->boff.push_back(off);
        off += size_t(m->dout.back());
        m->wtoff.push_back(toff);
        toff += round_up(size_t(m->din.back()) * m->dout.back(), 8);
    }
    m->nparam = off;
    m->nwt = toff;
    // initialisation: uniform(-a, a), a = sqrt(3 / fan_in) (unit variance per layer), biases 0;
    // splitmix64 stream from the seed, drawn on the host
    std::vector<float> P(off, 0.f);
    uint64_t state = seed;
    auto next = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return double(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < m->layers; ++l) {
        const double a = std::sqrt(3.0 / m->din[size_t(l)]);
        for (size_t i = 0; i < size_t(m->din[size_t(l)]) * m->dout[size_t(l)]; ++i)
            P[m->woff[size_t(l)] + i] = float((2.0 * next() - 1.0) * a);
    }
    kl_status st = KL_OK;
    auto chk = [&](cudaError_t e) {
        if (st == KL_OK && e != cudaSuccess) st = cuda_fail(e, "warm-start network allocation");
    };
    chk(cudaMalloc(&m->P, off * sizeof(float)));
    chk(cudaMalloc(&m->G, off * sizeof(float)));
    chk(cudaMalloc(&m->M, off * sizeof(float)));
    chk(cudaMalloc(&m->V, off * sizeof(float)));
    chk(cudaMalloc(&m->Wb, off * sizeof(bf16)));
    chk(cudaMalloc(&m->Wt, std::max<size_t>(toff, 8) * sizeof(bf16)));
    if (st == KL_OK) st = ensure(m->status, sizeof(int));
    if (st == KL_OK) {
        chk(cudaMemcpy(m->P, P.data(), off * sizeof(float), cudaMemcpyHostToDevice));
        chk(cudaMemset(m->M, 0, off * sizeof(float)));
        chk(cudaMemset(m->V, 0, off * sizeof(float)));
        chk(cudaMemset(m->G, 0, off * sizeof(float)));
        chk(cudaMemset(m->status.ptr, 0, sizeof(int)));
    }
    if (st == KL_OK) st = refresh_copies(m, 0, 0.0, nullptr);
    if (st == KL_OK) chk(cudaStreamSynchronize(nullptr));
    if (st != KL_OK) {
        kl_mlp_destroy(m);
        return st;
    }
    *out = m;
    return KL_OK;
}

kl_status kl_mlp_params(kl_mlp m, float* host, int direction) {
    if (!m || !host) return fail(KL_ERR_INVALID_ARG, "null argument");
    if (direction == 0) {
        KL_CUDA(cudaMemcpy(host, m->P, m->nparam * sizeof(float), cudaMemcpyDeviceToHost));
    } else {
        KL_CUDA(cudaMemcpy(m->P, host, m->nparam * sizeof(float), cudaMemcpyHostToDevice));
        KL_TRY(refresh_copies(m, 0, 0.0, nullptr));
        KL_CUDA(cudaStreamSynchronize(nullptr));
    }
    return KL_OK;
}

kl_status kl_mlp_num_params(kl_mlp m, int64_t* n) {
    if (!m || !n) return fail(KL_ERR_INVALID_ARG, "null argument");
    *n = int64_t(m->nparam);
    return KL_OK;
}

kl_status kl_mlp_forward(kl_mlp m, const float* x_dev, int batch, float* out_dev, void* stream) {
    if (!m || (batch > 0 && (!x_dev || !out_dev)) || batch < 0) return fail(KL_ERR_INVALID_ARG, "bad argument");
    if (batch == 0) return KL_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    KL_TRY(forward_impl(m, x_dev, batch, s));
    KL_CUDA(cudaMemcpyAsync(out_dev, static_cast<float*>(m->hf.ptr) + m->aoff[size_t(m->layers)],
                            size_t(batch) * m->n_out * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return check_status(m, s);
}

kl_status kl_mlp_loss_grad(kl_mlp m, const float* x_dev, const float* tgt_dev, int batch, int k, int n, float* loss_dev,
                           float* grad_host, void* stream) {
    if (!m || !x_dev || !tgt_dev || !loss_dev || batch < 1 || k < 1 || n < 1 || int64_t(k) * n != m->n_out)
        return fail(KL_ERR_INVALID_ARG, "bad argument (the output must hold k vectors of length n)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    KL_TRY(forward_impl(m, x_dev, batch, s));
    KL_TRY(backward_impl(m, tgt_dev, batch, k, n, loss_dev, s));
    if (grad_host) KL_CUDA(cudaMemcpyAsync(grad_host, m->G, m->nparam * sizeof(float), cudaMemcpyDeviceToHost, s));
    return check_status(m, s);
}

kl_status kl_mlp_train(kl_mlp m, const float* x_dev, const float* tgt_dev, int samples, int k, int n, int epochs,
                       int batch, double lr, uint64_t seed, double* loss_host, void* stream) {
    if (!m || !x_dev || !tgt_dev || samples < 1 || k < 1 || n < 1 || int64_t(k) * n != m->n_out || epochs < 0 ||
        batch < 1)
        return fail(KL_ERR_INVALID_ARG, "bad argument (the output must hold k vectors of length n)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (batch > samples) batch = samples;
    const int nb = samples / batch;
    DevBuf xb, tb, lb, ib;
    KL_TRY(ensure(xb, size_t(batch) * m->n_in * sizeof(float)));
    KL_TRY(ensure(tb, size_t(batch) * m->n_out * sizeof(float)));
    KL_TRY(ensure(lb, size_t(std::max(1, epochs)) * nb * batch * sizeof(float)));
    KL_TRY(ensure(ib, size_t(samples) * sizeof(int)));
    std::vector<int> order(static_cast<size_t>(samples));
    for (int i = 0; i < samples; ++i) order[size_t(i)] = i;
    uint64_t state = seed;
    auto next = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    float* losses = static_cast<float*>(lb.ptr);
    kl_status st = KL_OK;
    for (int ep = 0; ep < epochs && st == KL_OK; ++ep) {
        // seeded shuffle (Fisher-Yates), one upload of the epoch's order
        for (int i = samples - 1; i > 0; --i) std::swap(order[size_t(i)], order[size_t(next() % uint64_t(i + 1))]);
        KL_CUDA(cudaStreamSynchronize(s));
        KL_CUDA(cudaMemcpy(ib.ptr, order.data(), size_t(samples) * sizeof(int), cudaMemcpyHostToDevice));
        const int* idx = static_cast<const int*>(ib.ptr);
        for (int bi = 0; bi < nb && st == KL_OK; ++bi) {
            const int b0 = bi * batch;
            gather_rows<<<blocks_for(size_t(batch) * m->n_in), 256, 0, s>>>(x_dev, idx + b0, batch, m->n_in,
                                                                             static_cast<float*>(xb.ptr));
            gather_rows<<<blocks_for(size_t(batch) * m->n_out), 256, 0, s>>>(tgt_dev, idx + b0, batch, m->n_out,
                                                                              static_cast<float*>(tb.ptr));
            KL_CUDA(cudaGetLastError());
            count_launches(2);
            st = forward_impl(m, static_cast<float*>(xb.ptr), batch, s);
            if (st == KL_OK)
                st = backward_impl(m, static_cast<float*>(tb.ptr), batch, k, n, losses + (size_t(ep) * nb + bi) * batch,
                                   s);
            if (st == KL_OK) st = refresh_copies(m, 1, lr, s);
        }
    }
    if (st == KL_OK) st = check_status(m, s);
    if (st == KL_OK && loss_host && epochs > 0) {
        std::vector<float> lh(size_t(epochs) * nb * batch);
        KL_CUDA(cudaMemcpy(lh.data(), losses, lh.size() * sizeof(float), cudaMemcpyDeviceToHost));
        for (int ep = 0; ep < epochs; ++ep) {
            double sum = 0.0;
            for (size_t j = 0; j < size_t(nb) * batch; ++j) sum += lh[size_t(ep) * nb * batch + j];
            loss_host[ep] = nb ? sum / (double(nb) * batch) : 0.0;
        }
    }
    cudaStreamSynchronize(s);
    release(xb);
    release(tb);
    release(lb);
    release(ib);
    return st;
}

void kl_mlp_destroy(kl_mlp m) {
    if (!m) return;
    if (m->P) cudaFree(m->P);
    if (m->G) cudaFree(m->G);
    if (m->M) cudaFree(m->M);
    if (m->V) cudaFree(m->V);
    if (m->Wb) cudaFree(m->Wb);
    if (m->Wt) cudaFree(m->Wt);
    release(m->hf);
    release(m->hb);
    release(m->ht);
    release(m->dzf);
    release(m->dzb);
    release(m->dzt);
    release(m->dh);
    release(m->part);
    release(m->gpart);
    release(m->gram);
    release(m->status);
    delete m;
}

}  // extern "C"
