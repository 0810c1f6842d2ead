// Learned warm start: a multilayer perceptron (bfloat16 weights and layer inputs, float32
// sums, tanh hidden layers, linear output) that maps problem parameters to the coefficients
// of k standard-form vectors on a coarse mesh, trained on eigenpairs the solver generates with
// a loss on orthogonal projectors, ||Y Y^T - V V^T||_F^2 / k (rotation and sign invariant):
//   loss = ||Y^T Y||_F^2 - 2 ||V^T Y||_F^2 + ||V^T V||_F^2,   dL/dY = 4 Y (Y^T Y) - 4 V (V^T Y).
//
// Kernels: a tiled GEMM for bfloat16 operands with float32 accumulation (any strides, so the
// forward product and both backward products use it; long contractions are split over CTAs
// and the splits added in a fixed order), bias + tanh epilogues, column sums, the per-sample
// Gram matrices of the loss, the loss gradient, and Adam (Kingma and Ba 2015, Algorithm 1)
// with float32 master weights and a bfloat16 copy refreshed after every step.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kl_internal.h"

struct kl_mlp_s {
    int n_in = 0, width = 0, depth = 0, n_out = 0;
    int layers = 0;
    std::vector<int> din, dout;                 // per layer
    std::vector<size_t> woff, boff;             // offsets into the flat parameter array
    size_t nparam = 0;
    float* P = nullptr;                         // float32 master parameters (weights then biases per layer)
    float* G = nullptr;                         // gradients
    float* M = nullptr;                         // Adam first moments
    float* V = nullptr;                         // Adam second moments
    __nv_bfloat16* Wb = nullptr;                // bfloat16 copy of the parameters
    int t = 0;                                  // Adam step
    kl::DevBuf act, actb, dz, dzb, part, gram, lossbuf;
};

namespace kl {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kGemmThreads = 256;

// C[m][n] (+)= sum_k A(m,k) B(k,n) over k in [k0, k1); A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn].
// Output of split z to out + z * M * N (row-major, float32).
__global__ void __launch_bounds__(kGemmThreads)
gemm_bf16_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int64_t sam, int64_t sak,
                 const __nv_bfloat16* __restrict__ B, int64_t sbk, int64_t sbn, float* __restrict__ out, int kchunk) {
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
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
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
                              int tanh_act, float* __restrict__ out, __nv_bfloat16* __restrict__ outb) {
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

// dz = dh * (1 - h^2) with h = tanh(z) kept from the forward pass; bfloat16 copy
__global__ void tanh_backward(const float* __restrict__ dh, const float* __restrict__ h, size_t n, float* __restrict__ dz,
                              __nv_bfloat16* __restrict__ dzb) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const float v = dh[i] * (1.f - h[i] * h[i]);
        dz[i] = v;
        dzb[i] = __float2bfloat16_rn(v);
    }
}

__global__ void to_bf16(const float* __restrict__ x, size_t n, __nv_bfloat16* __restrict__ y) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// db[n] = sum over rows m of dz[m][n] (fixed order)
__global__ void column_sums(const float* __restrict__ dz, int M, int N, float* __restrict__ db) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int m = 0; m < M; ++m) s += dz[size_t(m) * N + n];
        db[n] = s;
    }
}

// per sample s (one CTA): YtY = Y^T Y and VtY = V^T Y (k x k), Y[i][a] = out[s][a*n + i],
// V[i][a] = tgt[s][a*n + i]; loss[s] = (||YtY||^2 - 2 ||VtY||^2 + ||V^T V||^2) / k
__global__ void loss_gram(const float* __restrict__ out, const float* __restrict__ tgt, int n, int k,
                          float* __restrict__ gram, float* __restrict__ loss) {
    extern __shared__ float sg[];        // YtY, VtY, VtV: 3 k*k
    const int s = blockIdx.x;
    const float* Y = out + size_t(s) * k * n;
    const float* V = tgt + size_t(s) * k * n;
    const int kk = k * k;
    for (int e = threadIdx.x; e < 3 * kk; e += blockDim.x) {
        const int which = e / kk, ab = e - which * kk, a = ab / k, b = ab - a * k;
        const float* X1 = which == 0 ? Y : V;
        const float* X2 = which == 2 ? V : Y;
        float acc = 0.f;
        for (int i = 0; i < n; ++i) acc = fmaf(X1[size_t(a) * n + i], X2[size_t(b) * n + i], acc);
        sg[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) gram[size_t(s) * 2 * kk + e] = sg[e];
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int e = 0; e < kk; ++e) l += sg[e] * sg[e] - 2.f * sg[kk + e] * sg[kk + e] + sg[2 * kk + e] * sg[2 * kk + e];
        loss[s] = l / float(k);
    }
}

// dY[s][b*n + i] = scale * (4 sum_a Y[i][a] YtY[a][b] - 4 sum_a V[i][a] VtY[a][b])
__global__ void loss_grad(const float* __restrict__ out, const float* __restrict__ tgt, const float* __restrict__ gram,
                          int n, int k, int samples, float scale, float* __restrict__ dy, __nv_bfloat16* __restrict__ dyb) {
    const size_t total = size_t(samples) * k * n;
    const int kk = k * k;
    for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
        const size_t s = idx / (size_t(k) * n);
        const size_t r = idx - s * size_t(k) * n;
        const int b = int(r / n), i = int(r - size_t(b) * n);
        const float* Y = out + s * k * n;
        const float* V = tgt + s * k * n;
        const float* YtY = gram + s * 2 * kk;
        const float* VtY = YtY + kk;
        float acc = 0.f;
        for (int a = 0; a < k; ++a) acc = fmaf(Y[size_t(a) * n + i], YtY[a * k + b], fmaf(-V[size_t(a) * n + i], VtY[a * k + b], acc));
        const float g = 4.f * scale * acc;
        dy[idx] = g;
        dyb[idx] = __float2bfloat16_rn(g);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            __nv_bfloat16* __restrict__ pb, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16_rn(pi);
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

// out (+ bias, act) = A x B with the strides described at gemm_bf16_kernel
kl_status gemm(kl_mlp m, int M, int N, int K, const __nv_bfloat16* A, int64_t sam, int64_t sak, const __nv_bfloat16* B,
               int64_t sbk, int64_t sbn, const float* bias, int act, float* out, __nv_bfloat16* outb, cudaStream_t s) {
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

size_t act_floats(kl_mlp m, int batch) {
    size_t t = size_t(batch) * m->n_in;
    for (int l = 0; l < m->layers; ++l) t += size_t(batch) * m->dout[l];
    return t;
}

// forward for `batch` rows of x (float32, batch x n_in); activations kept for backward
kl_status forward_impl(kl_mlp m, const float* x, int batch, cudaStream_t s) {
    KL_TRY(grow(m->act, act_floats(m, batch) * sizeof(float), s));
    KL_TRY(grow(m->actb, act_floats(m, batch) * sizeof(__nv_bfloat16), s));
    float* a = static_cast<float*>(m->act.ptr);
    __nv_bfloat16* ab = static_cast<__nv_bfloat16*>(m->actb.ptr);
    KL_CUDA(cudaMemcpyAsync(a, x, size_t(batch) * m->n_in * sizeof(float), cudaMemcpyDeviceToDevice, s));
    to_bf16<<<blocks_for(size_t(batch) * m->n_in), 256, 0, s>>>(a, size_t(batch) * m->n_in, ab);
    KL_CUDA(cudaGetLastError());
    size_t off = size_t(batch) * m->n_in;
    size_t prev = 0;
    for (int l = 0; l < m->layers; ++l) {
        const int di = m->din[l], dout = m->dout[l];
        const bool last = (l == m->layers - 1);
        KL_TRY(gemm(m, batch, dout, di, ab + prev, di, 1, m->Wb + m->woff[l], dout, 1, m->P + m->boff[l], last ? 0 : 1,
                    a + off, ab + off, s));
        prev = off;
        off += size_t(batch) * dout;
    }
    return KL_OK;
}

// loss of the current outputs against targets (float32, batch x k*n) and backward pass into m->G
kl_status backward_impl(kl_mlp m, const float* tgt, int batch, int k, int n, float* loss_dev, cudaStream_t s) {
    float* a = static_cast<float*>(m->act.ptr);
    __nv_bfloat16* ab = static_cast<__nv_bfloat16*>(m->actb.ptr);
    std::vector<size_t> off(size_t(m->layers) + 1);
    off[0] = 0;
    size_t o = size_t(batch) * m->n_in;
    for (int l = 0; l < m->layers; ++l) {
        off[size_t(l) + 1] = o;
        o += size_t(batch) * m->dout[l];
    }
    const float* out = a + off[size_t(m->layers)];
    KL_TRY(grow(m->gram, size_t(batch) * 2 * k * k * sizeof(float), s));
    const size_t smem = size_t(3) * k * k * sizeof(float);
    if (smem > 48 * 1024) return fail(KL_ERR_INVALID_ARG, "warm-start loss: k too large");
    loss_gram<<<batch, 256, smem, s>>>(out, tgt, n, k, static_cast<float*>(m->gram.ptr), loss_dev);
    KL_CUDA(cudaGetLastError());
    size_t maxw = size_t(m->n_out);
    for (int l = 0; l < m->layers; ++l) maxw = std::max(maxw, size_t(m->din[l]));
    KL_TRY(grow(m->dz, 2 * size_t(batch) * maxw * sizeof(float), s));
    KL_TRY(grow(m->dzb, 2 * size_t(batch) * maxw * sizeof(__nv_bfloat16), s));
    float* dz = static_cast<float*>(m->dz.ptr);
    float* dh = dz + size_t(batch) * maxw;
    __nv_bfloat16* dzb = static_cast<__nv_bfloat16*>(m->dzb.ptr);
    loss_grad<<<blocks_for(size_t(batch) * k * n), 256, 0, s>>>(out, tgt, static_cast<float*>(m->gram.ptr), n, k, batch,
                                                                1.f / float(k * batch), dz, dzb);
    KL_CUDA(cudaGetLastError());
    count_launches(2);
    for (int l = m->layers - 1; l >= 0; --l) {
        const int di = m->din[l], dout = m->dout[l];
        // dW = h_{l-1}^T dz  (di x dout), db = column sums of dz
        KL_TRY(gemm(m, di, dout, batch, ab + off[size_t(l)], 1, di, dzb, dout, 1, nullptr, 0, m->G + m->woff[l], nullptr, s));
        column_sums<<<(dout + 255) / 256, 256, 0, s>>>(dz, batch, dout, m->G + m->boff[l]);
        KL_CUDA(cudaGetLastError());
        count_launches(1);
        if (l == 0) break;
        // dh_{l-1} = dz W^T (batch x di), then through tanh
        KL_TRY(gemm(m, batch, di, dout, dzb, dout, 1, m->Wb + m->woff[l], 1, dout, nullptr, 0, dh, nullptr, s));
        tanh_backward<<<blocks_for(size_t(batch) * di), 256, 0, s>>>(dh, a + off[size_t(l)], size_t(batch) * di, dz, dzb);
        KL_CUDA(cudaGetLastError());
        count_launches(1);
    }
    return KL_OK;
}

kl_status adam_impl(kl_mlp m, double lr, cudaStream_t s) {
    m->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = float(1.0 - std::pow(0.9, m->t)), c2 = float(1.0 - std::pow(0.999, m->t));
    adam_kernel<<<blocks_for(m->nparam), 256, 0, s>>>(m->P, m->G, m->M, m->V, m->Wb, m->nparam, float(lr), b1, b2, 1e-8f,
                                                      c1, c2);
    KL_CUDA(cudaGetLastError());
    count_launches(1);
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
    size_t off = 0;
    for (int l = 0; l < m->layers; ++l) {
        m->din.push_back(l == 0 ? n_in : width);
        m->dout.push_back(l == m->layers - 1 ? n_out : width);
        m->woff.push_back(off);
        off += size_t(m->din.back()) * m->dout.back();
        m->boff.push_back(off);
        off += size_t(m->dout.back());
    }
    m->nparam = off;
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
    std::vector<__nv_bfloat16> Pb(off);
    for (size_t i = 0; i < off; ++i) Pb[i] = __float2bfloat16_rn(P[i]);
    kl_status st = KL_OK;
    auto chk = [&](cudaError_t e) {
        if (st == KL_OK && e != cudaSuccess) st = cuda_fail(e, "warm-start network allocation");
    };
    chk(cudaMalloc(&m->P, off * sizeof(float)));
    chk(cudaMalloc(&m->G, off * sizeof(float)));
    chk(cudaMalloc(&m->M, off * sizeof(float)));
    chk(cudaMalloc(&m->V, off * sizeof(float)));
    chk(cudaMalloc(&m->Wb, off * sizeof(__nv_bfloat16)));
    if (st == KL_OK) {
        chk(cudaMemcpy(m->P, P.data(), off * sizeof(float), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(m->Wb, Pb.data(), off * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
        chk(cudaMemset(m->M, 0, off * sizeof(float)));
        chk(cudaMemset(m->V, 0, off * sizeof(float)));
        chk(cudaMemset(m->G, 0, off * sizeof(float)));
    }
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
        std::vector<__nv_bfloat16> Pb(m->nparam);
        for (size_t i = 0; i < m->nparam; ++i) Pb[i] = __float2bfloat16_rn(host[i]);
        KL_CUDA(cudaMemcpy(m->Wb, Pb.data(), m->nparam * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
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
    size_t off = size_t(batch) * m->n_in;
    for (int l = 0; l < m->layers - 1; ++l) off += size_t(batch) * m->dout[size_t(l)];
    KL_CUDA(cudaMemcpyAsync(out_dev, static_cast<float*>(m->act.ptr) + off, size_t(batch) * m->n_out * sizeof(float),
                            cudaMemcpyDeviceToDevice, s));
    return KL_OK;
}

kl_status kl_mlp_loss_grad(kl_mlp m, const float* x_dev, const float* tgt_dev, int batch, int k, int n, float* loss_dev,
                           float* grad_host, void* stream) {
    if (!m || !x_dev || !tgt_dev || !loss_dev || batch < 1 || k < 1 || n < 1 || k * n != m->n_out)
        return fail(KL_ERR_INVALID_ARG, "bad argument (the output must hold k vectors of length n)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    KL_TRY(forward_impl(m, x_dev, batch, s));
    KL_TRY(backward_impl(m, tgt_dev, batch, k, n, loss_dev, s));
    if (grad_host) {
        KL_CUDA(cudaMemcpyAsync(grad_host, m->G, m->nparam * sizeof(float), cudaMemcpyDeviceToHost, s));
        KL_CUDA(cudaStreamSynchronize(s));
    }
    return KL_OK;
}

kl_status kl_mlp_train(kl_mlp m, const float* x_dev, const float* tgt_dev, int samples, int k, int n, int epochs,
                       int batch, double lr, uint64_t seed, double* loss_host, void* stream) {
    if (!m || !x_dev || !tgt_dev || samples < 1 || k < 1 || n < 1 || k * n != m->n_out || epochs < 0 || batch < 1)
        return fail(KL_ERR_INVALID_ARG, "bad argument (the output must hold k vectors of length n)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (batch > samples) batch = samples;
    DevBuf xb, tb, lb, ib;
    KL_TRY(ensure(xb, size_t(batch) * m->n_in * sizeof(float)));
    KL_TRY(ensure(tb, size_t(batch) * m->n_out * sizeof(float)));
    KL_TRY(ensure(lb, size_t(batch) * sizeof(float)));
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
    std::vector<float> lh(static_cast<size_t>(samples));
    for (int ep = 0; ep < epochs; ++ep) {
        // seeded shuffle (Fisher-Yates), one upload of the epoch's order
        for (int i = samples - 1; i > 0; --i) std::swap(order[size_t(i)], order[size_t(next() % uint64_t(i + 1))]);
        KL_CUDA(cudaStreamSynchronize(s));
        KL_CUDA(cudaMemcpy(ib.ptr, order.data(), size_t(samples) * sizeof(int), cudaMemcpyHostToDevice));
        const int* idx = static_cast<const int*>(ib.ptr);
        double ep_loss = 0.0;
        int used = 0;
        for (int b0 = 0; b0 + batch <= samples; b0 += batch) {
            gather_rows<<<blocks_for(size_t(batch) * m->n_in), 256, 0, s>>>(x_dev, idx + b0, batch, m->n_in,
                                                                             static_cast<float*>(xb.ptr));
            gather_rows<<<blocks_for(size_t(batch) * m->n_out), 256, 0, s>>>(tgt_dev, idx + b0, batch, m->n_out,
                                                                              static_cast<float*>(tb.ptr));
            KL_CUDA(cudaGetLastError());
            count_launches(2);
            KL_TRY(forward_impl(m, static_cast<float*>(xb.ptr), batch, s));
            KL_TRY(backward_impl(m, static_cast<float*>(tb.ptr), batch, k, n, static_cast<float*>(lb.ptr), s));
            KL_TRY(adam_impl(m, lr, s));
            if (loss_host) {
                KL_CUDA(cudaMemcpyAsync(lh.data(), lb.ptr, size_t(batch) * sizeof(float), cudaMemcpyDeviceToHost, s));
                KL_CUDA(cudaStreamSynchronize(s));
                for (int j = 0; j < batch; ++j) ep_loss += lh[size_t(j)];
                used += batch;
            }
        }
        if (loss_host) loss_host[ep] = used ? ep_loss / used : 0.0;
    }
    KL_CUDA(cudaStreamSynchronize(s));
    release(xb);
    release(tb);
    release(lb);
    release(ib);
    return KL_OK;
}

void kl_mlp_destroy(kl_mlp m) {
    if (!m) return;
    if (m->P) cudaFree(m->P);
    if (m->G) cudaFree(m->G);
    if (m->M) cudaFree(m->M);
    if (m->V) cudaFree(m->V);
    if (m->Wb) cudaFree(m->Wb);
    release(m->act);
    release(m->actb);
    release(m->dz);
    release(m->dzb);
    release(m->part);
    release(m->gram);
    release(m->lossbuf);
    delete m;
}

}  // extern "C"
