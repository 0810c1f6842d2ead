// Sum-factorised Kronecker contractions, stages 1-4 and 6-9 of Algorithm 1.
//
// (C_d (x) ... (x) C_1) vec(X) is applied as d mode products (Sec. 2.2): a block of
// tensors stored in vec order is viewed, for mode k, as [A][n][B] with B = n_1 ... n_{k-1}
// and A = n_{k+1} ... n_d, and every fibre along the middle index is multiplied by the
// small dense factor.  One thread computes one output entry; consecutive threads take
// consecutive b (or consecutive i when B == 1), so global loads and stores are coalesced
// and the factor is read from shared memory without bank conflicts.  The tensors are at
// most a few MB per vector and stay L2-resident between the mode passes.
#include "kl_internal.h"

namespace kl {
namespace {

constexpr int kContractThreads = 256;

constexpr size_t kFactorSmemMax = 48 * 1024;   // larger factors are read through L1/L2

template <typename Tin, typename Tc, typename Tout, bool kSmem>
__global__ void __launch_bounds__(kContractThreads)
contract_kernel(const Tin* __restrict__ X, int64_t ldx, Tout* __restrict__ Y, int64_t ldy,
                const Tc* __restrict__ Ct, int64_t A, int n, int m, int64_t B, int nvec,
                const Tc* __restrict__ scale) {
    extern __shared__ unsigned char smem_raw[];
    const Tc* sC = Ct;
    if (kSmem) {
        Tc* s = reinterpret_cast<Tc*>(smem_raw);
        for (int e = threadIdx.x; e < n * m; e += blockDim.x) s[e] = Ct[e];
        __syncthreads();
        sC = s;
    }

    const int64_t per_vec = A * m * B;
    const int64_t total = per_vec * nvec;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        int64_t v = idx / per_vec;
        int64_t r = idx - v * per_vec;
        int64_t b, i, a;
        if (B == 1) {
            b = 0;
            i = r % m;
            a = r / m;
        } else {
            b = r % B;
            int64_t ai = r / B;
            i = ai % m;
            a = ai / m;
        }
        const Tin* xf = X + v * ldx + a * n * B + b;
        Tc acc = Tc(0);
#pragma unroll 4
        for (int j = 0; j < n; ++j) acc = fma(sC[j * m + i], Tc(xf[int64_t(j) * B]), acc);
        if (scale) acc *= scale[r];
        Y[v * ldy + r] = Tout(acc);
    }
}

}  // namespace

template <typename Tin, typename Tc, typename Tout>
cudaError_t launch_contract(const Tin* X, int64_t ldx, Tout* Y, int64_t ldy, const Tc* Ct, int64_t A,
                            int n, int m, int64_t B, int nvec, const Tc* scale, cudaStream_t s) {
    int64_t total = A * m * B * nvec;
    if (total == 0) return cudaSuccess;
    int64_t blocks = (total + kContractThreads - 1) / kContractThreads;
    if (blocks > num_sms() * 16) blocks = num_sms() * 16;
    const size_t smem = size_t(n) * m * sizeof(Tc);
    count_launches(1);
    if (smem <= kFactorSmemMax)
        contract_kernel<Tin, Tc, Tout, true><<<int(blocks), kContractThreads, smem, s>>>(X, ldx, Y, ldy, Ct, A, n,
                                                                                        m, B, nvec, scale);
    else
        contract_kernel<Tin, Tc, Tout, false><<<int(blocks), kContractThreads, 0, s>>>(X, ldx, Y, ldy, Ct, A, n,
                                                                                      m, B, nvec, scale);
    return cudaGetLastError();
}

template cudaError_t launch_contract<double, double, double>(const double*, int64_t, double*, int64_t,
                                                             const double*, int64_t, int, int, int64_t,
                                                             int, const double*, cudaStream_t);
template cudaError_t launch_contract<double, float, float>(const double*, int64_t, float*, int64_t,
                                                           const float*, int64_t, int, int, int64_t, int,
                                                           const float*, cudaStream_t);
template cudaError_t launch_contract<float, float, float>(const float*, int64_t, float*, int64_t,
                                                          const float*, int64_t, int, int, int64_t, int,
                                                          const float*, cudaStream_t);
template cudaError_t launch_contract<float, float, double>(const float*, int64_t, double*, int64_t,
                                                           const float*, int64_t, int, int, int64_t, int,
                                                           const float*, cudaStream_t);
template cudaError_t launch_contract<double, float, double>(const double*, int64_t, double*, int64_t,
                                                            const float*, int64_t, int, int, int64_t,
                                                            int, const float*, cudaStream_t);

}  // namespace kl
