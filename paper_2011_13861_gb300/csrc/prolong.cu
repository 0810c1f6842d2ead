// Exact prolongation of standard-form vectors between nested trial spaces (the coarse-to-fine
// step of the learned warm start): one mode contraction per direction with
// Q_k = L_f^T P_k L_c^{-T} (built on the host by build_prolongation, setup.cpp).
#include <vector>

#include "kl_internal.h"

using namespace kl;

extern "C" kl_status kl_prolong(kl_handle coarse, kl_handle fine, const double* v_dev, double* y_dev, int nvec,
                                void* stream) {
    if (!coarse || !fine) return fail(KL_ERR_INVALID_ARG, "null handle");
    if (coarse->dim != fine->dim) return fail(KL_ERR_INVALID_ARG, "prolongation: dimensions differ");
    if (nvec < 0) return fail(KL_ERR_INVALID_ARG, "nvec < 0");
    if (nvec == 0) return KL_OK;
    if (!v_dev || !y_dev) return fail(KL_ERR_INVALID_ARG, "null vector pointer");
    const int d = coarse->dim;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // factors, uploaded transposed (n_c x n_f row-major): the contraction reads Ct[j * m + i]
    std::vector<double> host;
    std::vector<size_t> off(static_cast<size_t>(d));
    for (int k = 0; k < d; ++k) {
        std::vector<double> Q;
        KL_TRY(build_prolongation(coarse->dir[k], fine->dir[k], &Q));
        const int nf = fine->n[k], nc = coarse->n[k];
        off[size_t(k)] = host.size();
        for (int j = 0; j < nc; ++j)
            for (int i = 0; i < nf; ++i) host.push_back(Q[size_t(i) * nc + j]);
    }
    DevBuf fac;
    KL_TRY(ensure(fac, host.size() * sizeof(double)));
    KL_CUDA(cudaMemcpyAsync(fac.ptr, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    // ping-pong through the fine handle's workspace (every intermediate is at most N_f long)
    KL_TRY(ensure(fine->w_a, size_t(fine->N) * nvec * sizeof(double)));
    KL_TRY(ensure(fine->w_b, size_t(fine->N) * nvec * sizeof(double)));
    double* bufs[2] = {static_cast<double*>(fine->w_a.ptr), static_cast<double*>(fine->w_b.ptr)};
    const double* cur = v_dev;
    int64_t ldcur = coarse->N;
    const double* facs = static_cast<const double*>(fac.ptr);
    for (int k = 0; k < d; ++k) {
        // tensor [n_c,d .. n_c,k+1][n_c,k][n_f,k-1 .. n_f,1]: modes above k still coarse, below fine
        int64_t A = 1, B = 1;
        for (int i = k + 1; i < d; ++i) A *= coarse->n[i];
        for (int i = 0; i < k; ++i) B *= fine->n[i];
        const bool last = (k == d - 1);
        double* out = last ? y_dev : bufs[k % 2];
        const int64_t ldo = last ? fine->N : fine->N;
        cudaError_t e = launch_contract<double, double, double>(cur, ldcur, out, ldo, facs + off[size_t(k)], A,
                                                                coarse->n[k], fine->n[k], B, nvec, nullptr, s);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(s);
            release(fac);
            return cuda_fail(e, "prolongation contraction");
        }
        cur = out;
        ldcur = fine->N;
    }
    // the factor buffer is released once the contractions that read it are done
    KL_CUDA(cudaStreamSynchronize(s));
    release(fac);
    return KL_OK;
}
