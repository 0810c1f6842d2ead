// Allocation-free variant of the stage-5 kernel product (kl_covmv_noalloc).
//
// Who needs it: code that must not allocate device memory at the point where it applies the
// operator -- for example a solver step recorded while a CUDA stream is being captured into a
// graph (cudaMalloc is not allowed during capture), or an application that pre-allocates
// everything at start-up and forbids allocation afterwards.  kl_covmv may grow the handle's
// workspace on first use with a wider block; this entry point never does.  It takes its
// split-partial scratch from a fixed file-scope device array instead.
//
// The array is part of the library image: every GPU on which the library's module is loaded
// holds it (32 MiB) until the process exits.  In host code the name `g_stage5_scratch` is only
// a host-side stand-in, so its device address is looked up with cudaGetSymbolAddress once per
// device (with that device current) the first time this entry point runs there; that first
// call should therefore happen before any stream capture begins.  Every call shares the array:
// calls whose launches overlap on the GPU (different streams, or different host threads)
// race on it and must be ordered by the caller.  Nothing in it needs to start at zero: each
// call writes every partial it later reads.
#include <mutex>

#include "kl_internal.h"

namespace kl {
namespace {

constexpr int64_t kScratchDoubles = int64_t(4) << 20;   // 4 Mi doubles = 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_stage5_scratch[kScratchDoubles];

std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

kl_status scratch_address(double** out) {
    int dev = 0;
    KL_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(KL_ERR_INVALID_ARG, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_stage5_scratch);
        if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress(stage-5 scratch)");
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return KL_OK;
}

}  // namespace
}  // namespace kl

using namespace kl;

extern "C" kl_status kl_covmv_noalloc(kl_handle h, int precision, const double* u_dev, int64_t ldu, double* z_dev,
                                      int64_t ldz, int nvec, void* stream) {
    if (!h) return fail(KL_ERR_INVALID_ARG, "null handle");
    if (precision != KL_P_FP64) return fail(KL_ERR_INVALID_ARG, "kl_covmv_noalloc supports KL_P_FP64 only");
    if (nvec < 0) return fail(KL_ERR_INVALID_ARG, "nvec < 0");
    if (nvec == 0) return KL_OK;
    if (!u_dev || !z_dev) return fail(KL_ERR_INVALID_ARG, "null vector pointer");
    if (ldu < h->Nt || ldz < h->Nt) return fail(KL_ERR_INVALID_ARG, "leading dimension smaller than Ntilde");
    // the stage-5 launcher processes vectors in groups of up to 16; one group's partials
    // (splits x group x Ntilde doubles) must fit in the fixed scratch array
    const int group = nvec >= 16 ? 16 : nvec >= 8 ? 8 : nvec >= 4 ? 4 : nvec >= 2 ? 2 : 1;
    const int64_t per_split = int64_t(group) * h->Nt;
    if (per_split > kScratchDoubles)
        return fail(KL_ERR_INVALID_ARG,
                    "kl_covmv_noalloc: Ntilde x min(nvec,16) = " + std::to_string(per_split) +
                        " exceeds the fixed scratch of " + std::to_string(kScratchDoubles) +
                        " doubles (32 MiB); use kl_covmv or fewer vectors per call");
    int splits = covmv_splits(h->Nt, nvec, false);
    const int64_t fit = kScratchDoubles / per_split;
    if (splits > fit) splits = int(fit);
    double* scratch = nullptr;
    KL_TRY(scratch_address(&scratch));
    CovParams cp;
    cp.kind = h->kernel.kind;
    cp.poly_m = int(h->kernel.L);
    cp.Nt = h->Nt;
    cp.ldp = h->Nt;
    cp.P64 = h->dP;
    cp.P32 = h->fP;
    cp.tab = h->dTab;
    const double s2 = h->kernel.sigma * h->kernel.sigma;
    cudaError_t e = launch_covmv64(cp, u_dev, ldu, nvec, z_dev, ldz, s2, nullptr, scratch, splits,
                                   static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stage-5 kernel product (no-alloc)");
    return KL_OK;
}
