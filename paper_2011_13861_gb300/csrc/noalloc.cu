// Allocation-free variant of the stage-5 kernel product (kl_covmv_noalloc).
//
// Who needs it: callers that must not allocate device memory at the point where they apply
// the operator -- for example an application that takes all of its device memory at start-up
// (a fixed budget shared with other work) and forbids allocation afterwards, or a loop that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree between steps.
// kl_covmv may grow the handle's workspace on first use with a wider block; this entry point
// never does.  It takes its split-partial scratch from a fixed file-scope device array instead.
//
// The array is part of the library image: every GPU on which the library's module is loaded
// holds it (32 MiB) until the process exits.  In host code the name `g_stage5_scratch` is only
// a host-side stand-in, so its device address is looked up with cudaGetSymbolAddress once per
// device (with that device current) the first time this entry point runs there; that first
// call should therefore happen before any stream capture begins.  The address is cached
// together with the identity of the CUDA context it belongs to; after a cudaDeviceReset (or
// anything else that destroys and recreates the context) the next call sees a different
// context and looks the address up again, so a stale address is never used.  Every call
// shares the array: calls whose launches overlap on the GPU (different streams, or different
// host threads) race on it and must be ordered by the caller.  Nothing in it needs to start at
// zero: each call writes every partial it later reads.
#include <cuda.h>

#include <mutex>

#include "kl_internal.h"

namespace kl {
namespace {

constexpr int64_t kScratchDoubles = int64_t(4) << 20;   // 4 Mi doubles = 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_stage5_scratch[kScratchDoubles];

std::mutex g_scratch_mutex;

struct ScratchSlot {
    double* addr = nullptr;
    unsigned long long ctx_id = 0;   // cuCtxGetId of the context the address belongs to
    bool ctx_known = false;
};
ScratchSlot g_scratch[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Identity of the calling thread's current context, through driver entry points that the
// runtime hands out (no link-time dependency on the driver library).  False when the driver
// does not provide them or no context is current yet.
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

kl_status scratch_address(double** out) {
    int dev = 0;
    KL_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(KL_ERR_INVALID_ARG, "device ordinal above 63");
    unsigned long long id = 0;
    bool known = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchSlot& slot = g_scratch[dev];
    if (slot.addr && known && slot.ctx_known && slot.ctx_id == id) {
        *out = slot.addr;
        return KL_OK;
    }
    // first call on this device, a context that was recreated since, or a context whose
    // identity cannot be read: look the address up (this also makes the primary context current)
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_stage5_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress(stage-5 scratch)");
    if (!known) known = current_context_id(&id);
    slot.addr = static_cast<double*>(p);
    slot.ctx_id = id;
    slot.ctx_known = known;
    *out = slot.addr;
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
