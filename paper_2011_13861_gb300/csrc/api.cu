// C ABI entry points, handle set-up and the operator application of Algorithm 1.
#include <algorithm>
#include <math.h>

#include <atomic>
#include <chrono>
#include <type_traits>
#include <cstring>
#include <string>
#include <vector>

#include "kl_internal.h"

namespace kl {

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
}

const std::string& last_error_message() { return g_last_error; }

void count_launches(int n) { g_launches.fetch_add(uint64_t(n), std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

kl_status fail(kl_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

kl_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? KL_ERR_OOM : KL_ERR_CUDA;
}

kl_status ensure(DevBuf& b, size_t bytes) {
    if (b.bytes >= bytes) return KL_OK;
    if (b.ptr) {
        cudaError_t e = cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
    }
    cudaError_t e = cudaMalloc(&b.ptr, bytes);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    b.bytes = bytes;
    return KL_OK;
}

void release(DevBuf& b) {
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
}

namespace {

template <typename T>
kl_status upload(T** dst, const T* src, size_t count) {
    KL_CUDA(cudaMalloc(reinterpret_cast<void**>(dst), count * sizeof(T)));
    KL_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return KL_OK;
}

int64_t stride_of(kl_handle h) { return h->ldw; }

kl_status check_block(kl_handle h, const void* a, const void* b, int nvec, int64_t lda, int64_t rows_a,
                      int64_t ldb, int64_t rows_b) {
    if (!h) return fail(KL_ERR_INVALID_ARG, "null handle");
    if (nvec < 0) return fail(KL_ERR_INVALID_ARG, "nvec < 0");
    if (nvec == 0) return KL_OK;
    if (!a || !b) return fail(KL_ERR_INVALID_ARG, "null vector pointer");
    if (lda < rows_a || ldb < rows_b) return fail(KL_ERR_INVALID_ARG, "leading dimension smaller than the vector length");
    return KL_OK;
}

// workspace for nvec columns of the intermediate tensors
kl_status ensure_apply_ws(kl_handle h, int nvec, bool fp32, bool tc64 = false) {
    const int64_t ld = stride_of(h);
    KL_TRY(ensure(h->w_a, size_t(ld) * nvec * sizeof(double)));
    KL_TRY(ensure(h->w_b, size_t(ld) * nvec * sizeof(double)));
    if (fp32) {
        KL_TRY(ensure(h->w_f32a, size_t(ld) * nvec * sizeof(float)));
        KL_TRY(ensure(h->w_f32b, size_t(ld) * nvec * sizeof(float)));
    }
    const int s64 = covmv_splits(h->Nt, nvec, false), s32 = covmv_splits(h->Nt, nvec, true);
    const int sdf = covmv_df_splits(h->Nt);
    size_t groups = size_t(s64) * 16;
    if (size_t(s32) * 16 > groups) groups = size_t(s32) * 16;   // float32 groups: at most 16 vectors
    if (size_t(sdf) * 32 > groups) groups = size_t(sdf) * 32;
    size_t part = size_t(h->Nt) * groups;
    const size_t dfp = covmv_df_part_doubles(h->Nt, nvec);
    if (dfp > part) part = dfp;
    const size_t symp = sym_part_doubles(h->Nt, nvec);   // symmetric float64 / float32 / double-float tiles
    if (symp > part) part = symp;
    if (fp32) {
        const size_t tcp = covmv_tc_part_doubles(h->Nt);
        if (tcp > part) part = tcp;
        KL_TRY(ensure(h->w_tcimg, covmv_tc_image_bytes(h->Nt)));
    }
    if (tc64) {
        const bool sym = tc_symmetric_used(h->Nt);
        const size_t tcp = sym ? covmv_tcs64_part_doubles(h->Nt) : covmv_tc64_part_doubles(h->Nt);
        if (tcp > part) part = tcp;
        KL_TRY(ensure(h->w_tcimg, sym ? covmv_tcs64_image_bytes(h->Nt) : covmv_tc64_image_bytes(h->Nt)));
    }
    KL_TRY(ensure(h->w_part, part * sizeof(double)));
    return KL_OK;
}

CovParams cov_params(kl_handle h) {
    CovParams cp;
    cp.kind = h->kernel.kind;
    cp.poly_m = int(h->kernel.L);
    cp.Nt = h->Nt;
    cp.ldp = h->Nt;
    cp.P64 = h->dP;
    cp.P32 = h->fP;
    cp.tab = h->dTab;
    cp.Pdf = h->dfP;
    cp.tabdf = h->dfTab;
    cp.gscale = h->gscale;
    return cp;
}

}  // namespace

CovParams cov_params_of(kl_handle h) { return cov_params(h); }

kl_status host_wait(kl_handle h, cudaStream_t s) {
    if (!h->batch) return KL_OK;
    if (!h->host_sync) KL_CUDA(cudaEventCreateWithFlags(&h->host_sync, cudaEventBlockingSync | cudaEventDisableTiming));
    KL_CUDA(cudaEventRecord(h->host_sync, s));
    KL_CUDA(cudaEventSynchronize(h->host_sync));
    return KL_OK;
}

// Reads (and clears) the device status word written by kernels with bounded waits.
kl_status check_device_status(kl_handle h, cudaStream_t s) {
    int st = 0;
    KL_TRY(host_wait(h, s));
    KL_CUDA(cudaMemcpyAsync(&st, h->dStatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    KL_CUDA(cudaStreamSynchronize(s));
    if (st != 0) {
        KL_CUDA(cudaMemsetAsync(h->dStatus, 0, sizeof(int), s));
        return fail(KL_ERR_TIMEOUT, "a bounded wait in the tensor-core stage-5 kernel gave up");
    }
    return KL_OK;
}

// ---- stages 1-4: u = J . C v  (C = C_d (x) ... (x) C_1) ----------------------------------
template <typename Tc, typename Tout>
static kl_status forward_generic(kl_handle h, const double* v, int64_t ldv, Tout* u, int64_t ldu, int nvec,
                                 Tc* const* Ct, const Tc* J, void* bufA, void* bufB, cudaStream_t s) {
    const int d = h->dim;
    const int64_t ld = stride_of(h);
    // sizes: after processing modes < k the tensor is [n_d..n_{k}][nt_{k-1}..nt_1]
    const void* cur = v;
    int64_t ldcur = ldv;
    bool cur_is_double = true;
    if (sizeof(Tc) == sizeof(float) && d > 0) {
        // float32 arithmetic: round the input to float once (the same rounding the mode pass
        // would apply to every element it reads, n_1 times each) into the buffer mode 0 does not
        // write; mode 0 then runs float to float
        cudaError_t e = launch_to_float(v, ldv, static_cast<float*>(bufB), ld, h->N, nvec, s);
        if (e != cudaSuccess) return cuda_fail(e, "forward contraction");
        cur = bufB;
        ldcur = ld;
        cur_is_double = false;
    }
    for (int k = 0; k < d; ++k) {
        int64_t A = 1, B = 1;
        for (int i = k + 1; i < d; ++i) A *= h->n[i];
        for (int i = 0; i < k; ++i) B *= h->nt[i];
        const bool last = (k == d - 1);
        void* out = last ? static_cast<void*>(u) : ((k % 2 == 0) ? bufA : bufB);
        const int64_t ldo = last ? ldu : ld;
        cudaError_t e;
        const Tc* sc = last ? J : nullptr;
        if (cur_is_double) {
            if (last)
                e = launch_contract<double, Tc, Tout>(static_cast<const double*>(cur), ldcur, static_cast<Tout*>(out), ldo,
                                                      Ct[k], A, h->n[k], h->nt[k], B, nvec, sc, s);
            else
                e = launch_contract<double, Tc, Tc>(static_cast<const double*>(cur), ldcur, static_cast<Tc*>(out), ldo,
                                                    Ct[k], A, h->n[k], h->nt[k], B, nvec, sc, s);
        } else {
            if (last)
                e = launch_contract<Tc, Tc, Tout>(static_cast<const Tc*>(cur), ldcur, static_cast<Tout*>(out), ldo,
                                                  Ct[k], A, h->n[k], h->nt[k], B, nvec, sc, s);
            else
                e = launch_contract<Tc, Tc, Tc>(static_cast<const Tc*>(cur), ldcur, static_cast<Tc*>(out), ldo,
                                                Ct[k], A, h->n[k], h->nt[k], B, nvec, sc, s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "forward contraction");
        cur = out;
        ldcur = ldo;
        cur_is_double = std::is_same<Tc, double>::value;
    }
    return KL_OK;
}

// ---- stages 6-9 (J already applied to z by the stage-5 epilogue): y = C^T z -----------------
template <typename Tc>
static kl_status backward_generic(kl_handle h, const double* z, int64_t ldz, double* y, int64_t ldy, int nvec,
                                  Tc* const* C, void* bufA, void* bufB, cudaStream_t s) {
    const int d = h->dim;
    const int64_t ld = stride_of(h);
    const void* cur = z;
    int64_t ldcur = ldz;
    bool cur_is_double = true;
    for (int k = 0; k < d; ++k) {
        int64_t A = 1, B = 1;
        for (int i = k + 1; i < d; ++i) A *= h->nt[i];
        for (int i = 0; i < k; ++i) B *= h->n[i];
        const bool last = (k == d - 1);
        void* out = last ? static_cast<void*>(y) : ((k % 2 == 0) ? bufA : bufB);
        const int64_t ldo = last ? ldy : ld;
        cudaError_t e;
        if (cur_is_double) {
            if (last)
                e = launch_contract<double, Tc, double>(static_cast<const double*>(cur), ldcur, static_cast<double*>(out), ldo,
                                                        C[k], A, h->nt[k], h->n[k], B, nvec, nullptr, s);
            else
                e = launch_contract<double, Tc, Tc>(static_cast<const double*>(cur), ldcur, static_cast<Tc*>(out), ldo,
                                                    C[k], A, h->nt[k], h->n[k], B, nvec, nullptr, s);
        } else {
            if (last)
                e = launch_contract<Tc, Tc, double>(static_cast<const Tc*>(cur), ldcur, static_cast<double*>(out), ldo,
                                                    C[k], A, h->nt[k], h->n[k], B, nvec, nullptr, s);
            else
                e = launch_contract<Tc, Tc, Tc>(static_cast<const Tc*>(cur), ldcur, static_cast<Tc*>(out), ldo,
                                                C[k], A, h->nt[k], h->n[k], B, nvec, nullptr, s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "backward contraction");
        cur = out;
        ldcur = ldo;
        cur_is_double = std::is_same<Tc, double>::value;
    }
    return KL_OK;
}

kl_status forward_impl(kl_handle h, const double* v, int64_t ldv, double* u, int64_t ldu, int nvec,
                       cudaStream_t s) {
    KL_TRY(ensure_apply_ws(h, nvec, false));
    return forward_generic<double, double>(h, v, ldv, u, ldu, nvec, h->dCt, h->dJ, h->w_a.ptr, h->w_b.ptr, s);
}

kl_status covmv_impl(kl_handle h, int precision, const double* u, int64_t ldu, double* z, int64_t ldz,
                     int nvec, bool withJ, cudaStream_t s) {
    KL_TRY(ensure_apply_ws(h, nvec, precision == KL_P_FP32 || precision == KL_P_TC32, precision == KL_P_TC64));
    CovParams cp = cov_params(h);
    const double s2 = h->kernel.sigma * h->kernel.sigma;
    const double* J = withJ ? h->dJ : nullptr;
    cudaError_t e;
    if (precision == KL_P_TC64) {
        e = (tc_symmetric_used(h->Nt) ? launch_covmv_tcs64 : launch_covmv_tc64)(
            cp, u, ldu, nvec, z, ldz, s2, J, static_cast<double*>(h->w_part.ptr), h->w_tcimg.ptr, h->dStatus, s);
        if (e != cudaSuccess) return cuda_fail(e, "stage-5 kernel product (tensor cores, float64 class)");
        return KL_OK;
    }
    if (precision == KL_P_TC32) {
        float* uf = static_cast<float*>(h->w_f32a.ptr);
        const int64_t ld = stride_of(h);
        e = launch_to_float(u, ldu, uf, ld, h->Nt, nvec, s);
        if (e == cudaSuccess)
            e = launch_covmv_tc(cp, uf, ld, nvec, z, ldz, s2, J, static_cast<double*>(h->w_part.ptr),
                                h->w_tcimg.ptr, h->dStatus, s);
        if (e != cudaSuccess) return cuda_fail(e, "stage-5 kernel product (tensor cores)");
        return KL_OK;
    }
    if (precision == KL_P_FP64) {
        e = launch_covmv64_sym(cp, u, ldu, nvec, z, ldz, s2, J, static_cast<double*>(h->w_part.ptr),
                           covmv_splits(h->Nt, nvec, false), s);
    } else if (precision == KL_P_DF64) {
        e = launch_covmv_df(cp, u, ldu, nvec, z, ldz, s2, J, static_cast<double*>(h->w_part.ptr),
                            covmv_df_splits(h->Nt), s);
    } else {
        float* uf = static_cast<float*>(h->w_f32a.ptr);
        const int64_t ld = stride_of(h);
        e = launch_to_float(u, ldu, uf, ld, h->Nt, nvec, s);
        if (e == cudaSuccess)
            e = launch_covmv32_sym(cp, uf, ld, nvec, z, ldz, s2, J, static_cast<double*>(h->w_part.ptr),
                               covmv_splits(h->Nt, nvec, true), s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "stage-5 kernel product");
    return KL_OK;
}

kl_status backward_impl(kl_handle h, const double* z, int64_t ldz, double* y, int64_t ldy, int nvec,
                        bool zHasJ, cudaStream_t s) {
    KL_TRY(ensure_apply_ws(h, nvec, false));
    if (!zHasJ) {
        // stage 6 on its own: w = J . z into the second buffer (first buffer is the mode-1 output)
        double* tmp = static_cast<double*>(h->w_b.ptr);
        const int64_t ld = stride_of(h);
        // J . z as a 1 x 1 "contraction" with factor 1.0 (table entry 2^0) and scale J
        cudaError_t e = launch_contract<double, double, double>(z, ldz, tmp, ld, h->dTab /*entry 0 == 1.0*/, h->Nt, 1, 1,
                                                                1, nvec, h->dJ, s);
        if (e != cudaSuccess) return cuda_fail(e, "stage 6 scaling");
        // the mode passes read tmp once, so it can serve as the second ping-pong buffer
        return backward_generic<double>(h, tmp, ld, y, ldy, nvec, h->dC, h->w_a.ptr, tmp, s);
    }
    return backward_generic<double>(h, z, ldz, y, ldy, nvec, h->dC, h->w_a.ptr, h->w_b.ptr, s);
}

// Stage-5 event timing: while kl_eigs runs, every stage-5 launch group is bracketed by a
// pair of CUDA events on the launching stream; the pairs are read once the solve is done.
static kl_status prof_begin(kl_handle h, int kind, int nvec, cudaStream_t s, int* slot) {
    *slot = -1;
    if (!h->prof_on) return KL_OK;
    const int need = int(h->prof_rec.size()) * 2 + 2;
    while (int(h->prof_ev.size()) < need) {
        cudaEvent_t ev;
        KL_CUDA(cudaEventCreate(&ev));
        h->prof_ev.push_back(ev);
    }
    *slot = int(h->prof_rec.size()) * 2;
    h->prof_rec.push_back({*slot, kind, nvec});
    KL_CUDA(cudaEventRecord(h->prof_ev[*slot], s));
    return KL_OK;
}

static kl_status prof_end(kl_handle h, int slot, cudaStream_t s) {
    if (slot < 0) return KL_OK;
    KL_CUDA(cudaEventRecord(h->prof_ev[slot + 1], s));
    return KL_OK;
}

// stages 1-4 of an application in the workspace of `precision`: u (double, or float for the
// float32 paths) and the stage-5 output z (double)
kl_status apply_forward(kl_handle h, int precision, const double* v, int64_t ldv, int nvec, cudaStream_t s,
                        ApplyBufs* b) {
    const bool fp32 = (precision == KL_P_FP32 || precision == KL_P_TC32);
    KL_TRY(ensure_apply_ws(h, nvec, fp32, precision == KL_P_TC64));
    const int64_t ld = stride_of(h);
    double* A = static_cast<double*>(h->w_a.ptr);
    double* B = static_cast<double*>(h->w_b.ptr);
    b->ld = ld;
    if (!fp32) {
        // the mode passes ping-pong through A/B and end in `u`
        double* u = (h->dim % 2 == 1) ? A : B;
        KL_TRY(forward_generic<double, double>(h, v, ldv, u, ld, nvec, h->dCt, h->dJ, A, B, s));
        b->u = u;
        b->z = (u == A) ? B : A;
        return KL_OK;
    }
    float* FA = static_cast<float*>(h->w_f32a.ptr);
    float* FB = static_cast<float*>(h->w_f32b.ptr);
    float* u = (h->dim % 2 == 1) ? FA : FB;
    KL_TRY(forward_generic<float, float>(h, v, ldv, u, ld, nvec, h->fCt, h->fJ, FA, FB, s));
    b->u = u;
    b->z = A;
    return KL_OK;
}

// stages 6-9 from z (J already applied by stage 5)
kl_status apply_backward(kl_handle h, int precision, const ApplyBufs& b, double* y, int64_t ldy, int nvec,
                         cudaStream_t s) {
    const bool fp32 = (precision == KL_P_FP32 || precision == KL_P_TC32);
    double* A = static_cast<double*>(h->w_a.ptr);
    double* B = static_cast<double*>(h->w_b.ptr);
    if (!fp32) {
        double* other = (b.z == A) ? B : A;
        // mode 1 reads z into `other`; z is then free to serve as the second buffer
        return backward_generic<double>(h, b.z, b.ld, y, ldy, nvec, h->dC, other, b.z, s);
    }
    return backward_generic<float>(h, b.z, b.ld, y, ldy, nvec, h->fC, static_cast<float*>(h->w_f32a.ptr),
                                   static_cast<float*>(h->w_f32b.ptr), s);
}

kl_status apply_impl(kl_handle h, int precision, const double* v, int64_t ldv, double* y, int64_t ldy, int nvec,
                     cudaStream_t s) {
    if (nvec == 0) return KL_OK;
    ApplyBufs b;
    KL_TRY(apply_forward(h, precision, v, ldv, nvec, s, &b));
    const int64_t ld = b.ld;
    CovParams cp = cov_params(h);
    const double s2 = h->kernel.sigma * h->kernel.sigma;
    double* part = static_cast<double*>(h->w_part.ptr);
    int slot;
    const bool fp32 = (precision == KL_P_FP32 || precision == KL_P_TC32);
    KL_TRY(prof_begin(h, precision, nvec, s, &slot));
    if (h->batch && (precision == KL_P_FP32 || precision == KL_P_DF64)) {
        // many instances solved together: stage 5 joins the other instances' requests
        KL_TRY(batch_stage5(h, precision, b.u, ld, b.z, ld, nvec, true, s));
    } else {
        const double* u64 = static_cast<const double*>(b.u);
        const float* u32 = static_cast<const float*>(b.u);
        cudaError_t e;
        switch (precision) {
            case KL_P_DF64:
                e = launch_covmv_df(cp, u64, ld, nvec, b.z, ld, s2, h->dJ, part, covmv_df_splits(h->Nt), s);
                break;
            case KL_P_TC64:
                e = (tc_symmetric_used(h->Nt) ? launch_covmv_tcs64 : launch_covmv_tc64)(
                    cp, u64, ld, nvec, b.z, ld, s2, h->dJ, part, h->w_tcimg.ptr, h->dStatus, s);
                break;
            case KL_P_TC32:
                e = launch_covmv_tc(cp, u32, ld, nvec, b.z, ld, s2, h->dJ, part, h->w_tcimg.ptr, h->dStatus, s);
                break;
            case KL_P_FP32:
                e = launch_covmv32_sym(cp, u32, ld, nvec, b.z, ld, s2, h->dJ, part, covmv_splits(h->Nt, nvec, true), s);
                break;
            default:
                e = launch_covmv64_sym(cp, u64, ld, nvec, b.z, ld, s2, h->dJ, part, covmv_splits(h->Nt, nvec, false), s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "stage-5 kernel product");
    }
    KL_TRY(prof_end(h, slot, s));
    return apply_backward(h, precision, b, y, ldy, nvec, s);
}

}  // namespace kl

using namespace kl;

extern "C" {

kl_status kl_create(const kl_geometry* geom, const kl_space* space, const kl_kernel* kernel, kl_handle* out) {
    if (!geom || !space || !kernel || !out) return fail(KL_ERR_INVALID_ARG, "null argument to kl_create");
    *out = nullptr;
    const int d = geom->dim;
    if (d < 1 || d > 3) return fail(KL_ERR_INVALID_ARG, "dim must be 1, 2 or 3");
    if (geom->kind != KL_GEOM_BOX && geom->kind != KL_GEOM_NURBS) return fail(KL_ERR_INVALID_ARG, "unsupported geometry kind");
    if (kernel->kind < KL_K_EXP || kernel->kind > KL_K_POLY_TEST) return fail(KL_ERR_INVALID_ARG, "unknown kernel kind");
    if (!(kernel->sigma > 0.0) || !(kernel->L > 0.0) || !isfinite(kernel->sigma) || !isfinite(kernel->L))
        return fail(KL_ERR_INVALID_ARG, "sigma and L must be positive and finite");
    if (kernel->kind == KL_K_POLY_TEST && (kernel->L < 1.0 || kernel->L > 8.0))
        return fail(KL_ERR_INVALID_ARG, "polynomial test kernel needs 1 <= m = L <= 8");
    NurbsMap nm;
    KL_TRY(parse_geometry(geom, &nm));

    kl_handle h = new (std::nothrow) kl_handle_s();
    if (!h) return fail(KL_ERR_OOM, "host allocation failed");
    h->dim = d;
    h->kernel = *kernel;
    h->N = 1;
    h->Nt = 1;
    {
        const kl_status st = build_space(d, space, h->dir);
        if (st != KL_OK) {
            delete h;
            return st;
        }
    }
    for (int k = 0; k < d; ++k) {
        h->n[k] = h->dir[k].n;
        h->nt[k] = h->dir[k].nt;
        h->N *= h->n[k];
        h->Nt *= h->nt[k];
        if (geom->kind == KL_GEOM_BOX) {
            h->lo[k] = geom->lo[k];
            h->hi[k] = geom->hi[k];
        }
    }
    if (h->Nt > 2147483647LL || h->N > 2147483647LL) {
        delete h;
        return fail(KL_ERR_INVALID_ARG, "problem too large (more than 2^31-1 points)");
    }
    // largest intermediate tensor of the forward (n -> n~) and backward (n~ -> n) mode passes
    h->ldw = h->N > h->Nt ? h->N : h->Nt;
    for (int k = 0; k < d; ++k) {
        int64_t f = 1, b = 1;
        for (int i = 0; i < d; ++i) {
            f *= (i <= k) ? h->nt[i] : h->n[i];
            b *= (i <= k) ? h->n[i] : h->nt[i];
        }
        if (f > h->ldw) h->ldw = f;
        if (b > h->ldw) h->ldw = b;
    }
    {
        // mapped Greville points X = F(xh) in vec order (direction 1 fastest) and J = sqrt(det DF)
        const kl_status st = map_greville_points(geom, nm, h->dir, &h->X_host, &h->J_host);
        if (st != KL_OK) {
            delete h;
            return st;
        }
    }
    const int64_t Nt = h->Nt;
    // device copies: coordinates scaled per kernel kind
    const int kind = kernel->kind;
    const double L = kernel->L;
    const double log2e = 1.4426950408889634;
    double s64 = 1.0, s32 = 1.0;
    if (kind == KL_K_EXP || kind == KL_K_EXP_SEPARABLE) {
        s64 = 1.0 / L;
        s32 = log2e / L;
    } else if (kind == KL_K_GAUSS) {
        s64 = 1.0 / L;
        s32 = sqrt(log2e) / L;
    }
    // power of two bounding |Gamma| for the slicing of the tensor-core float64-class path:
    // |prod_d (1 + x_d x'_d)^m| <= prod_d (1 + max x_d^2)^m; the other kernels are <= 1
    h->gscale = 1.f;
    if (kind == KL_K_POLY_TEST) {
        double bound = 1.0;
        for (int c = 0; c < 3; ++c) {
            double mx = 0.0;
            for (int64_t i = 0; i < Nt; ++i) mx = fmax(mx, fabs(h->X_host[size_t(i) * 3 + c]));
            bound *= pow(1.0 + mx * mx, double(int(L)));
        }
        int e = 0;
        frexp(bound, &e);
        h->gscale = float(ldexp(1.0, -e));
    }
    std::vector<double> P(size_t(Nt) * 3);
    std::vector<float> Pf(size_t(Nt) * 3);
    for (int c = 0; c < 3; ++c)
        for (int64_t i = 0; i < Nt; ++i) {
            const double x = h->X_host[size_t(i) * 3 + c];
            P[size_t(c) * Nt + i] = x * s64;
            Pf[size_t(c) * Nt + i] = float(x * s32);
        }
    // double-float coordinates in grid form: heads on the grid q = 2^(E-23), where every scaled
    // coordinate is below 2^E in magnitude, tails the float remainders (|tail| <= q/2).  Head
    // differences are then exact, which the kernels' point differences rely on.  The
    // stationary kernels see differences only, so their points are first centred on the
    // bounding box (one more bit for domains away from the origin).
    double ctr[3] = {0.0, 0.0, 0.0};
    if (kind != KL_K_POLY_TEST && Nt > 0)
        for (int c = 0; c < 3; ++c) {
            const auto b = P.begin() + ptrdiff_t(c) * Nt;
            const auto mm = std::minmax_element(b, b + Nt);
            ctr[c] = 0.5 * (*mm.first + *mm.second);
        }
    double pmax = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int64_t i = 0; i < Nt; ++i) pmax = fmax(pmax, fabs(P[size_t(c) * Nt + i] - ctr[c]));
    int pe = 0;
    if (pmax > 0.0) frexp(pmax, &pe);
    const double q = ldexp(1.0, pe - 23);
    std::vector<float> Pdf(size_t(Nt) * 6);
    for (int c = 0; c < 3; ++c)
        for (int64_t i = 0; i < Nt; ++i) {
            const double x = P[size_t(c) * Nt + i] - ctr[c];
            const double xh = rint(x / q) * q;   // at most 2^23 grid steps: exact in float
            Pdf[size_t(c) * Nt + i] = float(xh);
            Pdf[size_t(3 + c) * Nt + i] = float(x - xh);
        }
    std::vector<float> tabdf(128);
    for (int j = 0; j < 64; ++j) {
        const double t = exp2(-double(j) / 64.0);
        tabdf[j] = float(t);
        tabdf[64 + j] = float(t - double(tabdf[j]));
    }
    const std::vector<double>& J = h->J_host;
    std::vector<float> Jf(static_cast<size_t>(Nt));
    for (int64_t i = 0; i < Nt; ++i) Jf[size_t(i)] = float(J[size_t(i)]);
    std::vector<double> tab(1024);   // 2^(j/1024) for the float64 exponential (Tang's method)
    for (int j = 0; j < 1024; ++j) tab[j] = exp2(double(j) / 1024.0);

    kl_status st = KL_OK;
    auto chk = [&](kl_status s2) {
        if (st == KL_OK) st = s2;
    };
    chk(upload(&h->dP, P.data(), P.size()));
    chk(upload(&h->fP, Pf.data(), Pf.size()));
    chk(upload(&h->dJ, J.data(), J.size()));
    chk(upload(&h->fJ, Jf.data(), Jf.size()));
    chk(upload(&h->dTab, tab.data(), tab.size()));
    chk(upload(&h->dfP, Pdf.data(), Pdf.size()));
    chk(upload(&h->dfTab, tabdf.data(), tabdf.size()));
    const int zero = 0;
    chk(upload(&h->dStatus, &zero, 1));
    for (int k = 0; k < d && st == KL_OK; ++k) {
        const Direction& D = h->dir[k];
        const int n = D.n, nt = D.nt;
        // forward factor C_k (nt x n); the contraction kernel wants Ct[j * m + i] = C[i][j]
        std::vector<double> Ct(size_t(n) * nt), Cb(size_t(nt) * n);
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < n; ++j) {
                Ct[size_t(j) * nt + i] = D.C[size_t(i) * n + j];
                // backward factor C_k^T (n x nt): layout Ct'[jj * n + ii] = C^T[ii][jj] = C[jj][ii]
                Cb[size_t(i) * n + j] = D.C[size_t(i) * n + j];
            }
        std::vector<float> Ctf(Ct.begin(), Ct.end()), Cbf(Cb.begin(), Cb.end());
        chk(upload(&h->dCt[k], Ct.data(), Ct.size()));
        chk(upload(&h->dC[k], Cb.data(), Cb.size()));
        chk(upload(&h->fCt[k], Ctf.data(), Ctf.size()));
        chk(upload(&h->fC[k], Cbf.data(), Cbf.size()));
        // L_k^{-T} as a contraction factor: out[i] = sum_j (L^{-T})[i][j] in[j];  layout [j*n + i] = Linv[j][i]
        std::vector<double> LT(size_t(n) * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) LT[size_t(j) * n + i] = D.Linv[size_t(j) * n + i];
        chk(upload(&h->dLinvT[k], LT.data(), LT.size()));
    }
    if (st == KL_OK) st = ensure_apply_ws(h, 1, true);
    if (st != KL_OK) {
        kl_destroy(h);
        return st;
    }
    *out = h;
    return KL_OK;
}

kl_status kl_size(kl_handle h, int64_t* N, int64_t* Ntilde) {
    if (!h) return fail(KL_ERR_INVALID_ARG, "null handle");
    if (N) *N = h->N;
    if (Ntilde) *Ntilde = h->Nt;
    return KL_OK;
}

kl_status kl_dims(kl_handle h, int* n, int* ntilde) {
    if (!h) return fail(KL_ERR_INVALID_ARG, "null handle");
    for (int k = 0; k < 3; ++k) {
        if (n) n[k] = h->n[k];
        if (ntilde) ntilde[k] = h->nt[k];
    }
    return KL_OK;
}

kl_status kl_apply_prec(kl_handle h, int precision, const double* v_dev, double* y_dev, int nvec, int64_t ldv,
                        void* stream) {
    KL_TRY(check_block(h, v_dev, y_dev, nvec, ldv, h ? h->N : 0, ldv, h ? h->N : 0));
    if (precision < KL_P_FP64 || precision > KL_P_TC64) return fail(KL_ERR_INVALID_ARG, "unknown precision");
    KL_TRY(apply_impl(h, precision, v_dev, ldv, y_dev, ldv, nvec, static_cast<cudaStream_t>(stream)));
    if (precision == KL_P_TC32 || precision == KL_P_TC64) return check_device_status(h, static_cast<cudaStream_t>(stream));
    return KL_OK;
}

kl_status kl_apply(kl_handle h, const double* v_dev, double* y_dev, int nvec, int64_t ldv, void* stream) {
    return kl_apply_prec(h, KL_P_FP64, v_dev, y_dev, nvec, ldv, stream);
}

kl_status kl_forward(kl_handle h, const double* v_dev, int64_t ldv, double* u_dev, int64_t ldu, int nvec,
                     void* stream) {
    KL_TRY(check_block(h, v_dev, u_dev, nvec, ldv, h ? h->N : 0, ldu, h ? h->Nt : 0));
    if (nvec == 0) return KL_OK;
    return forward_impl(h, v_dev, ldv, u_dev, ldu, nvec, static_cast<cudaStream_t>(stream));
}

kl_status kl_covmv(kl_handle h, int precision, const double* u_dev, int64_t ldu, double* z_dev, int64_t ldz,
                   int nvec, void* stream) {
    KL_TRY(check_block(h, u_dev, z_dev, nvec, ldu, h ? h->Nt : 0, ldz, h ? h->Nt : 0));
    if (precision < KL_P_FP64 || precision > KL_P_TC64) return fail(KL_ERR_INVALID_ARG, "unknown precision");
    if (nvec == 0) return KL_OK;
    KL_TRY(covmv_impl(h, precision, u_dev, ldu, z_dev, ldz, nvec, false, static_cast<cudaStream_t>(stream)));
    if (precision == KL_P_TC32 || precision == KL_P_TC64) return check_device_status(h, static_cast<cudaStream_t>(stream));
    return KL_OK;
}

kl_status kl_backward(kl_handle h, const double* z_dev, int64_t ldz, double* y_dev, int64_t ldy, int nvec,
                      void* stream) {
    KL_TRY(check_block(h, z_dev, y_dev, nvec, ldz, h ? h->Nt : 0, ldy, h ? h->N : 0));
    if (nvec == 0) return KL_OK;
    return backward_impl(h, z_dev, ldz, y_dev, ldy, nvec, false, static_cast<cudaStream_t>(stream));
}

kl_status kl_get_factor(kl_handle h, int k, double* C_host) {
    if (!h) return fail(KL_ERR_INVALID_ARG, "null handle");
    if (k < 0 || k >= h->dim) return fail(KL_ERR_INVALID_ARG, "direction out of range");
    if (C_host) std::memcpy(C_host, h->dir[k].C.data(), h->dir[k].C.size() * sizeof(double));
    return KL_OK;
}

kl_status kl_get_points(kl_handle h, double* X_host, double* J_host) {
    if (!h) return fail(KL_ERR_INVALID_ARG, "null handle");
    if (X_host) std::memcpy(X_host, h->X_host.data(), h->X_host.size() * sizeof(double));
    if (J_host)
        std::memcpy(J_host, h->J_host.data(), h->J_host.size() * sizeof(double));
    return KL_OK;
}

kl_status kl_to_bspline(kl_handle h, const double* vprime_dev, double* v_dev, int nvec, int64_t ld, void* stream) {
    KL_TRY(check_block(h, vprime_dev, v_dev, nvec, ld, h ? h->N : 0, ld, h ? h->N : 0));
    if (nvec == 0) return KL_OK;
    KL_TRY(ensure_apply_ws(h, nvec, false));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int d = h->dim;
    const int64_t lds = stride_of(h);
    const double* cur = vprime_dev;
    int64_t ldcur = ld;
    for (int k = 0; k < d; ++k) {
        int64_t A = 1, B = 1;
        for (int i = k + 1; i < d; ++i) A *= h->n[i];
        for (int i = 0; i < k; ++i) B *= h->n[i];
        const bool last = (k == d - 1);
        double* out = last ? v_dev : static_cast<double*>((k % 2 == 0) ? h->w_a.ptr : h->w_b.ptr);
        cudaError_t e = launch_contract<double, double, double>(cur, ldcur, out, last ? ld : lds, h->dLinvT[k], A,
                                                                h->n[k], h->n[k], B, nvec, nullptr, s);
        if (e != cudaSuccess) return cuda_fail(e, "L^{-T} contraction");
        cur = out;
        ldcur = last ? ld : lds;
    }
    return KL_OK;
}

kl_status kl_eigs(kl_handle h, int k, double tol, const kl_eig_opts* opts, double* evals_host, double* evecs_dev,
                  int64_t ldv, kl_eig_info* info, void* stream) {
    if (!h) return fail(KL_ERR_INVALID_ARG, "null handle");
    if (k < 1 || k > 64 || k >= h->N) return fail(KL_ERR_INVALID_ARG, "need 1 <= k <= 64 and k < N");
    if (!(tol > 0.0)) return fail(KL_ERR_INVALID_ARG, "tol must be positive");
    if (!evals_host) return fail(KL_ERR_INVALID_ARG, "evals_host is NULL");
    if (evecs_dev && ldv < h->N) return fail(KL_ERR_INVALID_ARG, "ldv < N");
    return eigs_impl(h, k, tol, opts, evals_host, evecs_dev, ldv, info, static_cast<cudaStream_t>(stream));
}

uint64_t kl_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* kl_last_error(void) { return g_last_error.c_str(); }

void kl_destroy(kl_handle h) {
    if (!h) return;
    for (int k = 0; k < 3; ++k) {
        if (h->dCt[k]) cudaFree(h->dCt[k]);
        if (h->dC[k]) cudaFree(h->dC[k]);
        if (h->fCt[k]) cudaFree(h->fCt[k]);
        if (h->fC[k]) cudaFree(h->fC[k]);
        if (h->dLinvT[k]) cudaFree(h->dLinvT[k]);
    }
    if (h->dP) cudaFree(h->dP);
    if (h->fP) cudaFree(h->fP);
    if (h->dJ) cudaFree(h->dJ);
    if (h->fJ) cudaFree(h->fJ);
    if (h->dTab) cudaFree(h->dTab);
    if (h->dfP) cudaFree(h->dfP);
    if (h->dfTab) cudaFree(h->dfTab);
    if (h->dStatus) cudaFree(h->dStatus);
    release(h->w_a);
    release(h->w_b);
    release(h->w_f32a);
    release(h->w_f32b);
    release(h->w_part);
    release(h->w_tcimg);
    if (h->batch_ready) cudaEventDestroy(h->batch_ready);
    if (h->host_sync) cudaEventDestroy(h->host_sync);
    for (cudaEvent_t ev : h->prof_ev) cudaEventDestroy(ev);
    delete h;
}

}  // extern "C"

extern "C" kl_status kl_set_sym_slot_limit(int64_t bytes) {
    if (bytes < 0) return fail(KL_ERR_INVALID_ARG, "kl_set_sym_slot_limit: negative byte count");
    set_sym_slot_limit(bytes);
    return KL_OK;
}

extern "C" kl_status kl_set_tc_symmetric(int enable) {
    set_tc_symmetric(enable != 0);
    return KL_OK;
}
