// Stage 5 of Algorithm 1 for many independent problems (instances of different sizes, kernels
// and geometries) in one persistent launch, and the rendezvous that lets per-instance
// eigensolver threads share that launch.
//
// Work decomposition.  Every request (instance, u block) is cut into items of 128 rows x one
// column range ("split"); items of all requests are numbered consecutively and a persistent
// grid of resident CTAs takes them from a global counter (atomicAdd: no spinning, no
// waiting), so uneven instances balance dynamically.  The kernel kind is read per item
// (CTA-uniform switch).  Each item writes its partial row sums to the request's slot region;
// one reduction launch combines the splits of every request in a fixed order (deterministic)
// and applies sigma^2 and J.  The request table and its header live in device memory, so the
// launch sequence (counter reset, kernel, reduction) is captured once into a CUDA graph per
// configuration and replayed with fixed parameters; only the table is uploaded per batch.
// The column split is chosen by timing candidate sizes on the first batch of a context.
//
// Arithmetic per precision is that of the single-instance kernels: KL_P_FP32 (float32
// kernel values, float32 sums over a split) and KL_P_DF64 (double-float values and sums).
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "df64.cuh"
#include "kernel32.cuh"
#include "kl_internal.h"

namespace kl {

struct BatchReq {
    CovParams cp;
    const void* U;       // float (KL_P_FP32) or double (KL_P_DF64), column-major, ldu
    int64_t ldu;
    double* Z;
    int64_t ldz;
    const double* J;     // null: no J factor
    double scale2;
    int nv;
    int64_t item_begin;  // first work item of this request
    int64_t splits;      // column ranges
    int64_t cps;         // columns per range
    int64_t part_off;    // doubles: splits x nv x Nt partial sums
    int64_t out_begin;   // first flat output index of this request in the reduction
};

struct BatchHdr {
    int nreq;
    int pad;
    int64_t total_items;
    int64_t total_out;
};

namespace {

constexpr int kBRows = 128;   // threads per CTA; rows per double-float item (one a thread)
// rows a thread of a float32 item: two (rows t and t + 128) up to 16 vectors, so that each
// shared-memory read of a column serves two kernel evaluations; one for wider groups, whose
// packed sums would need twice the registers
constexpr int rows_f32(int nv) { return nv <= 16 ? 2 : 1; }
// rows of one work item
inline int item_rows(int prec, int nv) { return prec == KL_P_FP32 ? kBRows * rows_f32(nv) : kBRows; }
constexpr int kBTile = 128;   // column tile staged in shared memory

__device__ __forceinline__ int find_req_item(const BatchReq* reqs, int nreq, int64_t item) {
    int lo = 0, hi = nreq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_req_out(const BatchReq* reqs, int nreq, int64_t idx) {
    int lo = 0, hi = nreq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].out_begin <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- double-float items
template <int KIND, int NV>
__device__ void df_item(const BatchReq& q, int64_t rb, int64_t sp, double* __restrict__ part, float (*sp6)[kBTile],
                        float2 (*su)[NV], const float* stab) {
    const CovParams& cp = q.cp;
    const int64_t Nt = cp.Nt;
    const double* U = static_cast<const double*>(q.U);
    const int64_t row = rb * kBRows + threadIdx.x;
    const bool valid = row < Nt;
    float rp[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) rp[k] = valid ? cp.Pdf[k * cp.ldp + row] : 0.f;
    const int64_t c_begin = sp * q.cps;
    int64_t c_end = c_begin + q.cps;
    if (c_end > Nt) c_end = Nt;
    float ah[NV], al[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        ah[v] = 0.f;
        al[v] = 0.f;
    }
    for (int64_t c0 = c_begin; c0 < c_end; c0 += kBTile) {
        __syncthreads();
        const int64_t c = c0 + threadIdx.x;
        const bool cv = c < c_end;
#pragma unroll
        for (int k = 0; k < 6; ++k) sp6[k][threadIdx.x] = cv ? cp.Pdf[k * cp.ldp + c] : 0.f;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const double u = (cv && v < q.nv) ? U[v * q.ldu + c] : 0.0;
            const float uh = __double2float_rn(u);
            su[threadIdx.x][v] = make_float2(uh, __double2float_rn(u - double(uh)));
        }
        __syncthreads();
        const int jmax = int(c_end - c0 < kBTile ? c_end - c0 : kBTile);
#pragma unroll 1
        for (int j = 0; j < jmax; ++j) {
            float cpj[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) cpj[k] = sp6[k][j];
            const df::F2 g = df::kernel_df<KIND>(rp, cpj, cp.poly_m, stab, stab + 64);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float2 u = su[j][v];
                const float ph = df::mul(g.h, u.x);
                float pe = df::fma_(g.h, u.x, -ph);
                pe = df::fma_(g.h, u.y, pe);
                pe = df::fma_(g.l, u.x, pe);
                const df::F2 s = df::two_sum(ah[v], ph);
                ah[v] = s.h;
                al[v] = df::add(al[v], df::add(s.l, pe));
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const df::F2 r = df::fast_two_sum(ah[v], al[v]);
            ah[v] = r.h;
            al[v] = r.l;
        }
    }
    if (valid) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
            if (v < q.nv) part[q.part_off + (sp * q.nv + v) * Nt + row] = double(ah[v]) + double(al[v]);
    }
}

template <int NV>
__global__ void __launch_bounds__(kBRows)
batch_df_kernel(const BatchHdr* __restrict__ hdr, const BatchReq* __restrict__ reqs, int* __restrict__ counter,
                double* __restrict__ part) {
    __shared__ float sp6[6][kBTile];
    __shared__ float2 su[kBTile][NV];
    __shared__ float stab[128];
    __shared__ long long s_item;
    const int nreq = hdr->nreq;
    const int64_t total = hdr->total_items;
    if (nreq <= 0) return;
    stab[threadIdx.x] = reqs[0].cp.tabdf[threadIdx.x];   // the 2^(-j/64) table is the same for all
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const BatchReq& q = reqs[find_req_item(reqs, nreq, item)];
        const int64_t local = item - q.item_begin;
        const int64_t rb = local / q.splits, sp = local - rb * q.splits;
        switch (q.cp.kind) {
            case KL_K_EXP: df_item<KL_K_EXP, NV>(q, rb, sp, part, sp6, su, stab); break;
            case KL_K_GAUSS: df_item<KL_K_GAUSS, NV>(q, rb, sp, part, sp6, su, stab); break;
            case KL_K_EXP_SEPARABLE: df_item<KL_K_EXP_SEPARABLE, NV>(q, rb, sp, part, sp6, su, stab); break;
            default: df_item<KL_K_POLY_TEST, NV>(q, rb, sp, part, sp6, su, stab); break;
        }
    }
}

// ---------------------------------------------------------------- float32 items
template <int KIND, int NV>
__device__ void f32_item(const BatchReq& q, int64_t rb, int64_t sp, double* __restrict__ part, float4* sp3,
                         float (*su)[NV]) {
    constexpr int ROWS = rows_f32(NV);
    const CovParams& cp = q.cp;
    const int64_t Nt = cp.Nt;
    const float* U = static_cast<const float*>(q.U);
    const float* P = cp.P32;
    int64_t row[ROWS];
    float x0[ROWS], y0[ROWS], z0[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        row[r] = rb * (kBRows * ROWS) + threadIdx.x + r * kBRows;
        const bool valid = row[r] < Nt;
        x0[r] = valid ? P[row[r]] : 0.f;
        y0[r] = valid ? P[cp.ldp + row[r]] : 0.f;
        z0[r] = valid ? P[2 * cp.ldp + row[r]] : 0.f;
    }
    const int64_t c_begin = sp * q.cps;
    int64_t c_end = c_begin + q.cps;
    if (c_end > Nt) c_end = Nt;
    // even widths: the sums of vectors (v, v + 1) in one 64-bit register pair, one packed FMA
    constexpr bool PACK = (NV % 2 == 0);
    float acc[ROWS][PACK ? 1 : NV];
    unsigned long long acc2[ROWS][PACK ? NV / 2 : 1];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
#pragma unroll
        for (int v = 0; v < (PACK ? 1 : NV); ++v) acc[r][v] = 0.f;
#pragma unroll
        for (int w = 0; w < (PACK ? NV / 2 : 1); ++w) acc2[r][w] = 0ull;
    }
    for (int64_t c0 = c_begin; c0 < c_end; c0 += kBTile) {
        __syncthreads();
        const int64_t c = c0 + threadIdx.x;
        const bool cv = c < c_end;
        sp3[threadIdx.x] = cv ? make_float4(P[c], P[cp.ldp + c], P[2 * cp.ldp + c], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int v = 0; v < NV; ++v) su[threadIdx.x][v] = (cv && v < q.nv) ? U[v * q.ldu + c] : 0.f;
        __syncthreads();
        const int jmax = int(c_end - c0 < kBTile ? c_end - c0 : kBTile);
#pragma unroll 4
        for (int j = 0; j < jmax; ++j) {
            const float4 p = sp3[j];
            float g[ROWS];
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
                g[r] = kernel32<KIND>(x0[r] - p.x, y0[r] - p.y, z0[r] - p.z, x0[r], y0[r], z0[r], p.x, p.y, p.z,
                                      cp.poly_m);
            if constexpr (PACK) {
                unsigned long long g2[ROWS];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) g2[r] = f2_dup(g[r]);
#pragma unroll
                for (int w = 0; w < NV / 2; ++w) {
                    const unsigned long long uu = *reinterpret_cast<const unsigned long long*>(&su[j][2 * w]);
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) acc2[r][w] = f2_fma(g2[r], uu, acc2[r][w]);
                }
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const float uu = su[j][v];
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) acc[r][v] = fmaf(g[r], uu, acc[r][v]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        if (row[r] < Nt) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                float a;
                if constexpr (PACK)
                    a = (v & 1) ? f2_hi(acc2[r][v >> 1]) : f2_lo(acc2[r][v >> 1]);
                else
                    a = acc[r][v];
                if (v < q.nv) part[q.part_off + (sp * q.nv + v) * Nt + row[r]] = double(a);
            }
        }
    }
}

template <int NV>
__global__ void __launch_bounds__(kBRows)
batch_f32_kernel(const BatchHdr* __restrict__ hdr, const BatchReq* __restrict__ reqs, int* __restrict__ counter,
                 double* __restrict__ part) {
    __shared__ float4 sp3[kBTile];
    __shared__ __align__(16) float su[kBTile][NV];
    __shared__ long long s_item;
    const int nreq = hdr->nreq;
    const int64_t total = hdr->total_items;
    if (nreq <= 0) return;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const BatchReq& q = reqs[find_req_item(reqs, nreq, item)];
        const int64_t local = item - q.item_begin;
        const int64_t rb = local / q.splits, sp = local - rb * q.splits;
        switch (q.cp.kind) {
            case KL_K_EXP: f32_item<KL_K_EXP, NV>(q, rb, sp, part, sp3, su); break;
            case KL_K_GAUSS: f32_item<KL_K_GAUSS, NV>(q, rb, sp, part, sp3, su); break;
            case KL_K_EXP_SEPARABLE: f32_item<KL_K_EXP_SEPARABLE, NV>(q, rb, sp, part, sp3, su); break;
            default: f32_item<KL_K_POLY_TEST, NV>(q, rb, sp, part, sp3, su); break;
        }
    }
}

// z[v][row] = scale2 * J[row] * sum over splits (fixed order), every request in one launch
__global__ void batch_reduce(const BatchHdr* __restrict__ hdr, const BatchReq* __restrict__ reqs,
                             const double* __restrict__ part) {
    const int nreq = hdr->nreq;
    const int64_t total = hdr->total_out;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const BatchReq& q = reqs[find_req_out(reqs, nreq, idx)];
        const int64_t Nt = q.cp.Nt;
        const int64_t local = idx - q.out_begin;
        const int64_t v = local / Nt, row = local - v * Nt;
        double s = 0.0;
        for (int64_t sp = 0; sp < q.splits; ++sp) s += part[q.part_off + (sp * q.nv + v) * Nt + row];
        s *= q.scale2;
        if (q.J) s *= q.J[row];
        q.Z[v * q.ldz + row] = s;
    }
}

int batch_nv(int nv) { return nv <= 4 ? 4 : nv <= 8 ? 8 : nv <= 12 ? 12 : nv <= 16 ? 16 : 32; }

template <int NV>
cudaError_t occupancy_grid(int prec, int* grid) {
    int per_sm = 0;
    cudaError_t e = (prec == KL_P_DF64)
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_df_kernel<NV>, kBRows, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_f32_kernel<NV>, kBRows, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    *grid = num_sms() * per_sm;
    return cudaSuccess;
}

template <int NV>
cudaError_t launch_items(int prec, int grid, const BatchHdr* hdr, const BatchReq* reqs, int* counter, double* part,
                         cudaStream_t s) {
    if (prec == KL_P_DF64)
        batch_df_kernel<NV><<<grid, kBRows, 0, s>>>(hdr, reqs, counter, part);
    else
        batch_f32_kernel<NV><<<grid, kBRows, 0, s>>>(hdr, reqs, counter, part);
    return cudaGetLastError();
}

}  // namespace

// ----------------------------------------------------------------------------------------
// host side: one batch = a list of requests of the same precision
// ----------------------------------------------------------------------------------------
struct BatchRequest {
    kl_handle h;
    const void* U;
    int64_t ldu;
    double* Z;
    int64_t ldz;
    int nv;
    bool withJ;
};

struct BatchExec {
    // device resources
    DevBuf table, part, counter;
    // pinned staging for the table uploads, a ring so that filling the next table waits only
    // for an upload several batches back
    static constexpr int kRing = 4;
    struct Slot {
        BatchHdr* host = nullptr;      // header followed by the request table
        size_t cap = 0;
        cudaEvent_t uploaded = nullptr;
    } ring[kRing];
    int ring_pos = 0;
    std::map<long long, long long> tuned_cps;          // (prec, NV) -> columns per split
    std::map<long long, cudaGraphExec_t> graphs;       // (prec, NV, cps) -> captured sequence
    int last_cps = 0;
    double last_ms = 0.0;

    void clear_graphs() {
        for (auto& g : graphs) cudaGraphExecDestroy(g.second);
        graphs.clear();
    }
    ~BatchExec() {
        clear_graphs();
        for (Slot& sl : ring) {
            if (sl.uploaded) cudaEventSynchronize(sl.uploaded);
            if (sl.host) cudaFreeHost(sl.host);
            if (sl.uploaded) cudaEventDestroy(sl.uploaded);
        }
        release(table);
        release(part);
        release(counter);
    }
};

namespace {

constexpr int kMaxSplits = 16;

// fill the table for a column split size; returns the partial-sum doubles needed
size_t build_table(const std::vector<BatchRequest>& reqs, int rows_per_item, long long cps_target, BatchHdr* hdr,
                   BatchReq* tbl) {
    int64_t item = 0, out = 0;
    size_t part = 0;
    for (size_t i = 0; i < reqs.size(); ++i) {
        const BatchRequest& r = reqs[i];
        const int64_t Nt = r.h->Nt;
        BatchReq& q = tbl[i];
        std::memset(&q, 0, sizeof(q));
        q.cp = cov_params_of(r.h);
        q.U = r.U;
        q.ldu = r.ldu;
        q.Z = r.Z;
        q.ldz = r.ldz;
        q.J = r.withJ ? r.h->dJ : nullptr;
        q.scale2 = r.h->kernel.sigma * r.h->kernel.sigma;
        q.nv = r.nv;
        int64_t splits = (Nt + cps_target - 1) / cps_target;
        if (splits > kMaxSplits) splits = kMaxSplits;
        if (splits < 1) splits = 1;
        q.cps = (Nt + splits - 1) / splits;
        q.splits = (Nt + q.cps - 1) / q.cps;
        q.item_begin = item;
        q.part_off = int64_t(part);
        q.out_begin = out;
        item += ((Nt + rows_per_item - 1) / rows_per_item) * q.splits;
        part += size_t(q.splits) * size_t(r.nv) * size_t(Nt);
        out += int64_t(r.nv) * Nt;
    }
    hdr->nreq = int(reqs.size());
    hdr->pad = 0;
    hdr->total_items = item;
    hdr->total_out = out;
    return part;
}

template <int NV>
kl_status run_batch_nv(BatchExec& X, const std::vector<BatchRequest>& reqs, int prec, cudaStream_t s,
                       bool may_tune) {
    const size_t nreq = reqs.size();
    const size_t tbl_bytes = sizeof(BatchHdr) + nreq * sizeof(BatchReq);
    KL_TRY(ensure(X.counter, sizeof(int)));
    int grid = 0;
    KL_CUDA(occupancy_grid<NV>(prec, &grid));
    const long long key = (long long)prec * 1000 + NV;

    auto upload_and_run = [&](long long cps, bool use_graph) -> kl_status {
        BatchExec::Slot& sl = X.ring[X.ring_pos];
        X.ring_pos = (X.ring_pos + 1) % BatchExec::kRing;
        if (!sl.uploaded) KL_CUDA(cudaEventCreateWithFlags(&sl.uploaded, cudaEventDisableTiming));
        KL_CUDA(cudaEventSynchronize(sl.uploaded));   // this slot's previous upload has been read
        if (sl.cap < tbl_bytes) {
            if (sl.host) cudaFreeHost(sl.host);
            sl.host = nullptr;
            sl.cap = 0;
            KL_CUDA(cudaMallocHost(reinterpret_cast<void**>(&sl.host), tbl_bytes * 2));
            sl.cap = tbl_bytes * 2;
        }
        BatchReq* tbl = reinterpret_cast<BatchReq*>(sl.host + 1);
        const size_t part_doubles = build_table(reqs, item_rows(prec, NV), cps, sl.host, tbl);
        if (sl.host->total_items > 2147483647LL) return fail(KL_ERR_INVALID_ARG, "batch too large (work items)");
        if (X.part.bytes < part_doubles * sizeof(double) || X.table.bytes < tbl_bytes) {
            KL_CUDA(cudaStreamSynchronize(s));
            X.clear_graphs();
            KL_TRY(ensure(X.part, part_doubles * sizeof(double) + 256));
            KL_TRY(ensure(X.table, 2 * tbl_bytes));
        }
        KL_CUDA(cudaMemcpyAsync(X.table.ptr, sl.host, tbl_bytes, cudaMemcpyHostToDevice, s));
        KL_CUDA(cudaEventRecord(sl.uploaded, s));
        const BatchHdr* hdr = static_cast<const BatchHdr*>(X.table.ptr);
        const BatchReq* dreq = reinterpret_cast<const BatchReq*>(hdr + 1);
        int* counter = static_cast<int*>(X.counter.ptr);
        double* part = static_cast<double*>(X.part.ptr);
        const int rblocks = num_sms() * 8;
        if (!use_graph) {
            KL_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
            KL_CUDA(launch_items<NV>(prec, grid, hdr, dreq, counter, part, s));
            batch_reduce<<<rblocks, 256, 0, s>>>(hdr, dreq, part);
            KL_CUDA(cudaGetLastError());
            count_launches(2);
            return KL_OK;
        }
        const long long gkey = key * 100000000LL + cps;
        auto it = X.graphs.find(gkey);
        if (it == X.graphs.end()) {
            cudaStream_t cs;
            KL_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaMemsetAsync(counter, 0, sizeof(int), cs);
                launch_items<NV>(prec, grid, hdr, dreq, counter, part, cs);
                batch_reduce<<<rblocks, 256, 0, cs>>>(hdr, dreq, part);
                e = cudaStreamEndCapture(cs, &g);
            }
            cudaGraphExec_t ge = nullptr;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) return cuda_fail(e, "batched stage 5: graph capture");
            it = X.graphs.emplace(gkey, ge).first;
        }
        KL_CUDA(cudaGraphLaunch(it->second, s));
        count_launches(2);
        return KL_OK;
    };

    auto tuned = X.tuned_cps.find(key);
    if (tuned == X.tuned_cps.end() && !may_tune) {
        X.last_cps = 2048;   // until a representative batch has been timed
        return upload_and_run(2048, false);
    }
    if (tuned == X.tuned_cps.end()) {
        // time the candidate column splits on this batch (each run computes the full result)
        const long long cand[4] = {1024, 2048, 4096, 8192};
        cudaEvent_t e0, e1;
        KL_CUDA(cudaEventCreate(&e0));
        KL_CUDA(cudaEventCreate(&e1));
        long long best = cand[0];
        float best_ms = 1e30f;
        for (long long c : cand) {
            KL_CUDA(cudaEventRecord(e0, s));
            KL_TRY(upload_and_run(c, false));
            KL_CUDA(cudaEventRecord(e1, s));
            KL_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            KL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        X.tuned_cps[key] = best;
        X.last_cps = int(best);
        X.last_ms = best_ms;
        // the last candidate's result is complete; run the chosen size once more so that the
        // graph for it exists (and the output is that of the chosen configuration)
        return upload_and_run(best, true);
    }
    X.last_cps = int(tuned->second);
    return upload_and_run(tuned->second, true);
}

}  // namespace

kl_status run_batch(BatchExec& X, const std::vector<BatchRequest>& reqs, int prec, cudaStream_t s,
                    bool may_tune = true) {
    if (reqs.empty()) return KL_OK;
    if (prec != KL_P_FP32 && prec != KL_P_DF64) return fail(KL_ERR_INVALID_ARG, "batched stage 5: precision");
    int nv = 0;
    for (const auto& r : reqs) nv = r.nv > nv ? r.nv : nv;
    switch (batch_nv(nv)) {
        case 4: return run_batch_nv<4>(X, reqs, prec, s, may_tune);
        case 8: return run_batch_nv<8>(X, reqs, prec, s, may_tune);
        case 12: return run_batch_nv<12>(X, reqs, prec, s, may_tune);
        case 16: return run_batch_nv<16>(X, reqs, prec, s, may_tune);
        default: return run_batch_nv<32>(X, reqs, prec, s, may_tune);
    }
}

// ----------------------------------------------------------------------------------------
// rendezvous of the per-instance solver threads
// ----------------------------------------------------------------------------------------
// how long a request waits for the other instances before its batch is launched anyway
// (microseconds; KL_BATCH_WINDOW_US overrides it, a negative value waits for every instance)
int batch_window_us() {
    static const int w = [] {
        const char* e = getenv("KL_BATCH_WINDOW_US");
        return e ? atoi(e) : 200;
    }();
    return w;
}

struct BatchRendezvous {
    std::mutex mu;
    std::condition_variable cv;
    int active = 0;
    int participants = 0;
    uint64_t generation = 0;
    kl_status error = KL_OK;
    std::string error_msg;
    struct Pending {
        BatchRequest r;
        int prec;
        cudaEvent_t ready;
    };
    std::vector<Pending> pending;
    cudaStream_t bs = nullptr;
    cudaEvent_t done = nullptr;
    BatchExec exec;
    int rounds = 0;
    long long requests = 0;
    std::vector<cudaEvent_t> tev;   // begin/end of every round on the batch stream

    // called with mu held once every active participant has submitted
    void launch_locked() {
        kl_status st = KL_OK;
        for (const auto& p : pending)
            if (cudaStreamWaitEvent(bs, p.ready, 0) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "batch wait");
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
            cudaEventRecord(e0, bs);
            tev.push_back(e0);
            tev.push_back(e1);
        } else {
            e1 = nullptr;
        }
        for (int prec : {KL_P_FP32, KL_P_DF64}) {
            std::vector<BatchRequest> g;
            for (const auto& p : pending)
                if (p.prec == prec) g.push_back(p.r);
            if (st == KL_OK && !g.empty()) {
                // the column split is timed on a batch holding most instances, not a straggler's
                const bool may_tune = int(g.size()) >= (participants < 8 ? participants : 8);
                st = run_batch(exec, g, prec, bs, may_tune);
                if (st != KL_OK) error_msg = last_error_message();
            }
        }
        if (e1) cudaEventRecord(e1, bs);
        requests += (long long)pending.size();
        if (st == KL_OK && cudaEventRecord(done, bs) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "batch record");
        if (st != KL_OK && error == KL_OK) error = st;
        pending.clear();
        ++rounds;
        ++generation;
        cv.notify_all();
    }
};

kl_status batch_stage5(kl_handle h, int prec, const void* U, int64_t ldu, double* Z, int64_t ldz, int nv,
                       bool withJ, cudaStream_t s) {
    BatchRendezvous* R = h->batch;
    if (!h->batch_ready) KL_CUDA(cudaEventCreateWithFlags(&h->batch_ready, cudaEventDisableTiming));
    KL_CUDA(cudaEventRecord(h->batch_ready, s));
    std::unique_lock<std::mutex> lk(R->mu);
    if (R->error != KL_OK) return fail(R->error, "batched stage 5 failed in another instance: " + R->error_msg);
    R->pending.push_back({BatchRequest{h, U, ldu, Z, ldz, nv, withJ}, prec, h->batch_ready});
    const uint64_t gen = R->generation;
    if (int(R->pending.size()) == R->active) {
        R->launch_locked();
    } else {
        // batching window: launch with every active instance, or with whatever is pending once
        // the window has passed (instances need different numbers of steps; nobody waits for
        // the slowest one)
        const int win = batch_window_us();
        const bool joined = R->cv.wait_for(lk, std::chrono::microseconds(win >= 0 ? win : 600000000),
                                           [&] { return R->generation != gen; });
        if (!joined) R->launch_locked();
    }
    if (R->error != KL_OK) return fail(R->error, "batched stage 5: " + R->error_msg);
    KL_CUDA(cudaStreamWaitEvent(s, R->done, 0));
    return KL_OK;
}

void batch_leave(BatchRendezvous* R) {
    std::unique_lock<std::mutex> lk(R->mu);
    --R->active;
    if (R->active > 0 && int(R->pending.size()) == R->active) R->launch_locked();
}

BatchRendezvous* batch_create(int participants, kl_status* st) {
    BatchRendezvous* R = new (std::nothrow) BatchRendezvous();
    if (!R) {
        *st = fail(KL_ERR_OOM, "host allocation failed");
        return nullptr;
    }
    R->active = participants;
    R->participants = participants;
    if (cudaStreamCreateWithFlags(&R->bs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&R->done, cudaEventDisableTiming) != cudaSuccess) {
        *st = cuda_fail(cudaGetLastError(), "batch stream");
        delete R;
        return nullptr;
    }
    *st = KL_OK;
    return R;
}

void batch_destroy(BatchRendezvous* R, int* rounds, int* cps, double* ms_stage5, long long* requests) {
    if (!R) return;
    if (R->bs) cudaStreamSynchronize(R->bs);
    if (rounds) *rounds = R->rounds;
    if (cps) *cps = R->exec.last_cps;
    if (requests) *requests = R->requests;
    double ms = 0.0;
    for (size_t i = 0; i + 1 < R->tev.size(); i += 2) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, R->tev[i], R->tev[i + 1]) == cudaSuccess) ms += t;
    }
    for (cudaEvent_t e : R->tev) cudaEventDestroy(e);
    if (ms_stage5) *ms_stage5 = ms;
    if (R->done) cudaEventDestroy(R->done);
    if (R->bs) cudaStreamDestroy(R->bs);
    delete R;
}

}  // namespace kl

// ----------------------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------------------
#include <mutex>
#include <thread>

namespace kl {
namespace {

std::mutex g_exec_mu;
std::map<int, BatchExec*> g_exec;   // per device, process lifetime

kl_status check_handles(kl_handle* hs, int count) {
    if (count < 0) return fail(KL_ERR_INVALID_ARG, "count < 0");
    if (count > 0 && !hs) return fail(KL_ERR_INVALID_ARG, "null handle array");
    for (int i = 0; i < count; ++i) {
        if (!hs[i]) return fail(KL_ERR_INVALID_ARG, "null handle in the batch");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(KL_ERR_INVALID_ARG, "a handle appears twice in the batch");
        if (hs[i]->batch) return fail(KL_ERR_INVALID_ARG, "a handle is already part of a running batch");
    }
    return KL_OK;
}

}  // namespace
}  // namespace kl

using namespace kl;

extern "C" {

kl_status kl_apply_batched(kl_handle* handles, int count, int precision, const double* const* v_dev,
                           double* const* y_dev, const int* nvec, const int64_t* ldv, void* stream) {
    KL_TRY(check_handles(handles, count));
    if (precision != KL_P_FP32 && precision != KL_P_DF64)
        return fail(KL_ERR_INVALID_ARG, "batched application supports KL_P_FP32 and KL_P_DF64");
    if (count > 0 && (!v_dev || !y_dev || !nvec)) return fail(KL_ERR_INVALID_ARG, "null argument array");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<ApplyBufs> bufs(static_cast<size_t>(count));
    std::vector<BatchRequest> reqs;
    for (int i = 0; i < count; ++i) {
        kl_handle h = handles[i];
        const int64_t ld = ldv ? ldv[i] : h->N;
        if (nvec[i] < 0 || nvec[i] > 32) return fail(KL_ERR_INVALID_ARG, "batched application: 0 <= nvec <= 32");
        if (nvec[i] == 0) continue;
        if (!v_dev[i] || !y_dev[i] || ld < h->N) return fail(KL_ERR_INVALID_ARG, "vector pointer or leading dimension");
        KL_TRY(apply_forward(h, precision, v_dev[i], ld, nvec[i], s, &bufs[size_t(i)]));
        reqs.push_back(BatchRequest{h, bufs[size_t(i)].u, bufs[size_t(i)].ld, bufs[size_t(i)].z, bufs[size_t(i)].ld,
                                    nvec[i], true});
    }
    {
        int dev = 0;
        KL_CUDA(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(g_exec_mu);
        BatchExec*& X = g_exec[dev];
        if (!X) X = new (std::nothrow) BatchExec();
        if (!X) return fail(KL_ERR_OOM, "host allocation failed");
        // the column split is timed only on batches of at least 8 instances
        KL_TRY(run_batch(*X, reqs, precision, s, count >= 8));
    }
    for (int i = 0; i < count; ++i) {
        if (nvec[i] == 0) continue;
        const int64_t ld = ldv ? ldv[i] : handles[i]->N;
        KL_TRY(apply_backward(handles[i], precision, bufs[size_t(i)], y_dev[i], ld, nvec[i], s));
    }
    return KL_OK;
}

kl_status kl_eigs_batched(kl_handle* handles, int count, int k, double tol, const kl_eig_opts* opts,
                          double* evals_host, double* const* evecs_dev, const int64_t* ldv, kl_eig_info* infos,
                          kl_status* statuses, kl_batch_info* binfo) {
    KL_TRY(check_handles(handles, count));
    if (count > 0 && !evals_host) return fail(KL_ERR_INVALID_ARG, "null evals_host");
    if (count == 0) return KL_OK;
    int dev = 0;
    KL_CUDA(cudaGetDevice(&dev));
    kl_status st = KL_OK;
    BatchRendezvous* R = batch_create(count, &st);
    if (!R) return st;
    for (int i = 0; i < count; ++i) handles[i]->batch = R;
    std::vector<kl_status> res(size_t(count), KL_OK);
    std::vector<std::string> msg(static_cast<size_t>(count));
    const auto t0 = std::chrono::steady_clock::now();
    {
        std::vector<std::thread> th;
        th.reserve(size_t(count));
        for (int i = 0; i < count; ++i) {
            th.emplace_back([&, i] {
                kl_status r = KL_OK;
                cudaStream_t s = nullptr;
                try {
                    if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                        r = cuda_fail(cudaGetLastError(), "instance stream");
                    } else {
                        const int64_t ld = ldv ? ldv[i] : handles[i]->N;
                        r = eigs_impl(handles[i], k, tol, opts, evals_host + size_t(i) * size_t(k),
                                      evecs_dev ? evecs_dev[i] : nullptr, ld, infos ? &infos[i] : nullptr, s);
                    }
                } catch (...) {
                    r = fail(KL_ERR_OOM, "host exception in a batched instance");
                }
                if (r != KL_OK) msg[size_t(i)] = last_error_message();
                res[size_t(i)] = r;
                batch_leave(R);
                if (s) {
                    cudaStreamSynchronize(s);
                    cudaStreamDestroy(s);
                }
            });
        }
        for (auto& t : th) t.join();
    }
    for (int i = 0; i < count; ++i) handles[i]->batch = nullptr;
    int rounds = 0, cps = 0;
    double ms5 = 0.0;
    long long nreq = 0;
    batch_destroy(R, &rounds, &cps, &ms5, &nreq);
    if (binfo) {
        binfo->rounds = rounds;
        binfo->cols_per_split = cps;
        binfo->ms_stage5 = ms5;
        binfo->requests = nreq;
        binfo->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    kl_status first = KL_OK;
    for (int i = 0; i < count; ++i) {
        if (statuses) statuses[i] = res[size_t(i)];
        if (first == KL_OK && res[size_t(i)] != KL_OK) {
            first = res[size_t(i)];
            set_error("instance " + std::to_string(i) + ": " + msg[size_t(i)]);
        }
    }
    return first;
}

}  // extern "C"
