// Building blocks shared by the tensor-core stage-5 kernels (tcgen05, sm_103a): shared-memory
// operand descriptors, MMA issue and commit, bounded mbarrier waits, bulk copies, and the
// persistent tile-range schedule.
#pragma once

#include <cstdint>

#include "kl_internal.h"

namespace kl {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row r, column k) inside a K-major, no-swizzle operand tile made of
// 16-column sub-tiles of sub_bytes each: core matrices of 8 rows x 16 bytes, 128 bytes between
// the two 8-column halves, 256 bytes between 8-row groups
__device__ __forceinline__ int kmajor_offset(int r, int k, int sub_bytes) {
    const int t = k >> 4, kk = k & 15;
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

// instruction descriptor, kind::f16: D float32, A and B bfloat16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// D (tensor memory) [+]= A B, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// the same with the descriptors given as low / high 32-bit words (the low word carries the start
// address, so per-MMA offsets are one 32-bit add)
__device__ __forceinline__ void mma_bf16_lo(uint32_t tmem_d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                            uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\t"
        "mov.b64 da, {%1, %2};\n\t"
        "mov.b64 db, {%3, %4};\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n\t}\n"
        :
        : "r"(tmem_d), "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive once on `bar` when every earlier tcgen05 operation of this thread has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

// the thread may sleep in the try_wait until the phase completes (at most ~0.1 ms per try)
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity; false after max_clocks SM clocks
// (default ~2 s at 2 GHz)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long max_clocks = 4000000000ll) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > max_clocks) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

// one bulk global -> shared copy whose completion is counted in bytes on `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// announce `bytes` of bulk copies on `bar` (one arrival), for copies issued with bulk_copy_tx
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// a bulk global -> shared copy counted on `bar` without an arrival of its own
__device__ __forceinline__ void bulk_copy_tx(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot_saddr, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot_saddr), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// generic-proxy shared-memory writes become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// 8 consecutive float32 accumulator columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* out) {
    uint32_t d[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = __uint_as_float(d[i]);
}

// the same without the wait: several loads in flight, then one tmem_ld_wait
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* d) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// tile range of CTA b when T tiles are cut into G contiguous ranges
__host__ __device__ __forceinline__ int64_t tile_begin(int64_t b, int64_t T, int64_t G) { return b * T / G; }

// Persistent schedule: tiles are (row block of 128, column chunk) pairs in row-block order,
// T = row blocks x len (len = column chunks), G CTAs with contiguous tile ranges; maxseg is the
// most row blocks one range touches.
struct Schedule {
    int64_t len = 0, T = 0, G = 0;
    int maxseg = 0;
};

inline cudaError_t make_schedule(int64_t Nt, int rows, int chunk, int ctas_per_sm, Schedule* sc) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    sc->len = (Nt + chunk - 1) / chunk;
    sc->T = ((Nt + rows - 1) / rows) * sc->len;
    sc->G = int64_t(sms) * ctas_per_sm;
    if (sc->G > sc->T) sc->G = sc->T;
    if (sc->G < 1) sc->G = 1;
    int64_t mx = 0;
    for (int64_t b = 0; b < sc->G; ++b) {
        const int64_t a = tile_begin(b, sc->T, sc->G), z = tile_begin(b + 1, sc->T, sc->G) - 1;
        const int64_t n = z / sc->len - a / sc->len + 1;
        if (n > mx) mx = n;
    }
    sc->maxseg = int(mx);
    return cudaSuccess;
}

// z[v][r] = scale2 * J[r] * (sum of the partial slots of r's row block, CTAs in increasing
// order); slot (b, seg) holds [nb][rows] doubles
template <int ROWS, int NB>
__global__ void slot_reduce(const double* __restrict__ part, int64_t Nt, int nv, int64_t len, int64_t T, int64_t G,
                            int maxseg, double* __restrict__ Z, int64_t ldz, double scale2,
                            const double* __restrict__ J) {
    const int64_t total = Nt * nv;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t v = idx / Nt, r = idx - v * Nt;
        const int64_t rb = r / ROWS, rl = r - rb * ROWS;
        const int64_t tlo = rb * len, thi = tlo + len - 1;
        // CTA owning tile t: the largest b with tile_begin(b) <= t
        const int64_t blo = ((tlo + 1) * G - 1) / T, bhi = ((thi + 1) * G - 1) / T;
        double s = 0.0;
        for (int64_t b = blo; b <= bhi; ++b) {
            const int64_t seg = rb - tile_begin(b, T, G) / len;
            s += part[((b * maxseg + seg) * NB + v) * ROWS + rl];
        }
        s *= scale2;
        if (J) s *= J[r];
        Z[v * ldz + r] = s;
    }
}

}  // namespace tc
}  // namespace kl
