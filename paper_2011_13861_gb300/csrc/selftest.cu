// Self-test of the bounded waits that every tensor-core kernel uses (failure detection without a
// GPU fault): one thread waits on an mbarrier that nothing ever completes, gives up after the
// requested time, records KL_ERR_TIMEOUT in a device status word and returns, so the host sees
// the same error status a stalled pipeline would produce and the context stays usable.
#include "kl_internal.h"
#include "tc_common.cuh"

namespace kl {
namespace {

__global__ void wait_selftest_kernel(long long max_clocks, int* status) {
    using namespace tc;
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);                         // one arrival expected, none ever made
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const bool ok = mbar_wait(b, 0, max_clocks);
    *status = ok ? int(KL_OK) : int(KL_ERR_TIMEOUT);
}

}  // namespace
}  // namespace kl

using namespace kl;

extern "C" kl_status kl_wait_selftest(double seconds, void* stream) {
    if (!(seconds > 0.0) || seconds > 2.0) return fail(KL_ERR_INVALID_ARG, "wait self-test: 0 < seconds <= 2");
    int dev = 0, khz = 0;
    KL_CUDA(cudaGetDevice(&dev));
    KL_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const long long max_clocks = (long long)(seconds * double(khz) * 1e3);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf st;
    KL_TRY(ensure(st, sizeof(int)));
    int h = -1;
    wait_selftest_kernel<<<1, 1, 0, s>>>(max_clocks, static_cast<int*>(st.ptr));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st.ptr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    release(st);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    count_launches(1);
    if (h == int(KL_ERR_TIMEOUT)) return fail(KL_ERR_TIMEOUT, "wait self-test: the bounded wait gave up as intended");
    return fail(KL_ERR_NUMERIC, "wait self-test: an mbarrier nothing arrives at completed");
}
