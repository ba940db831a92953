// ecc_selftest.cu -- makes the library's bounded device waits run out.
#include <cuda_runtime.h>

#include "ecc.h"
#include "ecc_internal.h"
#include "ecc_sync.cuh"

namespace ecc {
namespace {

// One warp: lane 0 spins on a global flag that nothing sets (the scan's
// look-back pattern), then waits on an mbarrier that nothing arrives on
// (the TMA ring's pattern); each gives up after limit_ns and records
// DEV_TIMEOUT.  out[0], out[1] = 1 when the respective wait gave up.
__global__ void wait_timeout_kernel(volatile int *flag, unsigned int *status, int *out,
                                    unsigned long long limit_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        sync::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        const int f = sync::flag_wait(flag, limit_ns);
        out[0] = f == 0;
        if (f == 0) atomicOr(status, DEV_TIMEOUT);
        const bool done = sync::mbar_wait(&bar, 0, limit_ns);
        out[1] = !done;
        if (!done) atomicOr(status, DEV_TIMEOUT);
    }
}

}  // namespace
}  // namespace ecc

using namespace ecc;

extern "C" ecc_status ecc_selftest_wait_timeout(int64_t limit_us, int32_t *gave_up, void *stream)
{
    if (limit_us < 1 || limit_us > 10 * 1000 * 1000 || !gave_up) {
        set_error("ecc_selftest_wait_timeout: limit_us must be in [1, 1e7] and gave_up non-NULL");
        return ECC_E_INVALID;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 4 * sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "ecc_selftest_wait_timeout: allocation");
    int h[4] = {0, 0, 0, 0};
    e = cudaMemsetAsync(d, 0, 4 * sizeof(int), s);
    if (e == cudaSuccess) {
        // d[0]: the flag nothing sets; d[1]: status word; d[2..3]: results
        wait_timeout_kernel<<<1, 32, 0, s>>>(d, reinterpret_cast<unsigned int *>(d + 1), d + 2,
                                             (unsigned long long)limit_us * 1000ull);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "ecc_selftest_wait_timeout");
    gave_up[0] = h[2];
    gave_up[1] = h[3];
    if (h[1] & DEV_TIMEOUT) {
        set_error("a bounded device-side wait gave up (as intended by the self-test)");
        return ECC_E_TIMEOUT;
    }
    return ECC_OK;
}
