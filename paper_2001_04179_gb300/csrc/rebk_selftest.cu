// rebk_selftest.cu -- self-test of the bounded device-wide waits (see include/rebk.h).
//
// The persistent kernels never wait without a limit: a device-wide wait that runs
// past its limit records REBK_BARRIER_TIMEOUT and the kernel returns, so the
// context stays usable.  This entry point makes such a wait run out on purpose,
// with the device-wide barrier and split-phase wait of rebk_device.cuh (the ones
// the sparse kernel uses): one CTA waits for a second CTA that was never launched.
// Nothing faults or traps; the waits end by their own limit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rebk.h"
#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {
namespace {

// out[0], out[1]: status after the barrier and after the split wait (0 or 6);
// out[2]: nanoseconds spent in both.
__global__ void selftest_wait_kernel(unsigned int *counter, int *status, unsigned long long timeout_ns,
                                     long long *out) {
    __shared__ int s_flag;
    const unsigned long long t0 = globaltimer_ns();
    // a barrier of a two-CTA launch, reached by this CTA alone
    const bool ok1 = grid_barrier(counter, 2u, status, timeout_ns, &s_flag);
    const int st1 = ok1 ? 0 : 6;
    // a split-phase wait for an arrival count nothing provides
    const bool ok2 = grid_wait(counter, 1000u, status, timeout_ns, &s_flag);
    if (threadIdx.x == 0) {
        out[0] = st1;
        out[1] = ok2 ? 0 : 6;
        out[2] = (long long)(globaltimer_ns() - t0);
    }
}

}  // namespace
}  // namespace rebk

extern "C" rebk_status rebk_selftest_waits(int64_t timeout_ns, int32_t *codes, double *elapsed_ms) {
    rebk::set_last_error("");
    if (!codes) {
        rebk::set_last_error("codes is NULL");
        return REBK_EINVAL;
    }
    if (timeout_ns < 1000 || timeout_ns > 1000000000) {
        rebk::set_last_error("timeout_ns must be in [1e3, 1e9]");
        return REBK_EINVAL;
    }
    unsigned int *counter = nullptr;
    int *status = nullptr;
    long long *out = nullptr;
    cudaError_t e = cudaMalloc(&counter, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&out, 3 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(counter, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
    if (e == cudaSuccess) {
        rebk::selftest_wait_kernel<<<1, 128>>>(counter, status, (unsigned long long)timeout_ns, out);
        e = cudaGetLastError();
    }
    long long host[3] = {0, 0, 0};
    int st = 0;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, out, sizeof(host), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(counter);
    cudaFree(status);
    cudaFree(out);
    if (e != cudaSuccess) {
        rebk::set_last_error(std::string("selftest: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA;
    }
    codes[0] = (int32_t)host[0];
    codes[1] = (int32_t)host[1];
    if (elapsed_ms) *elapsed_ms = (double)host[2] * 1e-6;
    return st == 6 ? REBK_BARRIER_TIMEOUT : REBK_OK;
}
