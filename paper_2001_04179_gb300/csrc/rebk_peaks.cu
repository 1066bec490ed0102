// rebk_peaks.cu -- two microbenchmarks that give the roofline denominators the
// driver's measured peaks do not cover: the FP64 FMA rate (the bound of the
// plain FP64 REBK path, whose block products are one FMA per element loaded)
// and the L2 read bandwidth (the bound of the sparse path, whose CSR / CSC
// working set stays in L2).  Timed with CUDA events on the given stream; the
// FP64 kernel also reads the SM clock it ran at (clock64 against the global
// timer), so a rate can be set against the clock.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "rebk.h"
#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {
namespace {

constexpr int kPeakThreads = 512;
constexpr int kFmaChains = 8;  // independent FMA chains per thread (latency hiding)

// Every thread runs kFmaChains independent chains a <- a * mul + add for
// `iters` steps: 2 * kFmaChains * iters FLOPs per thread.  The chains stay
// bounded (|mul| < 1) and the result is stored only when it equals a value it
// cannot take, so the compiler keeps every FMA and memory sees no traffic.
__global__ void __launch_bounds__(kPeakThreads) fp64_fma_kernel(int iters, double mul, double add, double *sink,
                                                                 unsigned long long *clk) {
    double a[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) a[c] = 1e-3 * (double)(threadIdx.x + c);
    unsigned long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        t0 = globaltimer_ns();
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) a[c] = fma(a[c], mul, add);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += a[c];
    if (s == -1.0) sink[blockIdx.x] = s;  // never true: |a| stays below add / (1 - mul)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = clock64() - c0;
        clk[1] = globaltimer_ns() - t0;
    }
}

// Reads the `words` 16-byte words of buf `reps` times, grid-stride, through L2
// only (ld.global.cg); the sum is stored only if it is NaN-free and equal to a
// sentinel, which it never is for the zeroed buffer (0 != 1).
__global__ void __launch_bounds__(kPeakThreads) l2_read_kernel(const float4 *buf, int64_t words, int reps,
                                                                float *sink) {
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < words; e += stride) {
            const float4 v = __ldcg(buf + e);
            acc += v.x + v.y + v.z + v.w;
        }
    }
    if (acc == 1.f) sink[blockIdx.x] = acc;
}

}  // namespace
}  // namespace rebk

using namespace rebk;

extern "C" rebk_status rebk_device_peaks(rebk_peaks *out, void *stream) {
    set_last_error("");
    if (!out) {
        set_last_error("out is NULL");
        return REBK_EINVAL;
    }
    *out = rebk_peaks{};
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double *sink = nullptr;
    unsigned long long *clk = nullptr;
    float4 *buf = nullptr;
    rebk_status result = REBK_OK;
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && result == REBK_OK) {
            set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
            result = e == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA;
        }
        return result == REBK_OK;
    };
    ck(cudaGetDevice(&dev), "cudaGetDevice") &&
        ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count") &&
        ck(cudaEventCreate(&e0), "event") && ck(cudaEventCreate(&e1), "event") &&
        ck(cudaMalloc(&sink, sizeof(double) * 4 * (size_t)std::max(sms, 1)), "cudaMalloc") &&
        ck(cudaMalloc(&clk, sizeof(unsigned long long) * 2), "cudaMalloc");
    // ---- FP64 FMA rate: 4 CTAs of 512 threads per SM, best of 3 ----
    if (result == REBK_OK) {
        const int grid = 4 * sms, iters = 1 << 13;
        float best = 1e30f;
        for (int rep = 0; rep < 4 && result == REBK_OK; ++rep) {
            ck(cudaEventRecord(e0, st), "event");
            fp64_fma_kernel<<<grid, kPeakThreads, 0, st>>>(iters, 0.999999, 1e-7, sink, clk);
            ck(cudaGetLastError(), "fp64_fma_kernel");
            ck(cudaEventRecord(e1, st), "event");
            ck(cudaEventSynchronize(e1), "event");
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, e0, e1), "event");
            if (rep > 0) best = std::min(best, ms);  // the first launch warms up
        }
        unsigned long long hc[2] = {0, 0};
        ck(cudaMemcpy(hc, clk, sizeof(hc), cudaMemcpyDeviceToHost), "clock readback");
        const double flops = 2.0 * kFmaChains * (double)iters * (double)grid * kPeakThreads;
        out->fp64_tflops = flops / (best * 1e-3) / 1e12;
        out->fp64_ms = best;
        out->sm_mhz = hc[1] > 0 ? 1e3 * (double)hc[0] / (double)hc[1] : 0.0;
    }
    // ---- L2 read bandwidth: a 48 MiB buffer (fits the L2), read 8 times a launch ----
    if (result == REBK_OK) {
        const int64_t bytes = 48ll << 20, words = bytes / 16;
        const int reps = 8;
        ck(cudaMalloc(&buf, bytes), "cudaMalloc") && ck(cudaMemsetAsync(buf, 0, bytes, st), "memset");
        float best = 1e30f;
        for (int rep = 0; rep < 4 && result == REBK_OK; ++rep) {
            ck(cudaEventRecord(e0, st), "event");
            l2_read_kernel<<<2 * sms, kPeakThreads, 0, st>>>(buf, words, reps, reinterpret_cast<float *>(sink));
            ck(cudaGetLastError(), "l2_read_kernel");
            ck(cudaEventRecord(e1, st), "event");
            ck(cudaEventSynchronize(e1), "event");
            float ms = 0.f;
            ck(cudaEventElapsedTime(&ms, e0, e1), "event");
            if (rep > 0) best = std::min(best, ms);
        }
        out->l2_gbs = (double)bytes * reps / (best * 1e-3) / 1e9;
        out->l2_ms = best;
        out->l2_bytes = (double)bytes;
    }
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (clk) cudaFree(clk);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return result;
}
