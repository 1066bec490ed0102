// rebk_noalloc.cu -- a solve entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: hosts that route every device
// allocation through their own allocator or memory budget and forbid any
// other allocation, and real-time services that must not take the driver's
// allocation locks (or risk an out-of-memory failure) inside their serving
// loop.  rebk_solve_noalloc serves them: it runs the same persistent FP64
// kernel as rebk_solve_ex for a fixed number of iterations, with all of its
// working memory in one statically sized device array that lives in this file.
// The call reads a few words back to the host and synchronises its stream.
//
// Scratch array.  g_noalloc_scratch (kNoallocBytes = 32 MiB) exists once on
// every GPU that loads the library and stays there until the process exits.
// It holds a zero-padded copy of A, the block norm tables and their prefix
// sums, the step coefficients, the sampled block indices of one launch, the
// cross-CTA accumulators and the barrier / status words.  Host code cannot use
// the array's name as a device address (in host code it is a host-side
// stand-in), so the device address is looked up with cudaGetSymbolAddress,
// once per device, on the first call made while that device is current.
//
// Every call shares the array and leaves its contents behind; the call clears
// what has to start at zero (accumulators, barrier counter, status) itself.
// Two calls whose GPU work overlaps (different streams, or different host
// threads on one device) race on the array and give wrong results: serialise
// them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "rebk.h"
#include "rebk_internal.h"

namespace rebk {
namespace {

constexpr size_t kNoallocBytes = 32ull << 20;  // 32 MiB per device
constexpr int kNoallocMaxDevices = 64;
constexpr int64_t kNoallocIdxChunk = 1 << 16;  // iterations sampled per launch

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

struct NoallocWorkspace {  // barrier counters, status word, iterations run
    unsigned int bar;
    unsigned int bar_x;
    int status;
    int64_t iters_done;
};

rebk_status na_fail(rebk_status s, const std::string &msg) {
    set_last_error(msg);  // reported by rebk_last_error()
    return s;
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
rebk_status scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(REBK_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoallocMaxDevices) return na_fail(REBK_EUNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return na_fail(REBK_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
    return REBK_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace rebk

using namespace rebk;

extern "C" rebk_status rebk_solve_noalloc(const double *A, int64_t m, int64_t n, int64_t lda,
                                          int64_t tau_row, int64_t tau_col, double alpha,
                                          const double *b, double *x, double *z, int64_t iters,
                                          uint64_t seed, void *stream) {
    set_last_error("");
    if (!A || !b || !x || !z) return na_fail(REBK_EINVAL, "A, b, x and z must be device pointers");
    if (m < 1 || n < 1 || lda < n) return na_fail(REBK_EINVAL, "need m, n >= 1 and lda >= n");
    if (tau_row < 1 || tau_col < 1) return na_fail(REBK_EINVAL, "tau must be >= 1");
    if (!(alpha > 0.0)) return na_fail(REBK_EINVAL, "alpha must be > 0 (no beta_max here)");
    if (iters < 0) return na_fail(REBK_EINVAL, "iters < 0");
    // Each of m and n alone must fit the array as doubles: this keeps every size
    // product below in range of size_t and the block counts in range of int.
    if (m > (int64_t)(kNoallocBytes / 8) || n > (int64_t)(kNoallocBytes / 8))
        return na_fail(REBK_EUNSUPPORTED, "problem needs more scratch than the " + std::to_string(kNoallocBytes) +
                                              " bytes rebk_solve_noalloc holds (m or n too large)");
    const int64_t tr = std::min(tau_row, m), tc = std::min(tau_col, n);
    if (tr > 512 || tc > 512) return na_fail(REBK_EUNSUPPORTED, "tau > 512");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);

    // ---- carve the scratch array ----
    const int64_t ldp = (n + 63) / 64 * 64;  // padded leading dimension of the copy
    const int s = (int)((m + tr - 1) / tr), t = (int)((n + tc - 1) / tc);
    const int acc_w = (int)((std::max(tc, tr + 1) + 31) / 32 * 32);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t oA = take(sizeof(double) * (size_t)m * ldp);
    const size_t onr = take(sizeof(double) * s), onc = take(sizeof(double) * t);
    const size_t ocr = take(sizeof(double) * s), occ = take(sizeof(double) * t);
    const size_t ocfr = take(sizeof(double) * s), ocfc = take(sizeof(double) * t);
    const size_t ocf32r = take(sizeof(float) * s), ocf32c = take(sizeof(float) * t);
    const size_t ofb = take(sizeof(int) * 2);
    const size_t oidx = take(sizeof(int32_t) * 2 * kNoallocIdxChunk);
    const size_t oacc = take(sizeof(double) * 6 * kAccReplicas * (size_t)acc_w);
    const size_t ows = take(sizeof(NoallocWorkspace));
    const size_t otab = take(sizeof(double) * (size_t)(m + n + 64 * n));  // norm-table scratch
    if (off > kNoallocBytes)
        return na_fail(REBK_EUNSUPPORTED,
                       "problem needs " + std::to_string(off) + " bytes of scratch; rebk_solve_noalloc holds " +
                           std::to_string(kNoallocBytes) + " (about m * ceil(n/64)*64 * 8 + 520 n bytes)");

    unsigned char *base = nullptr;
    rebk_status rs = scratch_address(&base);
    if (rs != REBK_OK) return rs;
    double *Ap = reinterpret_cast<double *>(base + oA);
    double *nr = reinterpret_cast<double *>(base + onr), *nc = reinterpret_cast<double *>(base + onc);
    double *cdf_r = reinterpret_cast<double *>(base + ocr), *cdf_c = reinterpret_cast<double *>(base + occ);
    double *cf_r = reinterpret_cast<double *>(base + ocfr), *cf_c = reinterpret_cast<double *>(base + ocfc);
    float *cf32_r = reinterpret_cast<float *>(base + ocf32r), *cf32_c = reinterpret_cast<float *>(base + ocf32c);
    int *fb = reinterpret_cast<int *>(base + ofb);
    int32_t *idx = reinterpret_cast<int32_t *>(base + oidx);
    double *acc = reinterpret_cast<double *>(base + oacc);
    NoallocWorkspace *ws = reinterpret_cast<NoallocWorkspace *>(base + ows);
    double *tab = reinterpret_cast<double *>(base + otab);

#define NA_CK(call)                                                                                \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess) return na_fail(REBK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

    // padded copy of A, norm tables, step coefficients (the previous call's
    // contents are overwritten)
    NA_CK(cudaMemcpy2DAsync(Ap, ldp * sizeof(double), A, lda * sizeof(double), n * sizeof(double), m,
                            cudaMemcpyDeviceToDevice, st));
    if (ldp > n)
        NA_CK(cudaMemset2DAsync(Ap + n, ldp * sizeof(double), 0, (ldp - n) * sizeof(double), m, st));
    NA_CK(block_tables(Ap, ldp, m, n, (int)tr, (int)tc, s, t, nr, nc, cdf_r, cdf_c, fb, tab, st));
    NA_CK(step_coefficients(nr, s, alpha, cf_r, cf32_r, st));
    NA_CK(step_coefficients(nc, t, alpha, cf_c, cf32_c, st));
    int fbh[2] = {0, 0};
    double fro2 = 0.0;
    NA_CK(cudaMemcpyAsync(fbh, fb, sizeof(fbh), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaMemcpyAsync(&fro2, cdf_r + (s - 1), sizeof(double), cudaMemcpyDeviceToHost, st));
    // Algorithm 1 starts from z = b, x = 0 (Section 3)
    NA_CK(cudaMemcpyAsync(z, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    NA_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    NA_CK(cudaStreamSynchronize(st));
    if (fro2 == 0.0 || iters == 0) return REBK_OK;  // A = 0: x = 0 = A^+ b

    // launch arguments of the plain FP64 persistent kernel
    GridArgs a;
    memset(&a, 0, sizeof(a));
    a.A = Ap;
    a.lda = ldp;
    a.m = m;
    a.n = n;
    a.tau_r = (int)tr;
    a.tau_c = (int)tc;
    a.s = s;
    a.t = t;
    a.cdf_r = cdf_r;
    a.cdf_c = cdf_c;
    a.nr = nr;
    a.nc = nc;
    a.coef_r = cf_r;
    a.coef_c = cf_c;
    a.fb_r = fbh[0];
    a.fb_c = fbh[1];
    a.alpha = alpha;
    a.seed = seed;
    a.stream = 0;
    a.z = z;
    a.x = x;
    a.beta = b;
    a.acc = acc;
    a.acc_w = acc_w;
    a.acc_r = acc_replicas(Mode::PlainF64);
    a.bar = &ws->bar;
    a.bar_x = &ws->bar_x;
    a.status = &ws->status;
    a.iters_done = &ws->iters_done;
    a.timeout_ns = kBarrierTimeoutNs;
    // CTA count: about 2048 block elements per CTA, at most one CTA per SM (the
    // persistent kernel's cooperative launch), more if the owned slices need them
    int dev = 0, sms = 0;
    NA_CK(cudaGetDevice(&dev));
    NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sms < 1) sms = 1;
    int G = (int)std::max<int64_t>(1, (tr * n + tc * m + 2047) / 2048);
    G = std::min(G, sms);
    for (;;) {
        a.nrow_cap = (int)((m + G - 1) / G) + 1;
        a.ncol_cap = (int)(8 * (((n + 7) / 8 + G - 1) / G)) + 8;
        if (grid_smem_bytes(Mode::PlainF64, a) <= 200 * 1024 || G >= sms) break;
        G = std::min(sms, G * 2);
    }
    const int maxG = grid_max_ctas(Mode::PlainF64, grid_smem_bytes(Mode::PlainF64, a));
    if (maxG < 1) return na_fail(REBK_EUNSUPPORTED, "persistent kernel does not fit on this GPU");
    G = std::min(G, maxG);
    a.nrow_cap = (int)((m + G - 1) / G) + 1;
    a.ncol_cap = (int)(8 * (((n + 7) / 8 + G - 1) / G)) + 8;
    if (grid_smem_bytes(Mode::PlainF64, a) > 227 * 1024)
        return na_fail(REBK_EUNSUPPORTED, "owned slices too large for shared memory");

    for (int64_t done = 0; done < iters;) {
        const int64_t chunk = std::min(iters - done, kNoallocIdxChunk);
        NA_CK(sample_blocks(seed, 0, done, chunk, cdf_r, s, cdf_c, t, fbh[0], fbh[1], idx, st));
        a.idx = idx;
        a.k0 = done;
        a.iters = chunk;
        // what has to start at zero: accumulators, barrier counter, status
        NA_CK(cudaMemsetAsync(acc, 0, sizeof(double) * 6 * kAccReplicas * (size_t)acc_w, st));
        NA_CK(cudaMemsetAsync(ws, 0, sizeof(NoallocWorkspace), st));
        NA_CK(launch_grid(Mode::PlainF64, a, G, st));
        NoallocWorkspace w;
        NA_CK(cudaMemcpyAsync(&w, ws, sizeof(w), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        if (w.status == 6) return na_fail(REBK_BARRIER_TIMEOUT, "device-wide barrier timed out");
        if (w.status == 5) return na_fail(REBK_DIVERGED, "iteration diverged (Inf/NaN)");
        // the call promises exactly `iters` iterations: anything else is an error
        if (w.status != 0 || w.iters_done != chunk)
            return na_fail(REBK_ECUDA, "persistent kernel ran " + std::to_string(w.iters_done) + " of " +
                                           std::to_string(chunk) + " iterations (status " +
                                           std::to_string(w.status) + ")");
        done += chunk;
    }
#undef NA_CK
    return REBK_OK;
}
