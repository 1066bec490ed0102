// rebk_tune.cu -- block-size autotuner of the dense solver (see include/rebk.h).
//
// Section 3 picks the block size tau and the step size alpha = c / beta_max by
// hand for each experiment; the time to a given error depends on tau twice:
// through the iteration count (the rates of Theorem main improve as beta_max
// falls with tau) and through the cost of one iteration on the device.  This
// file measures the product directly: for each candidate tau it builds a
// solver (rows and columns partitioned with the same tau, as in Section 3),
// sets alpha = c / max(beta^I_max, beta^J_max), runs `trials` solves to the
// requested tolerance and records the mean device time.  Host logic only: all
// arithmetic runs in the solver's kernels.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "rebk.h"
#include "rebk_internal.h"

namespace {

rebk_status tune_fail(rebk_status s, const std::string &msg) {
    rebk::set_last_error(msg);
    return s;
}

rebk_status tune_cuda(cudaError_t e, const char *what) {
    rebk::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA;
}

// One candidate: create, set alpha, warm the launch-shape choice, time the trials.
rebk_status tune_one(const double *A_dev, int64_t m, int64_t n, int64_t lda, const double *b,
                     const double *x_ref, int64_t tau, double c, int32_t storage, double tol,
                     int64_t max_iter, uint64_t seed, int32_t trials, const rebk_options &base, double *x,
                     rebk_tune_point *pt) {
    rebk_options o = base;
    o.tau_row = std::min(tau, m);
    o.tau_col = std::min(tau, n);
    if (storage != REBK_FP64) o.storage_mask |= 1 << storage;
    rebk_handle h = nullptr;
    rebk_status s = rebk_create(&h, A_dev, m, n, lda, 1, nullptr, 0.0, &o);
    if (s != REBK_OK) return s;
    double br = 0.0, bc = 0.0;
    s = rebk_beta_max(h, &br, &bc);
    const double bmax = std::max(br, bc);
    if (s == REBK_OK && bmax > 0.0) s = rebk_set_alpha(h, c / bmax);
    double alpha = 0.0;
    if (s == REBK_OK) s = rebk_get_alpha(h, &alpha);
    pt->tau = tau;
    pt->beta_max = bmax;
    pt->alpha = alpha;
    pt->iterations = 0;
    pt->device_ms = -1.0;
    pt->status = REBK_OK;
    rebk_solve_ext ext;
    memset(&ext, 0, sizeof(ext));
    ext.x_ref = x_ref;
    rebk_refine_opts ro;
    memset(&ro, 0, sizeof(ro));
    ro.storage = storage;
    rebk_stats st;
    auto run = [&](double t, int64_t iters, uint64_t sd) {
        return storage == REBK_FP64 ? rebk_solve_ex(h, b, x, t, iters, sd, &ext, &st)
                                    : rebk_solve_refined(h, b, x, t, iters, sd, &ro, &ext, &st);
    };
    // warm-up: the first solve of a handle also chooses the persistent kernel's CTA count
    if (s == REBK_OK) {
        s = run(0.0, std::min<int64_t>(max_iter, 256), seed ^ 0x9e3779b97f4a7c15ull);
        if (s == REBK_MAX_ITER) s = REBK_OK;
    }
    double ms = 0.0;
    int64_t its = 0;
    int32_t worst = REBK_OK;
    for (int32_t r = 0; s == REBK_OK && r < trials; ++r) {
        rebk_status q = run(tol, max_iter, seed + (uint64_t)r);
        if (q != REBK_OK && q != REBK_MAX_ITER && q != REBK_DIVERGED) {
            s = q;
            break;
        }
        if (q != REBK_OK) worst = q;
        ms += st.device_ms;
        its += st.iterations;
    }
    rebk_destroy(h);
    if (s != REBK_OK) return s;
    pt->iterations = its / trials;
    pt->status = worst;
    pt->device_ms = worst == REBK_OK ? ms / trials : -1.0;
    return REBK_OK;
}

}  // namespace

extern "C" {

rebk_status rebk_tune_tau(const double *A, int64_t m, int64_t n, int64_t lda, int A_on_device,
                          const double *b, const double *x_ref, const int64_t *taus, int32_t count,
                          double alpha_factor, int32_t storage, double tol, int64_t max_iter,
                          uint64_t seed, int32_t trials, const rebk_options *opt,
                          rebk_tune_point *points, int64_t *best_tau) {
    rebk::set_last_error("");
    if (!A || !b || !taus || !points || !best_tau) return tune_fail(REBK_EINVAL, "NULL argument");
    *best_tau = 0;
    if (m < 1 || n < 1 || lda < n) return tune_fail(REBK_EINVAL, "m, n >= 1 and lda >= n required");
    if (count < 1) return tune_fail(REBK_EINVAL, "count must be >= 1");
    for (int32_t i = 0; i < count; ++i)
        if (taus[i] < 1) return tune_fail(REBK_EINVAL, "every candidate tau must be >= 1");
    if (storage != REBK_FP64 && storage != REBK_FP32 && storage != REBK_BF16)
        return tune_fail(REBK_EINVAL, "unknown storage");
    if (!(tol > 0.0) || !std::isfinite(tol)) return tune_fail(REBK_EINVAL, "tol must be finite and > 0");
    if (max_iter < 1) return tune_fail(REBK_EINVAL, "max_iter must be >= 1");
    if (trials < 1) return tune_fail(REBK_EINVAL, "trials must be >= 1");
    if (!std::isfinite(alpha_factor)) return tune_fail(REBK_EINVAL, "alpha_factor is not finite");
    const double c = alpha_factor > 0.0 ? alpha_factor : 1.75;
    rebk_options base;
    memset(&base, 0, sizeof(base));
    if (opt) base = *opt;
    const cudaStream_t st = static_cast<cudaStream_t>(base.stream);

    // one device copy of A for all candidates (each solver keeps its own padded copy)
    const double *A_dev = A;
    double *A_tmp = nullptr, *x = nullptr;
    cudaError_t e = cudaSuccess;
    if (!A_on_device) {
        e = cudaMalloc(&A_tmp, sizeof(double) * (size_t)m * n);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(A_tmp, n * sizeof(double), A, lda * sizeof(double), n * sizeof(double), m,
                                  cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        A_dev = A_tmp;
    }
    if (e == cudaSuccess) e = cudaMalloc(&x, sizeof(double) * (size_t)n);
    if (e != cudaSuccess) {
        cudaFree(A_tmp);
        cudaFree(x);
        return tune_cuda(e, "tuner buffers");
    }
    const int64_t ld = A_on_device ? lda : n;
    rebk_status s = REBK_OK;
    for (int32_t i = 0; i < count && s == REBK_OK; ++i)
        s = tune_one(A_dev, m, n, ld, b, x_ref, taus[i], c, storage, tol, max_iter, seed, trials, base, x,
                     &points[i]);
    cudaFree(A_tmp);
    cudaFree(x);
    if (s != REBK_OK) return s;
    int best = -1;
    for (int32_t i = 0; i < count; ++i)
        if (points[i].status == REBK_OK && (best < 0 || points[i].device_ms < points[best].device_ms)) best = i;
    if (best < 0) return tune_fail(REBK_MAX_ITER, "no candidate reached the tolerance within max_iter");
    *best_tau = points[best].tau;
    return REBK_OK;
}

}  // extern "C"
