// rebk_spectral.cu -- extreme nonzero singular values of A for the step-size
// results of Section 2: Remark alpha's mean-optimal step 2||A||_F^2 / (sigma_1^2
// + sigma_r^2) with the rate delta of Theorem ner, and the rates eta, rho of
// Theorem main (which need sigma_r^2).
//
// Golub-Kahan-Lanczos bidiagonalisation on the device, FP64, with full
// reorthogonalisation (two classical Gram-Schmidt passes per vector):
//   u_1 = A r / ||A r|| (r random), alpha_1 v_1 = A^T u_1,
//   beta_{j+1} u_{j+1} = A v_j - alpha_j u_j,
//   alpha_{j+1} v_{j+1} = A^T u_{j+1} - beta_{j+1} v_j.
// In exact arithmetic every v_j lies in range(A^T) and every u_j in range(A), so
// the Ritz values lie in [sigma_r^2, sigma_1^2] and approach the ends from inside
// as k grows; they are exact once the Krylov space is invariant (rounding: see
// the end of lanczos_extremes).
// The products run in the FP64 sweep kernel of rebk_setup.cu; the two extreme
// eigenvalues of the tridiagonal come from Sturm-sequence bisection on the host.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {
namespace {

// c[j] = <M_j, w> for the columns M_j (length len, contiguous) j < cols; one CTA per column.
__global__ void gram_dots_kernel(const double *__restrict__ M, int64_t len, const double *__restrict__ w,
                                 double *__restrict__ c) {
    __shared__ double red[32];
    const double *col = M + (int64_t)blockIdx.x * len;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) s = fma(col[i], w[i], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) c[blockIdx.x] = t;
    }
}

// w -= sum_j c[j] M_j over the columns j < cols.
__global__ void gram_sub_kernel(double *__restrict__ w, const double *__restrict__ M, int64_t len, int cols,
                                const double *__restrict__ c) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int j = 0; j < cols; ++j) s = fma(-c[j], M[(int64_t)j * len + i], s);
        w[i] = s;
    }
}

// dst = (src - shift * prev) * scale  (prev may be NULL)
__global__ void combine_kernel(double *dst, const double *src, const double *__restrict__ prev, double shift,
                               double scale, int64_t len) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double s = src[i];
        if (prev) s = fma(-shift, prev[i], s);
        dst[i] = s * scale;
    }
}

// A start vector with entries in (-1, 1) from a 64-bit mix of (seed, i) (splitmix64).
__global__ void start_kernel(double *__restrict__ u, int64_t len, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9e3779b97f4a7c15ull * (uint64_t)(i + 1);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        u[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

unsigned grid_of(int64_t len) {
    int64_t g = (len + 255) / 256;
    return (unsigned)std::min<int64_t>(std::max<int64_t>(g, 1), 1024);
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm sequence).
int sturm_below(const std::vector<double> &d, const std::vector<double> &e, double x) {
    int count = 0;
    double q = 1.0;
    for (size_t i = 0; i < d.size(); ++i) {
        const double off = i > 0 ? e[i - 1] * e[i - 1] : 0.0;
        q = d[i] - x - (i > 0 ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;  // x hit a pivot exactly: count it as below
        if (q < 0.0) ++count;
    }
    return count;
}

// The idx-th smallest eigenvalue (0-based) by bisection inside the Gershgorin interval.
double tridiag_eig(const std::vector<double> &d, const std::vector<double> &e, int idx) {
    double lo = d[0], hi = d[0];
    for (size_t i = 0; i < d.size(); ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < d.size() ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_below(d, e, mid) > idx) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

cudaError_t lanczos_extremes(const double *A, int64_t lda, int64_t m, int64_t n, int steps, uint64_t seed,
                             cudaStream_t st, double *sigma1_sq, double *sigma_r_sq, int *steps_done) {
    *sigma1_sq = *sigma_r_sq = 0.0;
    *steps_done = 0;
    const int k = (int)std::min<int64_t>(steps, std::min(m, n));  // callers bound steps (<= 2048)
    double *U = nullptr, *V = nullptr, *w_m = nullptr, *w_n = nullptr, *c = nullptr, *nrm = nullptr;
    cudaError_t e = cudaMalloc(&U, sizeof(double) * (size_t)m * (k + 1));
    if (e == cudaSuccess) e = cudaMalloc(&V, sizeof(double) * (size_t)n * (k + 1));
    if (e == cudaSuccess) e = cudaMalloc(&w_m, sizeof(double) * (size_t)m);
    if (e == cudaSuccess) e = cudaMalloc(&w_n, sizeof(double) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&c, sizeof(double) * (size_t)(k + 2));
    if (e == cudaSuccess) e = cudaMalloc(&nrm, sizeof(double) * 2);
    auto norm_of = [&](const double *v, int64_t len, double *out) -> cudaError_t {
        cudaError_t r = sum_sq(v, len, nrm, st);
        double h[2] = {0.0, 0.0};
        if (r == cudaSuccess) r = cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (r == cudaSuccess) r = cudaStreamSynchronize(st);
        *out = std::sqrt(h[1]);
        return r;
    };
    // w <- w - M (M^T w), twice, over the first cols columns of M
    auto reorth = [&](double *w, const double *M, int64_t len, int cols) -> cudaError_t {
        for (int pass = 0; pass < 2 && cols > 0; ++pass) {
            gram_dots_kernel<<<cols, 256, 0, st>>>(M, len, w, c);
            gram_sub_kernel<<<grid_of(len), 256, 0, st>>>(w, M, len, cols, c);
        }
        return cudaGetLastError();
    };
    std::vector<double> al, be;  // alpha_1.., beta_2..
    double a0 = 0.0;
    if (e == cudaSuccess) {
        // u_1 = A r / ||A r|| for a random r: a start inside range(A) (see the end)
        start_kernel<<<grid_of(n), 256, 0, st>>>(w_n, n, seed);
        e = dual_sweep(A, lda, m, n, w_n, false, nullptr, false, w_m, nullptr, st);
        double nu = 0.0;
        if (e == cudaSuccess) e = norm_of(w_m, m, &nu);
        if (e == cudaSuccess && nu > 0.0) {
            combine_kernel<<<grid_of(m), 256, 0, st>>>(U, w_m, nullptr, 0.0, 1.0 / nu, m);
            e = dual_sweep(A, lda, m, n, nullptr, false, U, false, nullptr, w_n, st);  // A^T u_1
            double a = 0.0;
            if (e == cudaSuccess) e = norm_of(w_n, n, &a);
            a0 = a;
            if (e == cudaSuccess && a > 0.0) {
                combine_kernel<<<grid_of(n), 256, 0, st>>>(V, w_n, nullptr, 0.0, 1.0 / a, n);
                al.push_back(a);
            }
        }
    }
    // Breakdown: a new alpha or beta below 1e-10 of the largest so far (a lower bound
    // of sigma_1) means the Krylov space is invariant to rounding -- after two
    // Gram-Schmidt passes an exhausted direction leaves about 1e-16 sigma_1.
    // Singular values below 1e-10 sigma_1 therefore count as zero (numerical rank).
    double scale = a0;
    for (int j = 0; e == cudaSuccess && j < (int)al.size() && j < k; ++j) {
        const double tiny = 1e-10 * scale;
        // beta u_{j+1} = A v_j - alpha_j u_j, reorthogonalised against u_1..u_j
        const double *vj = V + (int64_t)j * n;
        double *uj = U + (int64_t)j * m, *un = U + (int64_t)(j + 1) * m;
        e = dual_sweep(A, lda, m, n, vj, false, nullptr, false, w_m, nullptr, st);
        if (e != cudaSuccess) break;
        combine_kernel<<<grid_of(m), 256, 0, st>>>(w_m, w_m, uj, al[j], 1.0, m);
        e = reorth(w_m, U, m, j + 1);
        double b = 0.0;
        if (e == cudaSuccess) e = norm_of(w_m, m, &b);
        if (e != cudaSuccess) break;
        be.push_back(b);
        if (!(b > tiny) || j + 1 >= k) break;  // invariant subspace, or the last step
        scale = std::max(scale, b);
        combine_kernel<<<grid_of(m), 256, 0, st>>>(un, w_m, nullptr, 0.0, 1.0 / b, m);
        // alpha v_{j+1} = A^T u_{j+1} - beta v_j, reorthogonalised against v_1..v_{j+1}
        e = dual_sweep(A, lda, m, n, nullptr, false, un, false, nullptr, w_n, st);
        if (e != cudaSuccess) break;
        combine_kernel<<<grid_of(n), 256, 0, st>>>(w_n, w_n, vj, b, 1.0, n);
        e = reorth(w_n, V, n, j + 1);
        double a = 0.0;
        if (e == cudaSuccess) e = norm_of(w_n, n, &a);
        if (e != cudaSuccess || !(a > tiny)) break;
        combine_kernel<<<grid_of(n), 256, 0, st>>>(V + (int64_t)(j + 1) * n, w_n, nullptr, 0.0, 1.0 / a, n);
        al.push_back(a);
        scale = std::max(scale, a);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(U);
    cudaFree(V);
    cudaFree(w_m);
    cudaFree(w_n);
    cudaFree(c);
    cudaFree(nrm);
    if (e != cudaSuccess || al.empty()) return e;
    // Two Rayleigh-Ritz matrices from the same coefficients (kk steps):
    //   v side: V^T A^T A V = B^T B, B the (kk+1) x kk lower bidiagonal (alpha on the
    //     diagonal, beta below), tridiagonal with diagonal alpha_j^2 + beta_{j+1}^2;
    //   u side: U^T A A^T U = Bh Bh^T, Bh its leading kk x kk block (the last beta
    //     dropped), with the same nonzero eigenvalues as Bh^T Bh.
    // In rounding, the recurrence scales the components of the v's along null(A) by
    // about beta / alpha per step and those of the u's along null(A^T) by about
    // alpha / beta, so one side stays inside range(A^T) (or range(A)) while the
    // other may pick up null directions whose Ritz values fall toward 0.  Ritz
    // values of a clean side lie in [sigma_r^2, sigma_1^2]: sigma_r^2 is taken as the
    // larger of the two sides' smallest values above 1e-12 lambda_max (numerical
    // zeros dropped), sigma_1^2 as the larger of their largest values.
    const int kk = (int)std::min(al.size(), be.size() > 0 ? be.size() : (size_t)1);
    double lmax = 0.0, lmin = 0.0;
    for (int side = 0; side < 2; ++side) {
        std::vector<double> d(kk), off(kk > 1 ? kk - 1 : 0);
        for (int j = 0; j < kk; ++j) {
            const bool with_beta = j + 1 < kk || side == 0;
            const double bj = (with_beta && j < (int)be.size()) ? be[j] : 0.0;
            d[j] = al[j] * al[j] + bj * bj;
            if (j + 1 < kk) off[j] = al[j + 1] * be[j];
        }
        const double top = tridiag_eig(d, off, kk - 1);
        const int zeros = sturm_below(d, off, 1e-12 * top);
        const double low = zeros < kk ? tridiag_eig(d, off, zeros) : 0.0;
        lmax = std::max(lmax, top);
        lmin = std::max(lmin, low);
    }
    *sigma1_sq = lmax;
    *sigma_r_sq = lmin;
    *steps_done = kk;
    return cudaSuccess;
}

}  // namespace rebk
