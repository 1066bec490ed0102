// rebk_free.cu -- Algorithm 1 with index sets drawn without a partition.
//
// Section 4 of Du, Si, Sun (arXiv:2001.04179) names variants of REBK whose
// random samplings do not depend on partitions.  The reading built here:
// iteration k draws tau_c column indices j_1..j_{tau_c} independently, each
// with probability ||A_{:,j}||^2 / ||A||_F^2, and tau_r row indices likewise
// with ||A_{i,:}||^2 / ||A||_F^2; A_J and A_I are the drawn columns and rows
// in draw order (repeats repeated) and the step is Algorithm 1's:
//   z <- z - alpha / ||A_J||_F^2 * A_J A_J^T z
//   x <- x - alpha / ||A_I||_F^2 * A_I^T (A_I x - b_I + z_I),
// ||A_J||_F^2 the sum of the drawn columns' squared norms.  Draw q of the
// column set of iteration k is slot q of Philox draw 2(k-1) (counter
// (2(k-1), q, 0, 0)), of the row set slot q of draw 2(k-1)+1.
//
// GB300 mapping.  One cooperative launch (one CTA per SM at most) runs many
// iterations.  CTA c owns a slice of rows (its z entries) and of columns (its
// x entries); no CTA reads another's z or x.  One device-wide barrier per
// iteration: round t applies x^{t-1} (needs r^{t-1}) and z^t (needs w^t) on
// the owned slices, then adds its partials of r^t = A_{I_t} x^{t-1} - b_I +
// z^t_I and of w^{t+1} = A_{J_{t+1}}^T z^t, and arrives.  The drawn rows
// are read from the row-major copy, the drawn columns from a transposed FP64
// copy A^T (built on the first partition-free solve), where each is one
// contiguous row: in the row-major copy a set of scattered columns costs one
// 32-byte sector, from anywhere in the matrix, per 8-byte element.  Partials
// meet in FP64 atomics on three rotating accumulator sets.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {
namespace {

constexpr int kFreeThreads = 256;
constexpr int kFreeWarps = kFreeThreads / 32;
constexpr int kCU = 4;             // owned rows / columns per lane in flight (the updates)
constexpr int kRU = 4;             // rows per warp in flight (row-wise products)
constexpr int kXCols = 32 * kCU;   // owned columns per pass of the x update

__global__ void free_sample_kernel(uint64_t seed, uint64_t stream, int64_t k0, int64_t K,
                                   const double *__restrict__ cdf_r, int m, const double *__restrict__ cdf_c, int n,
                                   int tau_r, int tau_c, int fb_r, int fb_c, int32_t *__restrict__ idx) {
    const int W = tau_c + tau_r;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < K * W;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t it = e / W;
        const int q = (int)(e - it * W);
        const uint64_t d = 2 * (uint64_t)(k0 + it);  // column draw of iteration k0 + it + 1
        if (q < tau_c) {
            idx[e] = pick_block(cdf_c, n, draw_uniform_slot(seed, stream, d, (uint64_t)q), fb_c);
        } else {
            idx[e] = pick_block(cdf_r, m, draw_uniform_slot(seed, stream, d + 1, (uint64_t)(q - tau_c)), fb_r);
        }
    }
}

// Shared memory: the draws of two consecutive iterations (J and I, by parity),
// w and r of the current round, reduction scratch, and the per-warp partial
// sums of the updates whose warps split a sum ([kFreeWarps][kXCols]).
struct FreeSmem {
    size_t jset, iset, w, r, red, part, total;
};

__host__ __device__ inline FreeSmem free_layout(int tau_r, int tau_c) {
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    FreeSmem L;
    size_t o = 0;
    L.jset = o; o = al(o + sizeof(int) * 2 * (size_t)tau_c);
    L.iset = o; o = al(o + sizeof(int) * 2 * (size_t)tau_r);
    L.w = o;    o = al(o + sizeof(double) * (size_t)tau_c);
    L.r = o;    o = al(o + sizeof(double) * (size_t)tau_r);
    L.red = o;  o = al(o + sizeof(double) * (kFreeWarps + 4));
    L.part = o; o = al(o + sizeof(double) * kFreeWarps * (size_t)kXCols);
    L.total = o;
    return L;
}

__global__ void __launch_bounds__(kFreeThreads, 1) rebk_free_kernel(const FreeArgs a) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const FreeSmem L = free_layout(a.tau_r, a.tau_c);
    int *sJ = reinterpret_cast<int *>(fsm + L.jset);   // [2][tau_c], slot t & 1 holds J_t
    int *sI = reinterpret_cast<int *>(fsm + L.iset);   // [2][tau_r], slot t & 1 holds I_t
    double *sw = reinterpret_cast<double *>(fsm + L.w);
    double *sr = reinterpret_cast<double *>(fsm + L.r);
    double *red = reinterpret_cast<double *>(fsm + L.red);
    double *part = reinterpret_cast<double *>(fsm + L.part);
    __shared__ int s_flag, s_test, s_bad_r, s_bad_w;  // one flag per decision of a round

    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *__restrict__ A = a.A;
    const double *__restrict__ AT = a.AT;  // n rows of ldt: A^T
    const int64_t m = a.m, n = a.n, lda = a.lda, ldt = a.ldt;
    const int64_t r0 = m * cta / G, r1 = m * (cta + 1) / G;  // owned rows (z)
    const int64_t c0 = n * cta / G, c1 = n * (cta + 1) / G;  // owned columns (x)
    const int tr = a.tau_r, tc = a.tau_c, W = tr + tc;
    constexpr int pw = kXCols;  // row stride of part
    const int64_t K = a.iters;
    const int aw = a.acc_w;
    const int64_t clr0 = (int64_t)aw * cta / G, clr1 = (int64_t)aw * (cta + 1) / G;  // this CTA's share
    double *z = a.z, *x = a.x;
    const bool check = a.x_ref != nullptr && a.check_every > 0;
    auto due = [&](int64_t k) {  // x^k is tested
        return check && k >= 1 && (a.check_offset + k) % a.check_every == 0;
    };
    auto load_draws = [&](int64_t t) {  // J_t and I_t (t = 1..K) into slot t & 1
        const int32_t *row = a.idx + (t - 1) * W;
        for (int q = tid; q < W; q += kFreeThreads) {
            const int v = __ldg(row + q);
            if (q < tc) sJ[(t & 1) * tc + q] = v;
            else sI[(t & 1) * tr + (q - tc)] = v;
        }
    };
    // partial of w^{t} = A_{R_c, J_t}^T z on the owned rows, into set `dst`: warps over
    // the drawn columns (kRU in flight), each a row of A^T, lanes over the owned rows
    auto partial_w = [&](int64_t t, double *dst) {
        const int *J = sJ + (t & 1) * tc;
        for (int qb = warp; qb < tc; qb += kFreeWarps * kRU) {
            double s[kRU];
            int64_t ju[kRU];
#pragma unroll
            for (int u = 0; u < kRU; ++u) {
                const int q = qb + u * kFreeWarps;
                ju[u] = q < tc ? J[q] : -1;
                s[u] = 0.0;
            }
            for (int64_t r = r0 + lane; r < r1; r += 32) {
                const double zr = z[r];
#pragma unroll
                for (int u = 0; u < kRU; ++u)
                    if (ju[u] >= 0) s[u] = fma(__ldg(AT + ju[u] * ldt + r), zr, s[u]);
            }
#pragma unroll
            for (int u = 0; u < kRU; ++u) {
                const double v = warp_sum(s[u]);
                const int q = qb + u * kFreeWarps;
                if (lane == 0 && q < tc && r1 > r0) atomicAdd(dst + tr + q, v);
            }
        }
    };

    if (K >= 1) {
        load_draws(1);
        __syncthreads();
        partial_w(1, a.acc);  // round 0: w^1 into set 0
    }
    grid_arrive(a.bar);
    int64_t done = K;
    for (int64_t t = 1; t <= K + 1; ++t) {
        if (!grid_wait(a.bar, (unsigned)G * (unsigned)t, a.status, a.timeout_ns, &s_flag)) {
            done = t > 2 ? t - 2 : 0;
            break;
        }
        const double *accS = a.acc + ((t - 1) % 3) * aw;
        // ---- the test on x^{t-2}, added in round t-1 ----
        if (tid == 0) {
            int stop = 0;
            if (t >= 2 && due(t - 2) && __ldcg(accS + tr + tc) <= a.tol2_abs) stop = 1;
            s_test = stop;
        }
        __syncthreads();
        if (s_test) {
            done = t - 2;
            break;
        }
        // ---- x^{t-1} = x^{t-2} - c_I A_{I_{t-1}}^T r^{t-1} on the owned columns ----
        if (t >= 2) {
            const int *I = sI + ((t - 1) & 1) * tr;
            for (int q = tid; q < tr; q += kFreeThreads) sr[q] = __ldcg(accS + q);
            if (tid == 0) {
                double f = 0.0;
                for (int q = 0; q < tr; ++q) f += __ldg(a.rn + I[q]);
                red[kFreeWarps] = a.alpha / f;
                int bad = 0;
                for (int q = 0; q < tr; ++q)
                    if (!isfinite(__ldcg(accS + q))) bad = 1;
                s_bad_r = bad;
            }
            __syncthreads();
            if (s_bad_r) {
                if (tid == 0) atomicExch(a.status, 5);
                done = t - 2;
                break;
            }
            const double cI = red[kFreeWarps];
            // lanes over kXCols owned columns (coalesced), warps over the drawn rows, the
            // warps' sums added in warp order
            for (int64_t cb = c0; cb < c1; cb += kXCols) {
                double acc[kCU];
#pragma unroll
                for (int u = 0; u < kCU; ++u) acc[u] = 0.0;
#pragma unroll 2
                for (int q = warp; q < tr; q += kFreeWarps) {
                    const double *Ai = A + (int64_t)I[q] * lda;
                    const double rq = sr[q];
#pragma unroll
                    for (int u = 0; u < kCU; ++u) {
                        const int64_t c = cb + lane + 32 * u;
                        if (c < c1) acc[u] = fma(__ldg(Ai + c), rq, acc[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < kCU; ++u) part[warp * pw + lane + 32 * u] = acc[u];
                __syncthreads();
                for (int e = tid; e < kXCols; e += kFreeThreads) {
                    const int64_t c = cb + e;
                    if (c < c1) {
                        double s = 0.0;
                        for (int w2 = 0; w2 < kFreeWarps; ++w2) s += part[w2 * pw + e];
                        x[c] -= cI * s;
                    }
                }
                __syncthreads();
            }
        }
        if (t == K + 1) break;
        // ---- z^t = z^{t-1} - c_J A_{R_c, J_t} w^t on the owned rows ----
        const int *J = sJ + (t & 1) * tc;
        for (int q = tid; q < tc; q += kFreeThreads) sw[q] = __ldcg(accS + tr + q);
        if (tid == 0) {
            double f = 0.0;
            for (int q = 0; q < tc; ++q) f += __ldg(a.cn + J[q]);
            red[kFreeWarps + 1] = a.alpha / f;
            int bad = 0;
            for (int q = 0; q < tc; ++q)
                if (!isfinite(__ldcg(accS + tr + q))) bad = 1;
            s_bad_w = bad;
        }
        __syncthreads();
        if (s_bad_w) {
            if (tid == 0) atomicExch(a.status, 5);
            done = t - 1;
            break;
        }
        const double cJ = red[kFreeWarps + 1];
        // lanes over kXCols owned rows (coalesced in A^T), warps over the drawn columns,
        // the warps' sums added in warp order
        for (int64_t rb = r0; rb < r1; rb += kXCols) {
            double acc[kCU];
#pragma unroll
            for (int u = 0; u < kCU; ++u) acc[u] = 0.0;
#pragma unroll 2
            for (int q = warp; q < tc; q += kFreeWarps) {
                const double *Aq = AT + (int64_t)J[q] * ldt;
                const double wq = sw[q];
#pragma unroll
                for (int u = 0; u < kCU; ++u) {
                    const int64_t r = rb + lane + 32 * u;
                    if (r < r1) acc[u] = fma(__ldg(Aq + r), wq, acc[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < kCU; ++u) part[warp * pw + lane + 32 * u] = acc[u];
            __syncthreads();
            for (int e = tid; e < kXCols; e += kFreeThreads) {
                const int64_t r = rb + e;
                if (r < r1) {
                    double s = 0.0;
                    for (int w2 = 0; w2 < kFreeWarps; ++w2) s += part[w2 * pw + e];
                    z[r] -= cJ * s;
                }
            }
            __syncthreads();
        }
        if (t + 1 <= K) load_draws(t + 1);  // J_{t+1}, I_{t+1} into the other slot
        __syncthreads();
        // ---- partials of round t into set t % 3 ----
        double *accT = a.acc + (t % 3) * aw;
        {
            const int *I = sI + (t & 1) * tr;
            // r^t: A_{i_q, C_c} x^{t-1} (+ z^t_i - b_i if owned); warps over the drawn rows
            // (kRU in flight), lanes over the owned columns
            for (int qb = warp; qb < tr; qb += kFreeWarps * kRU) {
                double s[kRU];
                int64_t iu[kRU];
#pragma unroll
                for (int u = 0; u < kRU; ++u) {
                    const int q = qb + u * kFreeWarps;
                    iu[u] = q < tr ? I[q] : -1;
                    s[u] = 0.0;
                }
                for (int64_t c = c0 + lane; c < c1; c += 32) {
                    const double xc = x[c];
#pragma unroll
                    for (int u = 0; u < kRU; ++u)
                        if (iu[u] >= 0) s[u] = fma(__ldg(A + iu[u] * lda + c), xc, s[u]);
                }
#pragma unroll
                for (int u = 0; u < kRU; ++u) {
                    double v = warp_sum(s[u]);
                    const int q = qb + u * kFreeWarps;
                    if (lane == 0 && q < tr) {
                        const int64_t i = iu[u];
                        if (i >= r0 && i < r1) v += z[i] - a.b[i];
                        if (c1 > c0 || (i >= r0 && i < r1)) atomicAdd(accT + q, v);
                    }
                }
            }
        }
        if (due(t - 1)) {  // ||x^{t-1} - x_ref||^2 over the owned columns
            double e2 = 0.0;
            for (int64_t c = c0 + tid; c < c1; c += kFreeThreads) {
                const double d = x[c] - a.x_ref[c];
                e2 = fma(d, d, e2);
            }
            e2 = warp_sum(e2);
            if (lane == 0) red[warp] = e2;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int w2 = 0; w2 < kFreeWarps; ++w2) s += red[w2];
                atomicAdd(accT + tr + tc, s);
            }
        }
        if (t + 1 <= K) partial_w(t + 1, accT);
        {  // clear this CTA's share of the set round t + 1 fills (read last in round t - 1)
            double *accN = a.acc + ((t + 1) % 3) * aw;
            for (int64_t e = clr0 + tid; e < clr1; e += kFreeThreads) accN[e] = 0.0;
        }
        grid_arrive(a.bar);
    }
    if (cta == 0 && tid == 0) *a.iters_done = done;
}

}  // namespace

size_t free_smem_bytes(int tau_r, int tau_c) { return free_layout(tau_r, tau_c).total; }

namespace {
// AT[j * ldt + i] = A[i * lda + j] for i < m, j < n, through 32 x 32 shared-memory
// tiles (both sides coalesced).
__global__ void transpose_f64_kernel(const double *__restrict__ A, int64_t lda, int64_t m, int64_t n,
                                     double *__restrict__ AT, int64_t ldt) {
    __shared__ double tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r, j = j0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < m && j < n) ? A[i * lda + j] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t j = j0 + r, i = i0 + threadIdx.x;
        if (j < n && i < m) AT[j * ldt + i] = tile[threadIdx.x][r];
    }
}
}  // namespace

cudaError_t transpose_f64(const double *A, int64_t lda, int64_t m, int64_t n, double *AT, int64_t ldt,
                          cudaStream_t st) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32));
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    transpose_f64_kernel<<<grid, dim3(32, 8), 0, st>>>(A, lda, m, n, AT, ldt);
    return cudaGetLastError();
}

cudaError_t free_sample(uint64_t seed, uint64_t stream, int64_t k0, int64_t K, const double *cdf_r, int64_t m,
                        const double *cdf_c, int64_t n, int tau_r, int tau_c, int fb_r, int fb_c, int32_t *idx,
                        cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    int64_t blocks = (K * (tau_r + tau_c) + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    free_sample_kernel<<<(unsigned)blocks, 256, 0, st>>>(seed, stream, k0, K, cdf_r, (int)m, cdf_c, (int)n, tau_r,
                                                         tau_c, fb_r, fb_c, idx);
    return cudaGetLastError();
}

int free_max_ctas(int tau_r, int tau_c) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = free_smem_bytes(tau_r, tau_c);
    if (cudaFuncSetAttribute(rebk_free_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rebk_free_kernel, kFreeThreads, smem) != cudaSuccess)
        return 0;
    return per >= 1 ? sms : 0;  // one CTA per SM
}

cudaError_t launch_free(const FreeArgs &a, int G, cudaStream_t st) {
    const size_t smem = free_smem_bytes(a.tau_r, a.tau_c);
    cudaError_t e = cudaFuncSetAttribute(rebk_free_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    FreeArgs copy = a;
    void *params[] = {&copy};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void *>(&rebk_free_kernel), dim3(G), dim3(kFreeThreads),
                                       params, smem, st);
}

}  // namespace rebk
