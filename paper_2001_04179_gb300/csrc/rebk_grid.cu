// rebk_grid.cu -- persistent fused REBK kernel for one system on the whole GPU.
//
// Algorithm 1 of Du, Si, Sun (arXiv:2001.04179), iteration k:
//   column step  w = A_{:,J}^T z,  z <- z - alpha/||A_{:,J}||_F^2 * A_{:,J} w
//   row step     r = A_{I,:} x - b_I + z_I,  x <- x - alpha/||A_{I,:}||_F^2 * A_{I,:}^T r
//
// Work split.  CTA c owns a slice of rows R_c (for the column step: the z
// entries and A_{R_c, J}) and a slice of columns C_c (for the row step: the x
// entries and A_{I, C_c}).  Both products of a step then split into per-CTA
// partial sums plus one cross-CTA reduction of a tau-vector (w or r), while
// the updates of z and x are local to their owners.
//
// One device-wide barrier per iteration.  The z-chain never reads x and the
// block indices do not depend on the data (counter-based Philox), so phase p
// does, between two barriers:
//   1. read the reduced w^p and r^{p-1} (and a stopping-test partial),
//   2. x update with block I_{p-1} and r^{p-1}   -> x^{p-1}   (own columns)
//   3. z update with block J_p and w^p           -> z^p       (own rows)
//   4. partial of w^{p+1} = A_{R_c, J_{p+1}}^T z^p           -> accumulator
//   5. partial of r^p = A_{I_p, C_c} x^{p-1} (+ z^p_l - b_l on owned rows)
//   6. (every check_every iterations) partial of ||x^{p-1} - x_ref||^2
// then the barrier.  Partial sums go to FP64 accumulators by atomic adds,
// replicated kAccReplicas times to spread contention; three rotating
// accumulator sets make reads, writes and clearing of consecutive phases
// independent.  The tiles for the next phase are prefetched into L2 with
// bulk prefetches one phase ahead.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {

namespace {

template <typename T> __device__ __forceinline__ T tzero() { return T(0); }
__device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t lmax(int64_t a, int64_t b) { return a > b ? a : b; }

// out(row) = sum_{c in [ca, cb)} A[row, c] * vin[c - ca] for rows [ra, rb).
// Rows are handled by groups of gs lanes (gs = power of two >= the number of
// 16-byte vectors in the column range, at most 32); each group handles U rows
// per pass so U loads are in flight per lane.
template <typename TA, typename TS, int U, typename Emit>
__device__ __forceinline__ void row_dots(const TA *__restrict__ A, int64_t lda, int64_t ra,
                                         int64_t rb, int64_t ca, int64_t cb,
                                         const TS *__restrict__ vin, Emit emit) {
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    if (rb <= ra || cb <= ca) return;
    const int64_t va = ca / V, vb = (cb + V - 1) / V;
    const int nv = (int)(vb - va);
    int gs = 1;
    while (gs < nv && gs < 32) gs <<= 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & (gs - 1);
    const int gpw = 32 / gs;
    const int g = warp * gpw + lane / gs;
    const int NG = kWarps * gpw;
    for (int64_t base = ra; base < rb; base += (int64_t)NG * U) {
        TS acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = tzero<TS>();
        for (int vc = 0; vc < nv; vc += gs) {
            const int vi = vc + sub;
            const int64_t col0 = (va + vi) * V;
            TS xv[V];
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int64_t c = col0 + e;
                xv[e] = (vi < nv && c >= ca && c < cb) ? vin[c - ca] : tzero<TS>();
            }
            TS a[U][V];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t r = base + g + (int64_t)u * NG;
                if (vi < nv && r < rb) {
                    IO::load(A + r * lda + col0, a[u]);
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e) a[u][e] = tzero<TS>();
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < V; ++e) acc[u] = fma(a[u][e], xv[e], acc[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            TS v = acc[u];
            for (int o = gs >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            const int64_t r = base + g + (int64_t)u * NG;
            if (sub == 0 && r < rb) emit(r, v);
        }
    }
}

// out(col) = sum_{r in [ra, rb)} A[r, col] * vrow[r - ra] for columns [ca, cb).
// Threads are laid out as (vector index, row group); each thread sums its
// vector over its rows, then the row groups are added through shared memory
// (red: kThreads * V elements).
template <typename TA, typename TS, int U, typename Emit>
__device__ __forceinline__ void col_sums(const TA *__restrict__ A, int64_t lda, int64_t ra,
                                         int64_t rb, int64_t ca, int64_t cb,
                                         const TS *__restrict__ vrow, TS *red, Emit emit) {
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    if (rb <= ra || cb <= ca) return;
    const int64_t va = ca / V, vb = (cb + V - 1) / V;
    const int nv = (int)(vb - va);
    for (int vc0 = 0; vc0 < nv; vc0 += kThreads) {
        const int nvc = min(kThreads, nv - vc0);
        const int NRG = kThreads / nvc;
        const int vi = threadIdx.x % nvc, rg = threadIdx.x / nvc;
        if (rg < NRG) {
            TS acc[V];
#pragma unroll
            for (int e = 0; e < V; ++e) acc[e] = tzero<TS>();
            const int64_t col0 = (va + vc0 + vi) * V;
            for (int64_t base = ra + rg; base < rb; base += (int64_t)NRG * U) {
                TS a[U][V];
                TS xr[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t r = base + (int64_t)u * NRG;
                    if (r < rb) {
                        IO::load(A + r * lda + col0, a[u]);
                        xr[u] = vrow[r - ra];
                    } else {
#pragma unroll
                        for (int e = 0; e < V; ++e) a[u][e] = tzero<TS>();
                        xr[u] = tzero<TS>();
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int e = 0; e < V; ++e) acc[e] = fma(a[u][e], xr[u], acc[e]);
            }
#pragma unroll
            for (int e = 0; e < V; ++e) red[rg * (nvc * V) + vi * V + e] = acc[e];
        }
        __syncthreads();
        for (int c = threadIdx.x; c < nvc * V; c += kThreads) {
            const int64_t col = (va + vc0) * V + c;
            if (col >= ca && col < cb) {
                TS sum = tzero<TS>();
                for (int q = 0; q < NRG; ++q) sum += red[q * (nvc * V) + c];
                emit(col, sum);
            }
        }
        __syncthreads();
    }
}

template <typename T> __device__ __forceinline__ bool finite_val(T v) { return isfinite(v); }

struct Smem {
    int *ring_j, *ring_i, *flags;
};

}  // namespace

template <typename TA, typename TS, bool CORR>
__global__ void __launch_bounds__(kThreads, 1) rebk_grid_kernel(const GridArgs args) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    constexpr int U = 4;

    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
    const TA *__restrict__ A = static_cast<const TA *>(args.A);
    const int64_t m = args.m, n = args.n, lda = args.lda;
    const int64_t nu = (n + 7) / 8;
    const int64_t r0 = m * cta / G, r1 = m * (cta + 1) / G;
    const int64_t c0 = lmin(n, 8 * (nu * cta / G)), c1 = lmin(n, 8 * (nu * (cta + 1) / G));
    const int nrow = (int)(r1 - r0), ncol = (int)(c1 - c0);

    // ---- shared memory carve-up (same layout as grid_smem_bytes()) ----
    const SmemLayout L = smem_layout(args.nrow_cap, args.ncol_cap, args.tau_r, args.tau_c, CORR,
                                     (int)sizeof(TS), V);
    int *ring_j = reinterpret_cast<int *>(smem_raw);
    int *ring_i = ring_j + kRing;
    int *flags = ring_i + kRing;  // [0] barrier ok, [1] stop code
    TS *zeta = reinterpret_cast<TS *>(smem_raw + L.zeta);
    TS *beta_own = reinterpret_cast<TS *>(smem_raw + L.beta);
    TS *v_own = reinterpret_cast<TS *>(smem_raw + L.v);    // CORR only
    TS *xi = reinterpret_cast<TS *>(smem_raw + L.xi);
    TS *s_own = reinterpret_cast<TS *>(smem_raw + L.s);    // CORR only
    TS *w = reinterpret_cast<TS *>(smem_raw + L.w);
    TS *rr = reinterpret_cast<TS *>(smem_raw + L.r);
    TS *red = reinterpret_cast<TS *>(smem_raw + L.red);
    double *dred = reinterpret_cast<double *>(smem_raw + L.red);  // reused for double block sums

    TS *gz = static_cast<TS *>(args.z);
    TS *gx = static_cast<TS *>(args.x);
    TS *gs_dual = static_cast<TS *>(args.sdual);
    TS *gv_dual = static_cast<TS *>(args.vdual);

    for (int i = tid; i < nrow; i += kThreads) {
        zeta[i] = gz[r0 + i];
        beta_own[i] = (TS)args.beta[r0 + i];
        if (CORR) v_own[i] = gv_dual[r0 + i];
    }
    for (int j = tid; j < ncol; j += kThreads) {
        xi[j] = gx[c0 + j];
        if (CORR) s_own[j] = gs_dual[c0 + j];
    }

    const int64_t K = args.iters;
    const int rep = cta % args.acc_r;
    const int aw = args.acc_w;
    const int64_t accset = (int64_t)args.acc_r * aw;
    const bool check = args.x_ref != nullptr && args.check_every > 0;

    // block indices of iteration k (1-based within this launch), sampled before
    // the launch, kept in a small ring in shared memory
    auto load_idx = [&](int64_t k) {
        ring_j[k % kRing] = __ldg(args.idx + 2 * (k - 1));
        ring_i[k % kRing] = __ldg(args.idx + 2 * (k - 1) + 1);
    };
    if (tid == 0) {
        for (int64_t k = 1; k <= 3 && k <= K; ++k) load_idx(k);
        flags[1] = 0;
    }
    __syncthreads();

    auto col_range = [&](int j, int64_t *a, int64_t *b) {
        *a = (int64_t)j * args.tau_c;
        *b = lmin(n, *a + args.tau_c);
    };
    auto row_range = [&](int i, int64_t *a, int64_t *b) {
        *a = (int64_t)i * args.tau_r;
        *b = lmin(m, *a + args.tau_r);
    };
    auto prefetch_col_tile = [&](int j) {  // A[R_c, J_j]
        int64_t a, b;
        col_range(j, &a, &b);
        for (int64_t r = r0 + tid; r < r1; r += kThreads)
            prefetch_l2_range(A + r * lda + a, A + r * lda + b);
    };
    auto prefetch_row_tile = [&](int i) {  // A[I_i, C_c]
        if (ncol == 0) return;
        int64_t a, b;
        row_range(i, &a, &b);
        for (int64_t r = a + tid; r < b; r += kThreads)
            prefetch_l2_range(A + r * lda + c0, A + r * lda + c1);
    };
    // partial of w for column block j over owned rows -> accumulator set `set`
    auto partial_w = [&](int j, double *accp) {
        int64_t ja, jb;
        col_range(j, &ja, &jb);
        col_sums<TA, TS, U>(A, lda, r0, r1, ja, jb, zeta, red, [&](int64_t col, TS v) {
            atomicAdd(accp + (col - ja), (double)v);
        });
    };

    // ---------------- phase 0 ----------------
    if (K >= 1) {
        prefetch_col_tile(ring_j[1 % kRing]);
        if (K >= 2) prefetch_col_tile(ring_j[2 % kRing]);
        prefetch_row_tile(ring_i[1 % kRing]);
        partial_w(ring_j[1 % kRing], args.acc + 0 * accset + (int64_t)rep * aw);
    }
    int64_t done = 0;
    int stop_code = 0;  // 0 running, 1 converged, 5 diverged, 6 timeout
    if (!grid_barrier(args.bar, (unsigned)G * 1u, args.status, args.timeout_ns, &flags[0])) return;

    // ---------------- phases 1 .. K+1 ----------------
    for (int64_t p = 1; p <= K + 1; ++p) {
        if (tid == kThreads - 1 && p + 3 <= K) load_idx(p + 3);
        if (p + 2 <= K) prefetch_col_tile(ring_j[(p + 2) % kRing]);
        if (p + 1 <= K) prefetch_row_tile(ring_i[(p + 1) % kRing]);

        const double *accr = args.acc + ((p - 1) % 3) * accset;
        const int jp = (p <= K) ? ring_j[p % kRing] : 0;
        const int ip1 = (p >= 2) ? ring_i[(p - 1) % kRing] : 0;
        int64_t ja = 0, jb = 0, ia = 0, ib = 0;
        if (p <= K) col_range(jp, &ja, &jb);
        if (p >= 2) row_range(ip1, &ia, &ib);
        const int wc = (int)(jb - ja), hr = (int)(ib - ia);

        // 1. reduced vectors
        if (tid < wc) {
            double sum = 0.0;
            for (int q = 0; q < args.acc_r; ++q) sum += ld_cg(accr + (int64_t)q * aw + tid);
            if (CORR) sum += args.gamma[ja + tid];
            w[tid] = (TS)sum;
        }
        if (tid < hr) {
            double sum = 0.0;
            for (int q = 0; q < args.acc_r; ++q) sum += ld_cg(accr + (int64_t)q * aw + args.tau_c + tid);
            rr[tid] = (TS)sum;
        }
        if (tid == 0) {
            int code = 0;
            const int64_t kc = p - 2;  // iterate whose error partial was formed in phase p-1
            if (check && kc >= 1 && (args.check_offset + kc) % args.check_every == 0) {
                double e2 = 0.0;
                for (int q = 0; q < args.acc_r; ++q)
                    e2 += ld_cg(accr + (int64_t)q * aw + args.tau_c + args.tau_r);
                if (e2 <= args.tol2_abs) code = 1;
            }
            flags[1] = code;
        }
        __syncthreads();
        if (tid < 32) {  // divergence: a reduced product is Inf/NaN
            bool bad = false;
            for (int l = tid; l < wc; l += 32) bad |= !finite_val(w[l]);
            for (int l = tid; l < hr; l += 32) bad |= !finite_val(rr[l]);
            bad = __any_sync(0xffffffffu, bad);
            if (tid == 0 && bad && flags[1] == 0) flags[1] = 5;
        }
        __syncthreads();
        stop_code = flags[1];
        if (stop_code == 1) {
            done = p - 2;
            break;
        }
        if (stop_code == 5) {
            done = p - 1;
            break;
        }

        // 2. x update with I_{p-1}
        if (p >= 2) {
            const TS cI = (TS)(args.alpha / args.nr[ip1]);
            col_sums<TA, TS, U>(A, lda, ia, ib, c0, c1, rr, red, [&](int64_t col, TS v) {
                xi[col - c0] -= cI * v;
            });
            if (CORR) {
                const int64_t la = lmax(ia, r0), lb = lmin(ib, r1);
                for (int64_t l = la + tid; l < lb; l += kThreads) v_own[l - r0] -= cI * rr[l - ia];
            }
        }
        if (p == K + 1) {
            done = K;
            break;
        }

        // 3. z update with J_p
        {
            const TS cJ = (TS)(args.alpha / args.nc[jp]);
            row_dots<TA, TS, U>(A, lda, r0, r1, ja, jb, w, [&](int64_t row, TS v) {
                zeta[row - r0] -= cJ * v;
            });
            if (CORR) {
                const int64_t la = lmax(ja, c0), lb = lmin(jb, c1);
                for (int64_t l = la + tid; l < lb; l += kThreads) s_own[l - c0] += cJ * w[l - ja];
            }
        }
        __syncthreads();

        double *accw = args.acc + (p % 3) * accset + (int64_t)rep * aw;
        // 4. partial of w^{p+1}
        if (p < K) partial_w(ring_j[(p + 1) % kRing], accw);

        // 5. partial of r^p = A_{I_p, C_c} x^{p-1} + (z^p - b) on owned rows
        {
            const int ipc = ring_i[p % kRing];
            int64_t qa, qb;
            row_range(ipc, &qa, &qb);
            if (ncol > 0) {
                row_dots<TA, TS, U>(A, lda, qa, qb, c0, c1, xi, [&](int64_t row, TS v) {
                    atomicAdd(accw + args.tau_c + (row - qa), (double)v);
                });
            }
            const int64_t la = lmax(qa, r0), lb = lmin(qb, r1);
            for (int64_t l = la + tid; l < lb; l += kThreads)
                atomicAdd(accw + args.tau_c + (l - qa), (double)(zeta[l - r0] - beta_own[l - r0]));
        }

        // 6. stopping-test partial for x^{p-1}
        if (check && (p - 1) >= 1 && (args.check_offset + p - 1) % args.check_every == 0) {
            double e2 = 0.0;
            for (int j = tid; j < ncol; j += kThreads) {
                const double xb = args.x_base ? args.x_base[c0 + j] : 0.0;
                const double d = xb + (double)xi[j] - args.x_ref[c0 + j];
                e2 += d * d;
            }
            e2 = warp_sum(e2);
            __syncthreads();  // red may still be read by col_sums callers above
            if ((tid & 31) == 0) dred[tid >> 5] = e2;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int q = 0; q < kWarps; ++q) s += dred[q];
                atomicAdd(accw + args.tau_c + args.tau_r, s);
            }
        }

        // clear the set used two phases ahead
        if (cta == 0) {
            double *accz = args.acc + ((p + 1) % 3) * accset;
            for (int64_t q = tid; q < accset; q += kThreads) accz[q] = 0.0;
        }
        if (!grid_barrier(args.bar, (unsigned)G * (unsigned)(p + 1), args.status, args.timeout_ns,
                          &flags[0]))
            return;
    }

    // ---- write back the owned slices ----
    for (int i = tid; i < nrow; i += kThreads) {
        gz[r0 + i] = zeta[i];
        if (CORR) gv_dual[r0 + i] = v_own[i];
    }
    for (int j = tid; j < ncol; j += kThreads) {
        gx[c0 + j] = xi[j];
        if (CORR) gs_dual[c0 + j] = s_own[j];
    }
    if (cta == 0 && tid == 0) {
        *args.iters_done = done;
        if (stop_code == 5) atomicExch(args.status, 5);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int vec_width(Mode mode) { return mode == Mode::PlainF64 ? 2 : (mode == Mode::CorrF32 ? 4 : 8); }
static size_t ts_size(Mode mode) { return mode == Mode::PlainF64 ? 8 : 4; }

size_t grid_smem_bytes(Mode mode, const GridArgs &a) {
    return smem_layout(a.nrow_cap, a.ncol_cap, a.tau_r, a.tau_c, mode != Mode::PlainF64,
                       (int)ts_size(mode), vec_width(mode))
        .total;
}

__global__ void sample_kernel(uint64_t seed, uint64_t stream, int64_t k0, int64_t K,
                              const double *__restrict__ cdf_r, int s, const double *__restrict__ cdf_c,
                              int t, int fb_r, int fb_c, int32_t *__restrict__ idx) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 2 * K;
         e += (int64_t)gridDim.x * blockDim.x) {
        // draw d = 2(k0 + k - 1) + {0: column, 1: row} for entry e = 2(k - 1) + {0, 1}
        const uint64_t d = 2 * (uint64_t)k0 + (uint64_t)e;
        const double u = draw_uniform(seed, stream, d);
        idx[e] = (e & 1) ? pick_block(cdf_r, s, u, fb_r) : pick_block(cdf_c, t, u, fb_c);
    }
}

cudaError_t sample_blocks(uint64_t seed, uint64_t stream, int64_t k0, int64_t K, const double *cdf_r,
                          int s, const double *cdf_c, int t, int fb_r, int fb_c, int32_t *idx,
                          cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    int64_t blocks = (2 * K + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    sample_kernel<<<(unsigned)blocks, 256, 0, st>>>(seed, stream, k0, K, cdf_r, s, cdf_c, t, fb_r, fb_c,
                                                    idx);
    return cudaGetLastError();
}

template <typename TA, typename TS, bool CORR> static void *kernel_ptr() {
    return reinterpret_cast<void *>(&rebk_grid_kernel<TA, TS, CORR>);
}

static void *mode_kernel(Mode mode) {
    switch (mode) {
    case Mode::PlainF64: return kernel_ptr<double, double, false>();
    case Mode::CorrF32: return kernel_ptr<float, float, true>();
    default: return kernel_ptr<__nv_bfloat16, float, true>();
    }
}

int grid_max_ctas(Mode mode, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *k = mode_kernel(mode);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kThreads, smem) != cudaSuccess) return 0;
    return sms * (per > 1 ? 1 : per);  // one CTA per SM
}

cudaError_t launch_grid(Mode mode, const GridArgs &a, int G, cudaStream_t st) {
    const size_t smem = grid_smem_bytes(mode, a);
    void *k = mode_kernel(mode);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    GridArgs copy = a;
    void *params[] = {&copy};
    return cudaLaunchCooperativeKernel(k, dim3(G), dim3(kThreads), params, smem, st);
}

}  // namespace rebk
