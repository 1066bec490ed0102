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
// the updates of z and x stay with their owners.
//
// One device-wide barrier per iteration.  The z-chain never reads x and the
// block indices do not depend on the data (counter-based Philox, sampled
// before the launch), so phase p does, between two barriers:
//   1. read the reduced w^p and r^{p-1} (and a stopping-test partial),
//   2. x update with block I_{p-1} and r^{p-1}   -> x^{p-1}   (own columns)
//   3. z update with block J_p and w^p           -> z^p       (own rows)
//   4. partial of w^{p+1} = A_{R_c, J_{p+1}}^T z^p           -> accumulator
//   5. partial of r^p = A_{I_p, C_c} x^{p-1} (+ z^p_l - b_l on owned rows)
//   6. (every check_every iterations) partial of ||x^{p-1} - x_ref||^2
// then the barrier.  The tiles {A_{R_c,J_q}, A_{I_{q-1},C_c}} that phase q-1
// reads for its partials are the ones phase q reads for its updates.
//
// Tile movement.  With TMA (FP32 / BF16 storage) both tiles of iteration q
// are 2-D tensor copies into one of two shared-memory buffers, issued as soon
// as the buffer's previous pair has been used (one phase ahead) and waited on
// through an mbarrier with a bounded spin.  Without TMA (FP64 storage, whose
// two tile pairs do not fit in shared memory) the tiles are read from global
// memory after line prefetches into L2 one phase ahead.
//
// Partial sums go to accumulators of the arithmetic type by atomic adds,
// replicated to spread contention; three rotating accumulator sets keep the
// reads, writes and clearing of consecutive phases apart.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {

namespace {

template <typename T> __device__ __forceinline__ T tzero() { return T(0); }
__device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t lmax(int64_t a, int64_t b) { return a > b ? a : b; }

// 16-byte vector load from global (read-only path) or shared memory.
template <typename TA, typename TS, bool SM>
__device__ __forceinline__ void vload(const TA *p, TS (&o)[VecIO<TA, TS>::V]) {
    using IO = VecIO<TA, TS>;
    if constexpr (!SM) {
        IO::load(p, o);
    } else {
        IO::load_shared((uint32_t)__cvta_generic_to_shared(p), o);
    }
}

// Sum over the gs (>= 4) lanes of a group of 4 row partials; returns the full
// sum of row *row_u in every lane (transpose reduction: a lane keeps the half
// of the rows its partner does not, so every add is a useful one).
template <typename TS>
__device__ __forceinline__ TS group_reduce4(TS (&acc)[4], int gs, int sub, int *row_u) {
    const int h1 = gs >> 1, h2 = gs >> 2;
    const bool hi = (sub & h1) != 0;
    TS k0 = hi ? acc[2] : acc[0], k1 = hi ? acc[3] : acc[1];
    const TS s0 = hi ? acc[0] : acc[2], s1 = hi ? acc[1] : acc[3];
    k0 += __shfl_xor_sync(0xffffffffu, s0, h1);
    k1 += __shfl_xor_sync(0xffffffffu, s1, h1);
    const bool hi2 = (sub & h2) != 0;
    TS k = hi2 ? k1 : k0;
    const TS s = hi2 ? k0 : k1;
    k += __shfl_xor_sync(0xffffffffu, s, h2);
    for (int o = h2 >> 1; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    *row_u = (hi ? 2 : 0) + (hi2 ? 1 : 0);
    return k;
}

// out(row) = sum_{c in [ca, cb)} A[row, c] * vin[c - ca] for rows [ra, rb).
// A addresses element (r, c) at A + r * lda + c.  Rows go to groups of gs
// lanes (gs = power of two >= the number of 16-byte vectors of the range, at
// most 32); each group handles 4 rows per pass.
template <typename TA, typename TS, bool SM, typename Emit>
__device__ __forceinline__ void row_dots(const TA *A, int64_t lda, int64_t ra, int64_t rb, int64_t ca,
                                         int64_t cb, const TS *__restrict__ vin, Emit emit) {
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    constexpr int U = 4;
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
                    vload<TA, TS, SM>(A + r * lda + col0, a[u]);
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
        if (gs >= 4) {
            int ru = 0;
            const TS v = group_reduce4<TS>(acc, gs, sub, &ru);
            const int64_t r = base + g + (int64_t)ru * NG;
            if ((sub & ((gs >> 2) - 1)) == 0 && r < rb) emit(r, v);
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                TS v = acc[u];
                for (int o = gs >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                const int64_t r = base + g + (int64_t)u * NG;
                if (sub == 0 && r < rb) emit(r, v);
            }
        }
    }
}

// out(col) = sum_{r in [ra, rb)} A[r, col] * vrow[r - ra] for columns [ca, cb).
// Threads are laid out as (vector index, row group); each thread sums its
// vector over its rows, then the row groups are added through shared memory
// (red: kThreads * V elements).
template <typename TA, typename TS, bool SM, typename Emit>
__device__ __forceinline__ void col_sums(const TA *A, int64_t lda, int64_t ra, int64_t rb, int64_t ca,
                                         int64_t cb, const TS *__restrict__ vrow, TS *red, Emit emit) {
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    constexpr int U = 4;
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
                        vload<TA, TS, SM>(A + r * lda + col0, a[u]);
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

// ---------------------------------------------------------------------------
// TMA / mbarrier helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long timeout_ns) {
    uint32_t done = 0;
    unsigned long long t0 = 0;
    for (uint32_t spins = 0;; ++spins) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (spins == 0) t0 = globaltimer_ns();
        if ((spins & 63u) == 63u && globaltimer_ns() - t0 > timeout_ns) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void prefetch_line(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

}  // namespace

template <typename TA, typename TS, bool CORR, bool TMA>
__global__ void __launch_bounds__(kThreads, 1) rebk_grid_kernel(const __grid_constant__ GridArgs args) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;

    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
    const TA *__restrict__ A = static_cast<const TA *>(args.A);
    const int64_t m = args.m, n = args.n, lda = args.lda;
    const int64_t nu = (n + 7) / 8;
    const int64_t r0 = m * cta / G, r1 = m * (cta + 1) / G;
    const int64_t c0 = lmin(n, 8 * (nu * cta / G)), c1 = lmin(n, 8 * (nu * (cta + 1) / G));
    const int nrow = (int)(r1 - r0), ncol = (int)(c1 - c0);

    // ---- shared memory carve-up (same layout as grid_smem_bytes()) ----
    const SmemLayout L = smem_layout(args.nrow_cap, args.ncol_cap, args.tau_r, args.tau_c, CORR,
                                     (int)sizeof(TS), V, TMA ? args.tile_c_bytes : 0,
                                     TMA ? args.tile_r_bytes : 0);
    int *ring_j = reinterpret_cast<int *>(smem_raw);
    int *ring_i = ring_j + kRing;
    int *flags = ring_i + kRing;  // [0] barrier ok, [1] stop code, [2] tile wait failed
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw + 96);  // two mbarriers
    TS *zeta = reinterpret_cast<TS *>(smem_raw + L.zeta);
    TS *beta_own = reinterpret_cast<TS *>(smem_raw + L.beta);
    TS *v_own = reinterpret_cast<TS *>(smem_raw + L.v);    // CORR only
    TS *xi = reinterpret_cast<TS *>(smem_raw + L.xi);
    TS *s_own = reinterpret_cast<TS *>(smem_raw + L.s);    // CORR only
    TS *w = reinterpret_cast<TS *>(smem_raw + L.w);
    TS *rr = reinterpret_cast<TS *>(smem_raw + L.r);
    TS *red = reinterpret_cast<TS *>(smem_raw + L.red);
    auto tile_c = [&](int b) { return reinterpret_cast<TA *>(smem_raw + (b ? L.tc1 : L.tc0)); };
    auto tile_r = [&](int b) { return reinterpret_cast<TA *>(smem_raw + (b ? L.tr1 : L.tr0)); };

    TS *gz = static_cast<TS *>(args.z);
    TS *gx = static_cast<TS *>(args.x);
    TS *gs_dual = static_cast<TS *>(args.sdual);
    TS *gv_dual = static_cast<TS *>(args.vdual);
    TS *accbase = static_cast<TS *>(args.acc);
    const TS *coef_r = static_cast<const TS *>(args.coef_r);
    const TS *coef_c = static_cast<const TS *>(args.coef_c);

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

    TS *ring_cj = reinterpret_cast<TS *>(smem_raw + L.ringc);          // step coefficients
    TS *ring_ci = ring_cj + kRing;
    auto load_idx = [&](int64_t k) {
        const int j = __ldg(args.idx + 2 * (k - 1)), i = __ldg(args.idx + 2 * (k - 1) + 1);
        ring_j[k % kRing] = j;
        ring_i[k % kRing] = i;
        ring_cj[k % kRing] = coef_c[j];
        ring_ci[k % kRing] = coef_r[i];
    };
    auto col_range = [&](int j, int64_t *a, int64_t *b) {
        *a = (int64_t)j * args.tau_c;
        *b = lmin(n, *a + args.tau_c);
    };
    auto row_range = [&](int i, int64_t *a, int64_t *b) {
        *a = (int64_t)i * args.tau_r;
        *b = lmin(m, *a + args.tau_r);
    };
    if (tid == 0) {
        for (int64_t k = 1; k <= 4 && k <= K; ++k) load_idx(k);
        flags[1] = 0;
        flags[2] = 0;
        flags[3] = 0;
        if (TMA) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    __syncthreads();

    // ---------------- tile sources ----------------
    // TileSet(q) = {A[R_c, J_q] if 1 <= q <= K, A[I_{q-1}, C_c] if 2 <= q <= K+1},
    // in buffer q % 2 (TMA) or read from global (no TMA).
    // per-buffer state, kept in scalars (uniform across the CTA)
    uint32_t par0 = 0u, par1 = 0u;     // mbarrier phase parity to wait for
    bool pend0 = false, pend1 = false;  // copies issued and not yet waited for
    int xc0 = 0, xc1 = 0;               // x origin (column) of the column tile
    auto issue_tiles = [&](int64_t q) {  // TMA: called by all threads, thread 0 issues
        const int b = (int)(q & 1);
        const bool hasc = (q >= 1 && q <= K && nrow > 0);
        const bool hasr = (q >= 2 && q <= K + 1 && ncol > 0);
        int x0 = 0;
        if (hasc) {
            int64_t ja, jb;
            col_range(ring_j[q % kRing], &ja, &jb);
            x0 = (int)(ja / args.tma_vx * args.tma_vx);
        }
        if (b) { xc1 = x0; pend1 = hasc || hasr; } else { xc0 = x0; pend0 = hasc || hasr; }
        if (tid == 0 && (hasc || hasr)) {
            fence_proxy_async();
            const uint32_t bytes = (hasc ? (uint32_t)args.tile_c_bytes_tx : 0u) +
                                   (hasr ? (uint32_t)args.tile_r_bytes_tx : 0u);
            mbar_expect_tx(&mbar[b], bytes);
            if (hasc) {
                for (int bx = 0; bx < args.nbox_c; ++bx)
                    tma_load_2d(tile_c(b) + (size_t)bx * args.bh_c * args.bw_c, &args.tmap_c, x0,
                                (int)(r0 + (int64_t)bx * args.bh_c), &mbar[b]);
            }
            if (hasr) {
                int64_t ia, ib;
                row_range(ring_i[(q - 1) % kRing], &ia, &ib);
                tma_load_2d(tile_r(b), &args.tmap_r, (int)c0, (int)ia, &mbar[b]);
            }
        }
    };
    auto wait_buffer = [&](int b) -> bool {
        const bool pend = b ? pend1 : pend0;
        if (!pend) return true;
        const bool ok = mbar_wait(&mbar[b], b ? par1 : par0, args.timeout_ns);
        if (b) { par1 ^= 1u; pend1 = false; } else { par0 ^= 1u; pend0 = false; }
        return ok;
    };
    auto wait_tiles = [&](int64_t q) -> bool { return wait_buffer((int)(q & 1)); };
    // before leaving the kernel: no tensor copy may still be writing shared memory
    auto drain = [&]() {
        if (TMA) {
            wait_buffer(0);
            wait_buffer(1);
        }
    };
    // base pointer and leading dimension addressing element (r, c) of the
    // column tile of J_q / the row tile of I_{q-1} in absolute coordinates
    auto ctile = [&](int64_t q, int64_t *ld) -> const TA * {
        if (!TMA) {
            *ld = lda;
            return A;
        }
        const int b = (int)(q & 1);
        *ld = args.bw_c;
        return tile_c(b) - r0 * (int64_t)args.bw_c - (b ? xc1 : xc0);
    };
    auto rtile = [&](int64_t q, int64_t ia, int64_t *ld) -> const TA * {
        if (!TMA) {
            *ld = lda;
            return A;
        }
        const int b = (int)(q & 1);
        *ld = args.bw_r;
        return tile_r(b) - ia * (int64_t)args.bw_r - c0;
    };
    // line prefetch of TileSet(q) into L2 (no-TMA path), spread over threads
    auto prefetch_tiles = [&](int64_t q) {
        constexpr int64_t LINE = 128 / sizeof(TA);
        if (q >= 1 && q <= K && nrow > 0) {
            int64_t ja, jb;
            col_range(ring_j[q % kRing], &ja, &jb);
            const int64_t l0 = ja / LINE;
            const int nl = (int)((jb + LINE - 1) / LINE - l0);
            for (int e = tid; e < nrow * nl; e += kThreads) {
                const int rr_ = e / nl, l = e - rr_ * nl;
                prefetch_line(A + (r0 + rr_) * lda + (l0 + l) * LINE);
            }
        }
        if (q >= 2 && q <= K + 1 && ncol > 0) {
            int64_t ia, ib;
            row_range(ring_i[(q - 1) % kRing], &ia, &ib);
            const int64_t l0 = c0 / LINE;
            const int nl = (int)((c1 + LINE - 1) / LINE - l0), h = (int)(ib - ia);
            for (int e = tid; e < h * nl; e += kThreads) {
                const int rr_ = e / nl, l = e - rr_ * nl;
                prefetch_line(A + (ia + rr_) * lda + (l0 + l) * LINE);
            }
        }
    };
    auto partial_w = [&](int64_t q, TS *accp) {  // over own rows, column block J_q
        int64_t ja, jb, ld;
        col_range(ring_j[q % kRing], &ja, &jb);
        const TA *T = ctile(q, &ld);
        col_sums<TA, TS, TMA>(T, ld, r0, r1, ja, jb, zeta, red, [&](int64_t col, TS v) {
            atomicAdd(accp + (col - ja), v);
        });
    };

    // ---------------- phase 0 ----------------
    int64_t done = 0;
    int stop_code = 0;  // 0 running, 1 converged, 5 diverged, 6 timeout
    if (K >= 1) {
        if (TMA) {
            issue_tiles(1);
            issue_tiles(2);
            if (!wait_tiles(1)) flags[2] = 1;
        } else {
            prefetch_tiles(1);
            prefetch_tiles(2);
        }
        __syncthreads();
        if (flags[2] == 0) partial_w(1, accbase + (int64_t)rep * aw);
    }
    if (flags[2] != 0 && tid == 0) atomicExch(args.status, 6);
    if (!grid_barrier(args.bar, (unsigned)G * 1u, args.status, args.timeout_ns, &flags[0]) || flags[2] != 0) {
        drain();
        return;
    }

    // ---------------- phases 1 .. K+1 ----------------
    for (int64_t p = 1; p <= K + 1; ++p) {
        if (tid == kThreads - 1 && p + 4 <= K) load_idx(p + 4);
        if (!TMA) prefetch_tiles(p + 2);

        const TS *accr = accbase + ((p - 1) % 3) * accset;
        const int jp = (p <= K) ? ring_j[p % kRing] : 0;
        const int ip1 = (p >= 2) ? ring_i[(p - 1) % kRing] : 0;
        int64_t ja = 0, jb = 0, ia = 0, ib = 0;
        if (p <= K) col_range(jp, &ja, &jb);
        if (p >= 2) row_range(ip1, &ia, &ib);
        const int wc = (int)(jb - ja), hr = (int)(ib - ia);

        // 1. reduced vectors (flags[3]: a reduced product is Inf/NaN)
        static_assert(kAccReplicas == 4, "step 1 reads four replicas");
        if (tid < wc) {
            const TS *q0 = accr + tid;
            const TS a0 = ld_cg_t(q0), a1 = ld_cg_t(q0 + aw), a2 = ld_cg_t(q0 + 2 * aw),
                     a3 = ld_cg_t(q0 + 3 * aw);
            TS sum = (a0 + a1) + (a2 + a3);
            if (CORR) sum += (TS)args.gamma[ja + tid];
            w[tid] = sum;
            if (!finite_val(sum)) flags[3] = 1;
        }
        if (tid < hr) {
            const TS *q0 = accr + args.tau_c + tid;
            const TS a0 = ld_cg_t(q0), a1 = ld_cg_t(q0 + aw), a2 = ld_cg_t(q0 + 2 * aw),
                     a3 = ld_cg_t(q0 + 3 * aw);
            const TS sum = (a0 + a1) + (a2 + a3);
            rr[tid] = sum;
            if (!finite_val(sum)) flags[3] = 1;
        }
        if (tid == kThreads - 2) {
            int code = 0;
            const int64_t kc = p - 2;  // iterate whose error partial was formed in phase p-1
            if (check && kc >= 1 && (args.check_offset + kc) % args.check_every == 0) {
                TS e2 = tzero<TS>();
                for (int q = 0; q < kAccReplicas; ++q)
                    e2 += ld_cg_t(accr + (int64_t)q * aw + args.tau_c + args.tau_r);
                if ((double)e2 <= args.tol2_abs) code = 1;
            }
            flags[1] = code;
        }
        __syncthreads();
        stop_code = flags[1];
        if (stop_code == 0 && flags[3] != 0) stop_code = 5;
        if (stop_code == 1) {
            done = p - 2;
            break;
        }
        if (stop_code == 5) {
            done = p - 1;
            break;
        }

        // 2. x update with I_{p-1} (row tile of TileSet(p))
        if (p >= 2) {
            const TS cI = ring_ci[(p - 1) % kRing];
            int64_t ld;
            const TA *T = rtile(p, ia, &ld);
            col_sums<TA, TS, TMA>(T, ld, ia, ib, c0, c1, rr, red, [&](int64_t col, TS v) {
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

        // 3. z update with J_p (column tile of TileSet(p))
        {
            const TS cJ = ring_cj[p % kRing];
            int64_t ld;
            const TA *T = ctile(p, &ld);
            row_dots<TA, TS, TMA>(T, ld, r0, r1, ja, jb, w, [&](int64_t row, TS v) {
                zeta[row - r0] -= cJ * v;
            });
            if (CORR) {
                const int64_t la = lmax(ja, c0), lb = lmin(jb, c1);
                for (int64_t l = la + tid; l < lb; l += kThreads) s_own[l - c0] += cJ * w[l - ja];
            }
        }
        __syncthreads();

        // TileSet(p) has been used: its buffer takes TileSet(p + 2); TileSet(p + 1)
        // (loaded during the previous phase) must have landed for the partials.
        if (TMA) {
            issue_tiles(p + 2);
            if (!wait_tiles(p + 1)) flags[2] = 1;
            __syncthreads();
            if (flags[2] != 0) {
                if (tid == 0) atomicExch(args.status, 6);
                drain();
                return;  // the other CTAs give up at their next barrier
            }
        }

        TS *accw = accbase + (p % 3) * accset + (int64_t)rep * aw;
        // 4. partial of w^{p+1}
        if (p < K) partial_w(p + 1, accw);

        // 5. partial of r^p = A_{I_p, C_c} x^{p-1} + (z^p - b) on owned rows (TileSet(p+1))
        {
            int64_t qa, qb;
            row_range(ring_i[p % kRing], &qa, &qb);
            if (ncol > 0) {
                int64_t ld;
                const TA *T = rtile(p + 1, qa, &ld);
                row_dots<TA, TS, TMA>(T, ld, qa, qb, c0, c1, xi, [&](int64_t row, TS v) {
                    atomicAdd(accw + args.tau_c + (row - qa), v);
                });
            }
            const int64_t la = lmax(qa, r0), lb = lmin(qb, r1);
            for (int64_t l = la + tid; l < lb; l += kThreads)
                atomicAdd(accw + args.tau_c + (l - qa), zeta[l - r0] - beta_own[l - r0]);
        }

        // 6. stopping-test partial for x^{p-1}
        if (check && (p - 1) >= 1 && (args.check_offset + p - 1) % args.check_every == 0) {
            double e2 = 0.0;
            for (int j = tid; j < ncol; j += kThreads) {
                const double xb = args.x_base ? args.x_base[c0 + j] : 0.0;
                const double d = xb + (double)xi[j] - args.x_ref[c0 + j];
                e2 = fma(d, d, e2);
            }
            e2 = warp_sum(e2);
            double *dred = reinterpret_cast<double *>(red);
            __syncthreads();
            if ((tid & 31) == 0) dred[tid >> 5] = e2;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int q = 0; q < kWarps; ++q) s += dred[q];
                atomicAdd(accw + args.tau_c + args.tau_r, (TS)s);
            }
        }

        // clear the set used two phases ahead
        if (cta == 0) {
            TS *accz = accbase + ((p + 1) % 3) * accset;
            for (int64_t q = tid; q < accset; q += kThreads) accz[q] = tzero<TS>();
        }
        if (!grid_barrier(args.bar, (unsigned)G * (unsigned)(p + 1), args.status, args.timeout_ns,
                          &flags[0])) {
            drain();
            return;
        }
    }
    drain();

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
static int ts_size(Mode mode) { return mode == Mode::PlainF64 ? 8 : 4; }
int storage_size(Mode mode) { return mode == Mode::PlainF64 ? 8 : (mode == Mode::CorrF32 ? 4 : 2); }

size_t grid_smem_bytes(Mode mode, const GridArgs &a) {
    return smem_layout(a.nrow_cap, a.ncol_cap, a.tau_r, a.tau_c, mode != Mode::PlainF64, ts_size(mode),
                       vec_width(mode), a.use_tma ? a.tile_c_bytes : 0, a.use_tma ? a.tile_r_bytes : 0)
        .total;
}

// Box geometry of the TMA tiles (nrow_cap / ncol_cap set); false if TMA cannot be used.
bool tma_geometry(Mode mode, GridArgs &a) {
    const int es = storage_size(mode);
    const int vx = 16 / es;  // elements per 16 bytes
    a.tma_vx = vx;
    // column tile: own rows x tau_c, widened to cover a start rounded down to 16 bytes
    a.bw_c = (a.tau_c % vx == 0) ? a.tau_c : ((a.tau_c + vx - 1) / vx) * vx + vx;
    a.bh_c = a.nrow_cap <= 256 ? a.nrow_cap : 256;
    a.nbox_c = (a.nrow_cap + a.bh_c - 1) / a.bh_c;
    // row tile: tau_r rows x own columns (start is a multiple of 8 elements)
    a.bw_r = ((a.ncol_cap + vx - 1) / vx) * vx;
    if (a.bw_c > 256 || a.bw_r > 256 || a.tau_r > 256 || a.bh_c < 1) return false;
    a.tile_c_bytes_tx = (int64_t)a.nbox_c * a.bh_c * a.bw_c * es;
    a.tile_r_bytes_tx = (int64_t)a.tau_r * a.bw_r * es;
    a.tile_c_bytes = (a.tile_c_bytes_tx + 127) / 128 * 128;
    a.tile_r_bytes = (a.tile_r_bytes_tx + 127) / 128 * 128;
    return true;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor maps of the stored matrix (m rows of lda elements) with the two box shapes.
cudaError_t tma_encode(Mode mode, GridArgs &a) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int es = storage_size(mode);
    const CUtensorMapDataType dt = mode == Mode::PlainF64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : mode == Mode::CorrF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint64_t dims[2] = {(cuuint64_t)a.lda, (cuuint64_t)a.m};
    cuuint64_t strides[1] = {(cuuint64_t)a.lda * es};
    cuuint32_t estr[2] = {1, 1};
    cuuint32_t boxc[2] = {(cuuint32_t)a.bw_c, (cuuint32_t)a.bh_c};
    cuuint32_t boxr[2] = {(cuuint32_t)a.bw_r, (cuuint32_t)a.tau_r};
    CUresult r1 = enc(&a.tmap_c, dt, 2, const_cast<void *>(a.A), dims, strides, boxc, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = enc(&a.tmap_r, dt, 2, const_cast<void *>(a.A), dims, strides, boxr, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) ? cudaSuccess : cudaErrorInvalidValue;
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

template <typename TA, typename TS, bool CORR, bool TMA> static void *kernel_ptr() {
    return reinterpret_cast<void *>(&rebk_grid_kernel<TA, TS, CORR, TMA>);
}

static void *mode_kernel(Mode mode, bool tma) {
    switch (mode) {
    case Mode::PlainF64: return kernel_ptr<double, double, false, false>();
    case Mode::CorrF32:
        return tma ? kernel_ptr<float, float, true, true>() : kernel_ptr<float, float, true, false>();
    default:
        return tma ? kernel_ptr<__nv_bfloat16, float, true, true>()
                   : kernel_ptr<__nv_bfloat16, float, true, false>();
    }
}

int grid_max_ctas(Mode mode, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *k = mode_kernel(mode, false);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kThreads, smem) != cudaSuccess) return 0;
    return sms * (per > 1 ? 1 : per);  // one CTA per SM
}

cudaError_t launch_grid(Mode mode, const GridArgs &a, int G, cudaStream_t st) {
    const size_t smem = grid_smem_bytes(mode, a);
    void *k = mode_kernel(mode, a.use_tma != 0);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    GridArgs copy = a;
    void *params[] = {&copy};
    return cudaLaunchCooperativeKernel(k, dim3(G), dim3(kThreads), params, smem, st);
}

}  // namespace rebk
