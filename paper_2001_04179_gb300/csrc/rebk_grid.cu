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
// Two chains on two warp groups.  The z iterates never read x, and the block
// indices do not depend on the data (counter-based Philox, sampled before the
// launch).  Each CTA therefore runs the column steps (the z chain) on kZWarps
// warps and the row steps (the x chain) on the other kXWarps warps, each group
// with its own named barrier and its own device-wide arrival counter:
//   z chain, step q: wait until every CTA's partial of w^q is in; z^q =
//       z^{q-1} - c_J A_{:,J_q} w^q on own rows; hand (z^q - b) on the own rows
//       of I_q to the x chain; partial of w^{q+1} = A_{R_c,J_{q+1}}^T z^q; arrive.
//   x chain, step p: take the hand-over of step p; partial of r^p =
//       A_{I_p,C_c} x^{p-1} (+ (z^p - b) on own rows, + a partial of
//       ||x^{p-1} - x_ref||^2 on test steps); arrive; wait until r^p is
//       complete; x^p = x^{p-1} - c_I A_{I_p,:}^T r^p on own columns.
// The device-wide round trip of one chain then overlaps the work of the other.
// The hand-over is a ring of kZRing slots with full / empty mbarriers, so the z
// chain runs at most kZRing steps ahead.  When the x chain stops at step p (the
// test on x^{p-1} passed), the z chain completes exactly step min(K, p + kZRing):
// the z written back does not depend on timing.
//
// Tile movement.  With TMA (FP32 / BF16 storage) each chain double-buffers its
// tiles (z chain: A_{R_c, J_q}; x chain: A_{I_p, C_c}) in shared memory; each
// 2-D tensor copy is issued as soon as its buffer has been used and waited on
// through an mbarrier with a bounded spin.  Without TMA (FP64 storage, whose
// tiles do not fit in shared memory) the tiles are read from global memory
// after line prefetches into L2 two steps ahead.
//
// Partial sums go to accumulators of the arithmetic type by atomic adds,
// replicated to spread contention; each chain rotates three accumulator sets so
// that the reads, writes and clearing of consecutive steps stay apart.
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

// Vector loads of V arithmetic-type values from shared memory (16-byte aligned).
__device__ __forceinline__ void lds_vec(const float *p, float (&t)[4]) {
    const float4 f = *reinterpret_cast<const float4 *>(p);
    t[0] = f.x; t[1] = f.y; t[2] = f.z; t[3] = f.w;
}
__device__ __forceinline__ void lds_vec(const float *p, float (&t)[8]) {
    const float4 f = *reinterpret_cast<const float4 *>(p), g = *reinterpret_cast<const float4 *>(p + 4);
    t[0] = f.x; t[1] = f.y; t[2] = f.z; t[3] = f.w;
    t[4] = g.x; t[5] = g.y; t[6] = g.z; t[7] = g.w;
}
__device__ __forceinline__ void lds_vec(const double *p, double (&t)[2]) {
    const double2 f = *reinterpret_cast<const double2 *>(p);
    t[0] = f.x; t[1] = f.y;
}

// Four consecutive atomic adds into global memory: one vector reduction when the
// address is 16-byte aligned (FP32), else four scalar ones.
__device__ __forceinline__ void red_add4(float *p, float a, float b, float c, float d) {
    if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0u) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                     : "memory");
    } else {
        atomicAdd(p, a);
        atomicAdd(p + 1, b);
        atomicAdd(p + 2, c);
        atomicAdd(p + 3, d);
    }
}
__device__ __forceinline__ void red_add4(double *p, double a, double b, double c, double d) {
    atomicAdd(p, a);
    atomicAdd(p + 1, b);
    atomicAdd(p + 2, c);
    atomicAdd(p + 3, d);
}

// Sum of the R replicas of one accumulator entry (fixed pairwise order).
template <int R, typename TS> __device__ __forceinline__ TS sum_replicas(const TS *p, int aw) {
    TS v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = ld_cg_t(p + (int64_t)q * aw);
#pragma unroll
    for (int h = R / 2; h > 0; h >>= 1)
#pragma unroll
        for (int q = 0; q < h; ++q) v[q] += v[q + h];
    return v[0];
}

// out(row) = sum_{c in [ca, cb)} A[row, c] * vin[c - ca] for rows [ra, rb), by
// a group of NT threads (gt = thread index in the group).  A addresses element
// (r, c) at A + r * lda + c.  Rows go to lane groups of gs lanes (gs in 4..32,
// chosen to minimise passes x vector loads per lane, then passes); each lane
// group handles 4 consecutive rows per pass and hands them to emit4(r, v0..v3)
// from one lane (emit(r, v) for the rows of an incomplete quad).
template <int NT, typename TA, typename TS, bool SM, typename Emit, typename Emit4>
__device__ __forceinline__ void row_dots(int gt, const TA *A, int64_t lda, int64_t ra, int64_t rb,
                                         int64_t ca, int64_t cb, const TS *__restrict__ vin, Emit emit,
                                         Emit4 emit4) {
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    constexpr int U = 4;
    constexpr int NW = NT / 32;
    if (rb <= ra || cb <= ca) return;
    const int64_t va = ca / V, vb = (cb + V - 1) / V;
    const int nv = (int)(vb - va);
    const int nr = (int)(rb - ra);
    int gs = 4;
    {
        int best = 0x7fffffff;
#pragma unroll
        for (int lc = 2; lc <= 5; ++lc) {  // gs = 1 << lc; divisions by constants only
            const int c = 1 << lc;
            const int rows_per_pass = NW * (32 >> lc) * U;
            const int passes = (nr + rows_per_pass - 1) / rows_per_pass;
            const int cost = passes * (((nv + c - 1) >> lc) * 8 + 1);
            if (cost < best) {
                best = cost;
                gs = c;
            }
        }
    }
    const int lane = gt & 31, warp = gt >> 5;
    const int sub = lane & (gs - 1);
    const int gpw = 32 / gs;
    const int g = warp * gpw + lane / gs;
    const int NG = NW * gpw;
    for (int64_t base = ra; base < rb; base += (int64_t)NG * U) {
        const int64_t rq = base + (int64_t)U * g;  // this lane group's quad
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
                const int64_t r = rq + u;
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
        {
            int ru = 0;
            const TS v = group_reduce4<TS>(acc, gs, sub, &ru);
            // lanes sub = 0, gs/4, gs/2, 3gs/4 hold rows rq + 0, 1, 2, 3
            const int q4 = gs >> 2;
            const TS v1 = __shfl_down_sync(0xffffffffu, v, q4);
            const TS v2 = __shfl_down_sync(0xffffffffu, v, 2 * q4);
            const TS v3 = __shfl_down_sync(0xffffffffu, v, 3 * q4);
            if (sub == 0) {
                if (rq + 3 < rb) {
                    emit4(rq, v, v1, v2, v3);
                } else {
                    if (rq < rb) emit(rq, v);
                    if (rq + 1 < rb) emit(rq + 1, v1);
                    if (rq + 2 < rb) emit(rq + 2, v2);
                }
            }
        }
    }
}

// out(col) = sum_{r in [ra, rb)} A[r, col] * vrow[r - ra] for columns [ca, cb),
// by a group of NT threads synchronised by sync().  Threads are laid out as
// (vector index, row group); each thread sums its vector over its rows, then the
// row groups are added through shared memory (red: NT * V elements), one thread
// per vector, which hands each quad of columns inside [ca, cb) to
// emit4(col, v0..v3) and the other columns to emit(col, v).
template <int NT, typename TA, typename TS, bool SM, typename Sync, typename Emit, typename Emit4>
__device__ __forceinline__ void col_sums(int gt, const TA *A, int64_t lda, int64_t ra, int64_t rb,
                                         int64_t ca, int64_t cb, const TS *__restrict__ vrow, TS *red,
                                         Sync sync, Emit emit, Emit4 emit4) {
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    constexpr int U = 4;
    if (rb <= ra || cb <= ca) return;
    const int64_t va = ca / V, vb = (cb + V - 1) / V;
    const int nv = (int)(vb - va);
    for (int vc0 = 0; vc0 < nv; vc0 += NT) {
        const int nvc = min(NT, nv - vc0);
        const int NRG = NT / nvc;
        const int vi = gt % nvc, rg = gt / nvc;
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
        sync();
        for (int c = gt; c < nvc; c += NT) {
            TS sum[V];
#pragma unroll
            for (int e = 0; e < V; ++e) sum[e] = tzero<TS>();
            for (int q = 0; q < NRG; ++q) {
                TS t[V];
                lds_vec(red + q * (nvc * V) + c * V, t);
#pragma unroll
                for (int e = 0; e < V; ++e) sum[e] += t[e];
            }
            const int64_t col0 = (va + vc0 + c) * V;
#pragma unroll
            for (int e4 = 0; e4 < V; e4 += 4) {
                if (V >= 4 && col0 + e4 >= ca && col0 + e4 + 3 < cb) {
                    emit4(col0 + e4, sum[e4], sum[(e4 + 1) % V], sum[(e4 + 2) % V], sum[(e4 + 3) % V]);
                } else {
#pragma unroll
                    for (int e = e4; e < e4 + 4 && e < V; ++e) {
                        const int64_t col = col0 + e;
                        if (col >= ca && col < cb) emit(col, sum[e]);
                    }
                }
            }
        }
        sync();
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// Tile products.  T: rows of ld elements, nvec 16-byte vectors per row, either a
// TMA-staged tile in shared memory (SM: 32-bit shared addresses) or a strided
// view of A in global memory (read-only path, more loads in flight).
// ---------------------------------------------------------------------------

// out(l) = sum_{t < nvec * V} T[l * ld + t] * vin[t] for rows l in [0, rows);
// vin (shared memory) holds nvec * V values, zero where the range has no column.
// Lane groups of gs lanes take 4 consecutive rows; emit4(l, v0..v3) for full
// quads, emit(l, v) for the rows of the last, incomplete one.
template <int NT, bool SM, typename TA, typename TS, typename Emit, typename Emit4>
__device__ __forceinline__ void tile_rowdot(int gt, const TA *T, int64_t ld, int rows, int nvec,
                                            const TS *vin, Emit emit, Emit4 emit4) {
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    constexpr int NW = NT / 32;
    if (rows <= 0 || nvec <= 0) return;
    int gs = 4;
    {
        int best = 0x7fffffff;
#pragma unroll
        for (int lc = 2; lc <= 5; ++lc) {
            const int rows_per_pass = NW * (32 >> lc) * 4;
            const int passes = (rows + rows_per_pass - 1) / rows_per_pass;
            const int cost = passes * ((((nvec + (1 << lc) - 1) >> lc)) * 8 + 1);
            if (cost < best) {
                best = cost;
                gs = 1 << lc;
            }
        }
    }
    const int lane = gt & 31, warp = gt >> 5;
    const int sub = lane & (gs - 1);
    const int g = warp * (32 / gs) + lane / gs;
    const int NG = NW * (32 / gs);
    const uint32_t vb = smem_u32(vin);
    // the pass loop is uniform over the warp (every lane takes part in the shuffles)
    for (int base = 0; base < rows; base += 4 * NG) {
        const int rq = base + 4 * g;
        const bool ok0 = rq < rows, ok1 = rq + 1 < rows, ok2 = rq + 2 < rows, ok3 = rq + 3 < rows;
        TS acc0 = tzero<TS>(), acc1 = tzero<TS>(), acc2 = tzero<TS>(), acc3 = tzero<TS>();
        uint32_t xa = vb + (uint32_t)sub * (uint32_t)(V * sizeof(TS));
        auto body = [&](const TS (&xv)[V], const TS (&t0)[V], const TS (&t1)[V], const TS (&t2)[V],
                        const TS (&t3)[V]) {
#pragma unroll
            for (int e = 0; e < V; ++e) {
                acc0 = fma(t0[e], xv[e], acc0);
                acc1 = fma(t1[e], xv[e], acc1);
                acc2 = fma(t2[e], xv[e], acc2);
                acc3 = fma(t3[e], xv[e], acc3);
            }
        };
        if constexpr (SM) {
            const uint32_t row_bytes = (uint32_t)ld * (uint32_t)sizeof(TA);
            uint32_t a = smem_u32(T) + (uint32_t)rq * row_bytes + (uint32_t)sub * 16u;
#pragma unroll 2
            for (int vi = ok0 ? sub : nvec; vi < nvec; vi += gs) {
                TS xv[V], t0[V], t1[V], t2[V], t3[V];
                IO::load_shared_ts(xa, xv);
                IO::load_shared(a, t0);
                if (ok1) IO::load_shared(a + row_bytes, t1); else IO::zero(t1);
                if (ok2) IO::load_shared(a + 2 * row_bytes, t2); else IO::zero(t2);
                if (ok3) IO::load_shared(a + 3 * row_bytes, t3); else IO::zero(t3);
                body(xv, t0, t1, t2, t3);
                a += (uint32_t)gs * 16u;
                xa += (uint32_t)(gs * V * sizeof(TS));
            }
        } else {
            const TA *a = T + (int64_t)rq * ld + (int64_t)sub * V;
            constexpr int UR = V == 2 ? 3 : 1;  // chunks of loads in flight (register budget)
#pragma unroll UR
            for (int vi = ok0 ? sub : nvec; vi < nvec; vi += gs) {
                TS xv[V], t0[V], t1[V], t2[V], t3[V];
                IO::load(a, t0);
                if (ok1) IO::load(a + ld, t1); else IO::zero(t1);
                if (ok2) IO::load(a + 2 * ld, t2); else IO::zero(t2);
                if (ok3) IO::load(a + 3 * ld, t3); else IO::zero(t3);
                IO::load_shared_ts(xa, xv);
                body(xv, t0, t1, t2, t3);
                a += (int64_t)gs * V;
                xa += (uint32_t)(gs * V * sizeof(TS));
            }
        }
        TS acc[4] = {acc0, acc1, acc2, acc3};
        int ru = 0;
        const TS v = group_reduce4<TS>(acc, gs, sub, &ru);
        const int q4 = gs >> 2;
        const TS v1 = __shfl_down_sync(0xffffffffu, v, q4);
        const TS v2 = __shfl_down_sync(0xffffffffu, v, 2 * q4);
        const TS v3 = __shfl_down_sync(0xffffffffu, v, 3 * q4);
        if (sub == 0 && ok0) {
            if (ok3) {
                emit4(rq, v, v1, v2, v3);
            } else {
                emit(rq, v);
                if (ok1) emit(rq + 1, v1);
                if (ok2) emit(rq + 2, v2);
            }
        }
    }
}

// out(vector t) = sum_{l < rows} T[l * ld + t * V + e] * vrow[l], e < V, for the
// nvec vectors t of a row, by a group of NT threads synchronised by sync();
// threads are (vector, row group) pairs whose partial sums meet in red (NT * V
// values).  emitv(t, sum[V]) once per vector.
template <int NT, bool SM, typename TA, typename TS, typename Sync, typename EmitV>
__device__ __forceinline__ void tile_colsum(int gt, const TA *T, int64_t ld, int rows, int nvec,
                                            const TS *vrow, TS *red, Sync sync, EmitV emitv) {
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    if (rows <= 0 || nvec <= 0) return;
    for (int vc0 = 0; vc0 < nvec; vc0 += NT) {
        const int nvc = min(NT, nvec - vc0);
        const int NRG = NT / nvc;
        const int vi = gt % nvc, rg = gt / nvc;
        if (rg < NRG) {
            TS acc[V];
#pragma unroll
            for (int e = 0; e < V; ++e) acc[e] = tzero<TS>();
            if constexpr (SM) {
                const uint32_t row_bytes = (uint32_t)ld * (uint32_t)sizeof(TA);
                uint32_t a = smem_u32(T) + (uint32_t)rg * row_bytes + (uint32_t)(vc0 + vi) * 16u;
                const uint32_t step = (uint32_t)NRG * row_bytes;
#pragma unroll 4
                for (int l = rg; l < rows; l += NRG) {
                    TS t[V];
                    IO::load_shared(a, t);
                    const TS xr = vrow[l];
#pragma unroll
                    for (int e = 0; e < V; ++e) acc[e] = fma(t[e], xr, acc[e]);
                    a += step;
                }
            } else {
                const TA *a = T + (int64_t)rg * ld + (int64_t)(vc0 + vi) * V;
                const int64_t step = (int64_t)NRG * ld;
                constexpr int UR = V == 2 ? 8 : 4;
#pragma unroll UR
                for (int l = rg; l < rows; l += NRG) {
                    TS t[V];
                    IO::load(a, t);
                    const TS xr = vrow[l];
#pragma unroll
                    for (int e = 0; e < V; ++e) acc[e] = fma(t[e], xr, acc[e]);
                    a += step;
                }
            }
            TS *dst = red + (rg * nvc + vi) * V;
#pragma unroll
            for (int e = 0; e < V; ++e) dst[e] = acc[e];
        }
        sync();
        for (int c = gt; c < nvc; c += NT) {
            TS sum[V];
            lds_vec(red + c * V, sum);
            for (int q = 1; q < NRG; ++q) {
                TS t[V];
                lds_vec(red + (q * nvc + c) * V, t);
#pragma unroll
                for (int e = 0; e < V; ++e) sum[e] += t[e];
            }
            emitv(vc0 + c, sum);
        }
        sync();
    }
}

template <typename T> __device__ __forceinline__ bool finite_val(T v) { return isfinite(v); }

// ---------------------------------------------------------------------------
// Named barriers, shared-memory flags, TMA / mbarrier helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ int ld_vol(const int *p) { return *reinterpret_cast<const volatile int *>(p); }
__device__ __forceinline__ void st_vol(int *p, int v) { *reinterpret_cast<volatile int *>(p) = v; }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One arrival (release at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Non-blocking test: has the phase with this parity completed (acquire at CTA scope)?
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
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

// Leader-side bounded poll: 0 once ready() holds; the nonzero code of quit() if
// that comes first; 6 (REBK_BARRIER_TIMEOUT) once timeout_ns have passed.
template <typename Ready, typename Quit>
__device__ __forceinline__ int lead_poll(Ready ready, Quit quit, unsigned long long timeout_ns) {
    if (ready()) return 0;
    const unsigned long long t0 = globaltimer_ns();
    for (uint32_t spins = 1;; ++spins) {
        const int q = quit();
        if (q != 0) return q;
        if (ready()) return 0;
        if ((spins & 63u) == 0u && globaltimer_ns() - t0 > timeout_ns) return 6;
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

// Shared-memory header (byte offsets below kSmemHeader).
constexpr int kHdrRingJ = 0;      // int[kRing]  z chain: J_k
constexpr int kHdrRingZI = 32;    // int[kRing]  z chain: I_k (rows handed over)
constexpr int kHdrRingXI = 64;    // int[kRing]  x chain: I_k
constexpr int kHdrZF = 96;        // int[4]      z-chain flags
constexpr int kHdrXF = 112;       // int[4]      x-chain flags
constexpr int kHdrCtl = 128;      // int[4]      [0] stop code (0, 1 converged, 5, 6), [1] stop step
constexpr int kHdrMbarC = 160;    // u64[2]      column tiles
constexpr int kHdrMbarR = 176;    // u64[2]      row tiles
constexpr int kHdrZFull = 192;    // u64[kZRing] hand-over slot written
constexpr int kHdrZEmpty = 224;   // u64[kZRing] hand-over slot consumed
constexpr int kHdrRingCJ = 256;   // TS[kRing]   z chain: alpha / ||A_{:,J_k}||^2
constexpr int kHdrRingCI = 320;   // TS[kRing]   x chain: alpha / ||A_{I_k,:}||^2
static_assert(kRing == 8 && kZRing <= 4 && kHdrRingCI + 64 <= (int)kSmemHeader, "header layout");

}  // namespace

template <typename TA, typename TS, bool CORR, bool TMA>
__global__ void __launch_bounds__(kThreads, 1) rebk_grid_kernel(const __grid_constant__ GridArgs args) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    using IO = VecIO<TA, TS>;
    constexpr int V = IO::V;
    constexpr int ZT = kZThreads, XT = kXThreads;
    constexpr int64_t ZR = kZRing;

    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
    const TA *__restrict__ A = static_cast<const TA *>(args.A);
    const int64_t m = args.m, n = args.n, lda = args.lda;
    const int64_t nu = (n + 7) / 8;
    const int64_t r0 = m * cta / G, r1 = m * (cta + 1) / G;
    const int64_t c0 = lmin(n, 8 * (nu * cta / G)), c1 = lmin(n, 8 * (nu * (cta + 1) / G));
    const int nrow = (int)(r1 - r0), ncol = (int)(c1 - c0);
    const int64_t K = args.iters;
    const int64_t tau_r = args.tau_r;

    // ---- shared memory carve-up (same layout as grid_smem_bytes()) ----
    const SmemLayout L = smem_layout(args.nrow_cap, args.ncol_cap, args.tau_r, args.tau_c, CORR,
                                     (int)sizeof(TS), V, TMA ? args.tile_c_bytes : 0,
                                     TMA ? args.tile_r_bytes : 0);
    int *ring_j = reinterpret_cast<int *>(smem_raw + kHdrRingJ);
    int *ring_zi = reinterpret_cast<int *>(smem_raw + kHdrRingZI);
    int *ring_xi = reinterpret_cast<int *>(smem_raw + kHdrRingXI);
    int *zf = reinterpret_cast<int *>(smem_raw + kHdrZF);  // [0] wait code, [1] non-finite w, [2] tile wait failed
    int *xf = reinterpret_cast<int *>(smem_raw + kHdrXF);  // [0] wait code, [1] test passed, [2] tile, [3] non-finite r
    int *ctl = reinterpret_cast<int *>(smem_raw + kHdrCtl);
    uint64_t *mbar_c = reinterpret_cast<uint64_t *>(smem_raw + kHdrMbarC);
    uint64_t *mbar_r = reinterpret_cast<uint64_t *>(smem_raw + kHdrMbarR);
    uint64_t *zfull = reinterpret_cast<uint64_t *>(smem_raw + kHdrZFull);
    uint64_t *zempty = reinterpret_cast<uint64_t *>(smem_raw + kHdrZEmpty);
    TS *ring_cj = reinterpret_cast<TS *>(smem_raw + kHdrRingCJ);
    TS *ring_ci = reinterpret_cast<TS *>(smem_raw + kHdrRingCI);
    TS *zeta = reinterpret_cast<TS *>(smem_raw + L.zeta);
    TS *beta_own = reinterpret_cast<TS *>(smem_raw + L.beta);
    TS *v_own = reinterpret_cast<TS *>(smem_raw + L.v);    // CORR only
    TS *xi = reinterpret_cast<TS *>(smem_raw + L.xi);
    TS *s_own = reinterpret_cast<TS *>(smem_raw + L.s);    // CORR only
    TS *w = reinterpret_cast<TS *>(smem_raw + L.w);
    TS *rr = reinterpret_cast<TS *>(smem_raw + L.r);
    TS *zr = reinterpret_cast<TS *>(smem_raw + L.zr);      // kZRing slots of tau_r
    TS *redz = reinterpret_cast<TS *>(smem_raw + L.redz);
    TS *redx = reinterpret_cast<TS *>(smem_raw + L.redx);
    auto tile_c = [&](int b) { return reinterpret_cast<TA *>(smem_raw + (b ? L.tc1 : L.tc0)); };
    auto tile_r = [&](int b) { return reinterpret_cast<TA *>(smem_raw + (b ? L.tr1 : L.tr0)); };

    TS *gz = static_cast<TS *>(args.z);
    TS *gx = static_cast<TS *>(args.x);
    TS *gs_dual = static_cast<TS *>(args.sdual);
    TS *gv_dual = static_cast<TS *>(args.vdual);
    const TS *coef_r = static_cast<const TS *>(args.coef_r);
    const TS *coef_c = static_cast<const TS *>(args.coef_c);
    const int32_t *idx = args.idx;

    // ---- state, index rings, barriers ----
    for (int i = tid; i < nrow; i += kThreads) {
        zeta[i] = gz[r0 + i];
        beta_own[i] = (TS)args.beta[r0 + i];
        if (CORR) v_own[i] = gv_dual[r0 + i];
    }
    for (int j = tid; j < ncol; j += kThreads) {
        xi[j] = gx[c0 + j];
        if (CORR) s_own[j] = gs_dual[c0 + j];
    }
    // x is read over whole row-tile rows: zero beyond the owned columns
    const int xpad = (args.ncol_cap + 7) / 8 * 8;
    for (int j = ncol + tid; j < xpad; j += kThreads) xi[j] = tzero<TS>();
    if (tid == 0) {
        for (int64_t k = 1; k <= 4 && k <= K; ++k) {
            const int j = __ldg(idx + 2 * (k - 1)), i = __ldg(idx + 2 * (k - 1) + 1);
            ring_j[k % kRing] = j;
            ring_zi[k % kRing] = i;
            ring_xi[k % kRing] = i;
            ring_cj[k % kRing] = coef_c[j];
            ring_ci[k % kRing] = coef_r[i];
        }
        for (int q = 0; q < 4; ++q) {
            zf[q] = 0;
            xf[q] = 0;
            ctl[q] = 0;
        }
        mbar_init(&mbar_c[0], 1);
        mbar_init(&mbar_c[1], 1);
        mbar_init(&mbar_r[0], 1);
        mbar_init(&mbar_r[1], 1);
        for (int q = 0; q < kZRing; ++q) {
            mbar_init(&zfull[q], 1);
            mbar_init(&zempty[q], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // replicas per accumulator entry: kAccReplicas (corrections), kAccReplicasF64 (plain FP64),
    // the same count acc_replicas() gives the host
    constexpr int RP = CORR ? kAccReplicas : kAccReplicasF64;
    const int rep = cta % RP;
    const int aw = args.acc_w;
    const int64_t accset = (int64_t)RP * aw;
    TS *accw_base = static_cast<TS *>(args.acc);   // w partials: 3 sets
    TS *accr_base = accw_base + 3 * accset;        // r partials (+ test partial at tau_r): 3 sets
    const bool check = args.x_ref != nullptr && args.check_every > 0;
    // Column blocks whose starts are all multiples of calign elements: the
    // contiguous partition's starts are multiples of tau_c (of its lowest set
    // bit), a given partition's of args.col_align.
    const int calign = args.col_off ? args.col_align : (args.tau_c & -args.tau_c);
    // column tiles start exactly at their block (every start on a 16-byte boundary)
    const bool fast_c = TMA && calign % args.tma_vx == 0;
    // global-memory column views start on a 16-byte vector (rows are 16-byte aligned)
    const bool fast_g = !TMA && calign % V == 0;
    const int wpad = (args.tau_c + 7) / 8 * 8;
    // Any CTA past the arrivals of step q may clear a set that step q + 1 fills:
    // every CTA has read it (step q - 1) before arriving, and nobody adds to it
    // before every CTA has arrived once more.  Each CTA clears a 1/G share.
    const int64_t clr0 = accset * cta / G, clr1 = accset * (cta + 1) / G;

    // block j of the columns / i of the rows: [off[j], off[j+1]) of a given
    // partition, else the contiguous blocks of tau_c / tau_r (Algorithm 1's
    // J_j and I_i)
    const int64_t *__restrict__ col_off = args.col_off;
    const int64_t *__restrict__ row_off = args.row_off;
    auto col_range = [&](int j, int64_t *a, int64_t *b) {
        if (col_off) {
            *a = __ldg(col_off + j);
            *b = __ldg(col_off + j + 1);
        } else {
            *a = (int64_t)j * args.tau_c;
            *b = lmin(n, *a + args.tau_c);
        }
    };
    auto row_range = [&](int i, int64_t *a, int64_t *b) {
        if (row_off) {
            *a = __ldg(row_off + i);
            *b = __ldg(row_off + i + 1);
        } else {
            *a = (int64_t)i * tau_r;
            *b = lmin(m, *a + tau_r);
        }
    };
    // a wait gave up after its time limit: record it for the host and for the other group
    auto give_up = [&](int code) {
        if (code == 6) atomicExch(args.status, 6);
        if (code == 5) atomicExch(args.status, 5);
        atomicCAS(&ctl[0], 0, code);
    };

    if (tid < ZT) {
        // =================== z chain: column steps ===================
        const int gt = tid;
        auto zsync = [&]() { named_sync(1, ZT); };

        // index ring: entry k = q + 4 is written at step q from registers loaded
        // one (coefficient) and two (indices) steps earlier
        int ld_j1 = 0, ld_i1 = 0, ld_j2 = 0, ld_i2 = 0;
        TS ld_c1 = tzero<TS>();
        if (gt == ZT - 1) {
            if (K >= 5) {
                ld_j1 = __ldg(idx + 8);
                ld_i1 = __ldg(idx + 9);
                ld_c1 = coef_c[ld_j1];
            }
            if (K >= 6) {
                ld_j2 = __ldg(idx + 10);
                ld_i2 = __ldg(idx + 11);
            }
        }
        auto loader = [&](int64_t q) {
            if (gt != ZT - 1) return;
            if (q + 4 <= K) {
                ring_j[(q + 4) % kRing] = ld_j1;
                ring_zi[(q + 4) % kRing] = ld_i1;
                ring_cj[(q + 4) % kRing] = ld_c1;
            }
            if (q + 5 <= K) {
                ld_j1 = ld_j2;
                ld_i1 = ld_i2;
                ld_c1 = coef_c[ld_j2];
            }
            if (q + 6 <= K) {
                ld_j2 = __ldg(idx + 2 * (q + 5));
                ld_i2 = __ldg(idx + 2 * (q + 5) + 1);
            }
        };

        // column tile of J_q (own rows) in buffer q % 2
        uint32_t cpar0 = 0u, cpar1 = 0u;
        bool cpend0 = false, cpend1 = false;
        int xc0 = 0, xc1 = 0;  // x origin of each buffer's copy
        auto issue_col = [&](int64_t q) {
            if (!TMA || q < 1 || q > K || nrow == 0) return;
            const int b = (int)(q & 1);
            int64_t ja, jb;
            col_range(ring_j[q % kRing], &ja, &jb);
            const int x0 = (int)(ja & ~(int64_t)(args.tma_vx - 1));  // tma_vx is 4 or 8
            if (b) { xc1 = x0; cpend1 = true; } else { xc0 = x0; cpend0 = true; }
            if (gt == 0) {
                fence_proxy_async();
                mbar_expect_tx(&mbar_c[b], (uint32_t)args.tile_c_bytes_tx);
                for (int bx = 0; bx < args.nbox_c; ++bx)
                    tma_load_2d(tile_c(b) + (size_t)bx * args.bh_c * args.bw_c, &args.tmap_c, x0,
                                (int)(r0 + (int64_t)bx * args.bh_c), &mbar_c[b]);
            }
        };
        auto wait_col = [&](int64_t q) -> bool {
            const int b = (int)(q & 1);
            const bool pend = b ? cpend1 : cpend0;
            if (!pend) return true;
            const bool ok = mbar_wait(&mbar_c[b], b ? cpar1 : cpar0, args.timeout_ns);
            if (b) { cpar1 ^= 1u; cpend1 = false; } else { cpar0 ^= 1u; cpend0 = false; }
            return ok;
        };
        auto ctile = [&](int64_t q, int64_t *ld) -> const TA * {
            if (!TMA) {
                *ld = lda;
                return A;
            }
            const int b = (int)(q & 1);
            *ld = args.bw_c;
            return tile_c(b) - r0 * (int64_t)args.bw_c - (b ? xc1 : xc0);
        };
        auto prefetch_col = [&](int64_t q) {  // no-TMA path: L2 line prefetch
            if (TMA || q < 1 || q > K || nrow == 0) return;
            constexpr int64_t LINE = 128 / sizeof(TA);
            int64_t ja, jb;
            col_range(ring_j[q % kRing], &ja, &jb);
            const int64_t l0 = ja / LINE;
            const int nl = (int)((jb + LINE - 1) / LINE - l0);
            for (int e = gt; e < nrow * nl; e += ZT) {
                const int rr_ = e / nl, l = e - rr_ * nl;
                prefetch_line(A + (r0 + rr_) * lda + (l0 + l) * LINE);
            }
        };
        auto partial_w = [&](int64_t q, TS *accp) {  // over own rows, column block J_q, with zeta
            int64_t ja, jb, ld;
            col_range(ring_j[q % kRing], &ja, &jb);
            const int wc = (int)(jb - ja);
            auto emitv = [&](int t, const TS(&sum)[V]) {
                if constexpr (V >= 4) {
#pragma unroll
                    for (int e4 = 0; e4 < V; e4 += 4) {
                        const int c = t * V + e4;
                        if (c + 3 < wc) {
                            red_add4(accp + c, sum[e4], sum[e4 + 1], sum[e4 + 2], sum[e4 + 3]);
                        } else {
                            for (int e = 0; e < 4; ++e)
                                if (c + e < wc) atomicAdd(accp + c + e, sum[e4 + e]);
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (t * V + e < wc) atomicAdd(accp + t * V + e, sum[e]);
                }
            };
            if constexpr (TMA) {
                if (fast_c) {
                    tile_colsum<ZT, true, TA, TS>(gt, tile_c((int)(q & 1)), args.bw_c, nrow, args.bw_c / V, zeta,
                                                  redz, zsync, emitv);
                    return;
                }
            } else {
                if (fast_g) {
                    tile_colsum<ZT, false, TA, TS>(gt, A + r0 * lda + ja, lda, nrow, (wc + V - 1) / V, zeta, redz,
                                                   zsync, emitv);
                    return;
                }
            }
            const TA *T = ctile(q, &ld);
            col_sums<ZT, TA, TS, TMA>(
                gt, T, ld, r0, r1, ja, jb, zeta, redz, zsync,
                [&](int64_t col, TS v) { atomicAdd(accp + (col - ja), v); },
                [&](int64_t col, TS v0, TS v1, TS v2, TS v3) { red_add4(accp + (col - ja), v0, v1, v2, v3); });
        };
        // stop signal for the z chain at step q: 5 / 6 at once; after a converged
        // stop of the x chain at step p, once q > min(K, p + kZRing)
        auto quit_z = [&](int64_t q) -> int {
            const int c = ld_vol(&ctl[0]);
            if (c == 5 || c == 6) return c;
            if (c == 1) {
                __threadfence_block();
                if (q > lmin(K, (int64_t)ld_vol(&ctl[1]) + ZR)) return 1;
            }
            return 0;
        };

        bool alive = K >= 1;
        if (alive) {
            issue_col(1);
            issue_col(2);
            prefetch_col(1);
            prefetch_col(2);
            if (!wait_col(1)) zf[2] = 1;
            zsync();
            if (zf[2] != 0) {
                if (gt == 0) give_up(6);
                alive = false;
            } else {
                partial_w(1, accw_base + (int64_t)rep * aw);
                zsync();
                if (gt == 0) red_release_gpu_add(args.bar, 1u);
            }
        }
        for (int64_t q = 1; alive && q <= K; ++q) {
            loader(q);
            if (gt == 0) {
                int code = lead_poll([&] { return ld_acquire_gpu(args.bar) >= (unsigned)G * (unsigned)q; },
                                     [&] { return quit_z(q); }, args.timeout_ns);
                if (code == 0 && q > ZR) {  // hand-over slot of step q - kZRing consumed
                    const uint32_t par = (uint32_t)(((q - 1) / ZR - 1) & 1);
                    code = lead_poll([&] { return mbar_test(&zempty[(q - 1) % ZR], par); },
                                     [&] { return quit_z(q); }, args.timeout_ns);
                }
                if (code == 6) give_up(6);
                zf[0] = code;
            }
            zsync();
            if (zf[0] != 0) break;

            // w^q = sum of the replicas (+ g_J in the correction form)
            const int jq = ring_j[q % kRing];
            int64_t ja, jb;
            col_range(jq, &ja, &jb);
            const int wc = (int)(jb - ja);
            const TS *accq = accw_base + ((q - 1) % 3) * accset;
            for (int t = gt; t < wpad; t += ZT) {
                if (t >= wc) {  // the z update reads w over whole tile rows
                    w[t] = tzero<TS>();
                    continue;
                }
                TS sum = sum_replicas<RP>(accq + t, aw);
                if (CORR) sum += (TS)args.gamma[ja + t];
                w[t] = sum;
                if (!finite_val(sum)) zf[1] = 1;
            }
            zsync();
            if (zf[1] != 0) {
                if (gt == 0) give_up(5);
                break;
            }
            // z^q on own rows; hand (z^q - b) on own rows of I_q to the x chain
            const TS cJ = ring_cj[q % kRing];
            int64_t ia, ib;
            row_range(ring_zi[q % kRing], &ia, &ib);
            TS *zslot = zr + ((q - 1) % ZR) * tau_r;
            {
                auto upd = [&](int64_t row, TS v) {
                    const TS nz = zeta[row - r0] - cJ * v;
                    zeta[row - r0] = nz;
                    if (row >= ia && row < ib) zslot[row - ia] = nz - beta_own[row - r0];
                };
                auto upd4 = [&](int64_t row, TS v0, TS v1, TS v2, TS v3) {
                    upd(row, v0);
                    upd(row + 1, v1);
                    upd(row + 2, v2);
                    upd(row + 3, v3);
                };
                bool done_fast = false;
                auto e1 = [&](int l, TS v) { upd(r0 + l, v); };
                auto e4 = [&](int l, TS v0, TS v1, TS v2, TS v3) { upd4(r0 + l, v0, v1, v2, v3); };
                if constexpr (TMA) {
                    if (fast_c) {
                        tile_rowdot<ZT, true, TA, TS>(gt, tile_c((int)(q & 1)), args.bw_c, nrow, args.bw_c / V, w, e1,
                                                      e4);
                        done_fast = true;
                    }
                } else {
                    if (fast_g) {  // w is zero from wc up to a multiple of 8
                        tile_rowdot<ZT, false, TA, TS>(gt, A + r0 * lda + ja, lda, nrow, (wc + V - 1) / V, w, e1, e4);
                        done_fast = true;
                    }
                }
                if (!done_fast) {
                    int64_t ld;
                    const TA *T = ctile(q, &ld);
                    row_dots<ZT, TA, TS, TMA>(gt, T, ld, r0, r1, ja, jb, w, upd, upd4);
                }
            }
            if (CORR) {
                const int64_t la = lmax(ja, c0), lb = lmin(jb, c1);
                for (int64_t l = la + gt; l < lb; l += ZT) s_own[l - c0] += cJ * w[l - ja];
            }
            zsync();
            if (gt == 0) mbar_arrive(&zfull[(q - 1) % ZR]);
            // column tile of J_q is used up: its buffer takes J_{q+2}
            issue_col(q + 2);
            prefetch_col(q + 2);
            if (q < K) {
                if (!wait_col(q + 1)) zf[2] = 1;
                zsync();
                if (zf[2] != 0) {
                    if (gt == 0) give_up(6);
                    break;
                }
                partial_w(q + 1, accw_base + (q % 3) * accset + (int64_t)rep * aw);
                {  // clear this CTA's share of the set read two steps ahead
                    TS *accz = accw_base + ((q + 1) % 3) * accset;
                    for (int64_t e = clr0 + gt; e < clr1; e += ZT) accz[e] = tzero<TS>();
                }
                zsync();
                if (gt == 0) red_release_gpu_add(args.bar, 1u);
            }
        }
        // no tensor copy may still be writing shared memory when the group leaves
        if (TMA) {
            wait_col(0);
            wait_col(1);
        }
        for (int i = gt; i < nrow; i += ZT) gz[r0 + i] = zeta[i];
        if (CORR)
            for (int j = gt; j < ncol; j += ZT) gs_dual[c0 + j] = s_own[j];
    } else {
        // =================== x chain: row steps ===================
        const int gt = tid - ZT;
        auto xsync = [&]() { named_sync(2, XT); };

        int ld_i1 = 0, ld_i2 = 0;
        TS ld_c1 = tzero<TS>();
        if (gt == XT - 1) {
            if (K >= 5) {
                ld_i1 = __ldg(idx + 9);
                ld_c1 = coef_r[ld_i1];
            }
            if (K >= 6) ld_i2 = __ldg(idx + 11);
        }
        auto loader = [&](int64_t p) {
            if (gt != XT - 1) return;
            if (p + 4 <= K) {
                ring_xi[(p + 4) % kRing] = ld_i1;
                ring_ci[(p + 4) % kRing] = ld_c1;
            }
            if (p + 5 <= K) {
                ld_i1 = ld_i2;
                ld_c1 = coef_r[ld_i2];
            }
            if (p + 6 <= K) ld_i2 = __ldg(idx + 2 * (p + 5) + 1);
        };

        // row tile of I_p (own columns) in buffer p % 2
        uint32_t rpar0 = 0u, rpar1 = 0u;
        bool rpend0 = false, rpend1 = false;
        auto issue_row = [&](int64_t p) {
            if (!TMA || p < 1 || p > K || ncol == 0) return;
            const int b = (int)(p & 1);
            if (b) rpend1 = true; else rpend0 = true;
            if (gt == 0) {
                int64_t ia, ib;
                row_range(ring_xi[p % kRing], &ia, &ib);
                fence_proxy_async();
                mbar_expect_tx(&mbar_r[b], (uint32_t)args.tile_r_bytes_tx);
                tma_load_2d(tile_r(b), &args.tmap_r, (int)c0, (int)ia, &mbar_r[b]);
            }
        };
        auto wait_row = [&](int64_t p) -> bool {
            const int b = (int)(p & 1);
            const bool pend = b ? rpend1 : rpend0;
            if (!pend) return true;
            const bool ok = mbar_wait(&mbar_r[b], b ? rpar1 : rpar0, args.timeout_ns);
            if (b) { rpar1 ^= 1u; rpend1 = false; } else { rpar0 ^= 1u; rpend0 = false; }
            return ok;
        };
        auto rtile = [&](int64_t p, int64_t ia, int64_t *ld) -> const TA * {
            if (!TMA) {
                *ld = lda;
                return A;
            }
            *ld = args.bw_r;
            return tile_r((int)(p & 1)) - ia * (int64_t)args.bw_r - c0;
        };
        auto prefetch_row = [&](int64_t p) {
            if (TMA || p < 1 || p > K || ncol == 0) return;
            constexpr int64_t LINE = 128 / sizeof(TA);
            int64_t ia, ib;
            row_range(ring_xi[p % kRing], &ia, &ib);
            const int64_t l0 = c0 / LINE;
            const int nl = (int)((c1 + LINE - 1) / LINE - l0), h = (int)(ib - ia);
            for (int e = gt; e < h * nl; e += XT) {
                const int rr_ = e / nl, l = e - rr_ * nl;
                prefetch_line(A + (ia + rr_) * lda + (l0 + l) * LINE);
            }
        };
        auto quit_x = [&]() -> int {
            const int c = ld_vol(&ctl[0]);
            return (c == 5 || c == 6) ? c : 0;
        };

        int64_t done = K;
        // steps p whose partial carries the test of x^{p-1}: (check_offset + p - 1) % check_every == 0
        int64_t to_test = 0;
        if (check) {
            const int64_t r = (args.check_offset + 1) % args.check_every;  // residue at p = 2
            to_test = r == 0 ? 0 : args.check_every - r;                  // steps until the next test, from p = 2
        }
        if (K >= 1) {
            issue_row(1);
            issue_row(2);
            prefetch_row(1);
            prefetch_row(2);
        }
        for (int64_t p = 1; p <= K; ++p) {
            loader(p);
            if (!wait_row(p)) xf[2] = 1;
            if (gt == 0) {  // hand-over of step p written
                const uint32_t par = (uint32_t)(((p - 1) / ZR) & 1);
                const int code = lead_poll([&] { return mbar_test(&zfull[(p - 1) % ZR], par); }, quit_x,
                                           args.timeout_ns);
                if (code == 6) give_up(6);
                xf[0] = code;
            }
            xsync();
            if (xf[2] != 0 || xf[0] != 0) {
                if (xf[2] != 0 && gt == 0) give_up(6);
                done = p - 1;
                break;
            }

            // partial of r^p: A_{I_p, C_c} x^{p-1} (+ (z^p - b) on own rows of I_p)
            int64_t ia, ib;
            row_range(ring_xi[p % kRing], &ia, &ib);
            TS *accp = accr_base + (p % 3) * accset + (int64_t)rep * aw;
            if (ncol > 0) {
                auto e1 = [&](int l, TS v) { atomicAdd(accp + l, v); };
                auto e4 = [&](int l, TS v0, TS v1, TS v2, TS v3) { red_add4(accp + l, v0, v1, v2, v3); };
                if constexpr (TMA) {
                    tile_rowdot<XT, true, TA, TS>(gt, tile_r((int)(p & 1)), args.bw_r, (int)(ib - ia), args.bw_r / V,
                                                  xi, e1, e4);
                } else {  // x is zero beyond the owned columns
                    tile_rowdot<XT, false, TA, TS>(gt, A + ia * lda + c0, lda, (int)(ib - ia), (ncol + V - 1) / V, xi,
                                                   e1, e4);
                }
            }
            {
                const TS *zslot = zr + ((p - 1) % ZR) * tau_r;
                const int64_t la = lmax(ia, r0), lb = lmin(ib, r1);
                for (int64_t l = la + gt; l < lb; l += XT) atomicAdd(accp + (l - ia), zslot[l - ia]);
            }
            // stopping-test partial for x^{p-1}
            bool due = false;
            if (check && p >= 2) {
                due = to_test == 0;
                to_test = due ? args.check_every - 1 : to_test - 1;
            }
            if (due) {
                double e2 = 0.0;
                for (int j = gt; j < ncol; j += XT) {
                    const double xb = args.x_base ? args.x_base[c0 + j] : 0.0;
                    const double d = xb + (double)xi[j] - args.x_ref[c0 + j];
                    e2 = fma(d, d, e2);
                }
                e2 = warp_sum(e2);
                double *dred = reinterpret_cast<double *>(redx);
                if ((gt & 31) == 0) dred[gt >> 5] = e2;
                xsync();
                if (gt == 0) {
                    double s = 0.0;
                    for (int q = 0; q < kXWarps; ++q) s += dred[q];
                    atomicAdd(accp + tau_r, (TS)s);
                }
            }
            {  // clear this CTA's share of the set read two steps ahead
                TS *accz = accr_base + ((p + 1) % 3) * accset;
                for (int64_t e = clr0 + gt; e < clr1; e += XT) accz[e] = tzero<TS>();
            }
            xsync();
            if (gt == 0) {
                mbar_arrive(&zempty[(p - 1) % ZR]);
                red_release_gpu_add(args.bar_x, 1u);
                const int code = lead_poll(
                    [&] { return ld_acquire_gpu(args.bar_x) >= (unsigned)G * (unsigned)p; }, quit_x,
                    args.timeout_ns);
                if (code == 6) give_up(6);
                xf[0] = code;
            }
            xsync();
            if (xf[0] != 0) {
                done = p - 1;
                break;
            }

            // r^p = sum of the replicas; stopping test on x^{p-1}
            const int hr = (int)(ib - ia);
            const TS *accq = accr_base + (p % 3) * accset;
            for (int t = gt; t < hr; t += XT) {
                const TS sum = sum_replicas<RP>(accq + t, aw);
                rr[t] = sum;
                if (!finite_val(sum)) xf[3] = 1;
            }
            if (gt == XT - 1) {
                int code = 0;
                if (due) {
                    const TS e2 = sum_replicas<RP>(accq + tau_r, aw);
                    if ((double)e2 <= args.tol2_abs) code = 1;
                }
                xf[1] = code;
            }
            xsync();
            if (xf[1] == 1) {  // x^{p-1} passed: the x chain stops, the z chain completes step p + kZRing
                done = p - 1;
                if (gt == 0) {
                    st_vol(&ctl[1], (int)p);
                    __threadfence_block();
                    atomicCAS(&ctl[0], 0, 1);
                }
                break;
            }
            if (xf[3] != 0) {
                done = p - 1;
                if (gt == 0) give_up(5);
                break;
            }
            // x^p on own columns (+ dual v on own rows of I_p)
            const TS cI = ring_ci[p % kRing];
            {
                auto emitv = [&](int t, const TS(&sum)[V]) {
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const int c = t * V + e;
                        if (c < ncol) xi[c] -= cI * sum[e];
                    }
                };
                if constexpr (TMA) {
                    tile_colsum<XT, true, TA, TS>(gt, tile_r((int)(p & 1)), args.bw_r, hr, args.bw_r / V, rr, redx,
                                                  xsync, emitv);
                } else if (ncol > 0) {
                    tile_colsum<XT, false, TA, TS>(gt, A + ia * lda + c0, lda, hr, (ncol + V - 1) / V, rr, redx, xsync,
                                                   emitv);
                }
            }
            if (CORR) {
                const int64_t la = lmax(ia, r0), lb = lmin(ib, r1);
                for (int64_t l = la + gt; l < lb; l += XT) v_own[l - r0] -= cI * rr[l - ia];
            }
            xsync();
            // row tile of I_p is used up: its buffer takes I_{p+2}
            issue_row(p + 2);
            prefetch_row(p + 2);
        }
        if (TMA) {
            wait_row(0);
            wait_row(1);
        }
        for (int j = gt; j < ncol; j += XT) gx[c0 + j] = xi[j];
        if (CORR)
            for (int i = gt; i < nrow; i += XT) gv_dual[r0 + i] = v_own[i];
        if (cta == 0 && gt == 0) *args.iters_done = done;
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
    // when some block starts off a 16-byte boundary
    const int calign = a.col_off ? a.col_align : (a.tau_c & -a.tau_c);
    a.bw_c = ((a.tau_c + vx - 1) / vx) * vx + (calign % vx == 0 ? 0 : vx);
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
