// rebk_batch.cu -- REBK for batches of independent systems (many A_i, each with
// up to eight right-hand sides), one persistent launch per refinement pass.
//
// Method: Algorithm 1 of Du, Si, Sun (arXiv:2001.04179) in the correction form
// used by rebk_solve_refined (FP32 inner iterations on an FP32 copy of A_i,
// FP64 residuals f = b - z - A x, g = A^T z and FP64 updates z -= A s,
// x += A^T v), applied to every system of the batch.
//
// GB300 mapping.  The systems are small (A_i of at most a few tens of MB), so a
// system belongs to one CTA, or to one thread-block cluster: the iteration needs
// only __syncthreads (and cluster barriers), no device barrier.  A persistent
// grid takes systems from a queue, longest predicted time first; the systems
// predicted to take the longest run on a cluster of CTAs (2 by default), which
// splits their rows and columns and adds the block products up through
// distributed shared memory, so that they do not set the pass's makespan alone
// on one SM.  The right-hand sides of a system share its
// block sequence, so every element of a sampled block that a CTA reads feeds
// eight FMAs per product: the column step is W = A_J^T dZ + G_J (tau x 8) and
// dZ -= cJ A_J W; the row step is R = A_I dX - F_I + dZ_I and dX -= cI A_I^T R.
// Block indices are drawn on the device (Philox4x64-10, key (seed, system),
// the counter layout of the single-system path) by one warp, 16 iterations at
// a time.  All per-RHS state is stored with a stride of 8 values.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "rebk.h"
#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {
namespace {

constexpr int kBT = 512;        // threads per CTA
constexpr int kBW = kBT / 32;   // warps
constexpr int kR = 8;           // right-hand-side stride
constexpr int kDraws = 32;      // block draws prepared at a time (16 iterations)
constexpr int kColRowsInFlight = 4;  // column step: row loads in flight per lane (fast path)
constexpr int64_t kPrefetchPoolBytes = 96ll << 20;  // FP32 matrix pool above which blocks are prefetched
constexpr int kDefaultCluster = 2;       // CTAs per cluster for the longest systems, library choice
constexpr double kIterFloorElems = 900.0;
constexpr double kDefaultJointFrac = 0.25;  // cluster threshold: this fraction of the mean load per CTA
constexpr int kTopCluster = 4;            // library choice: CTAs per cluster for the few longest systems
constexpr double kTopFrac = 2.0;          // ... those predicted at >= this x the mean load per SM
constexpr int kTopMax = 8;                // ... at most this many (their launch holds 4 x this SMs)  // per-iteration latency floor of a CTA, in units of the
                                           // cost of one block element at tau 16 (queue ordering)


// L2 prefetch of a block of the system's FP32 copy: rows [r0, r0 + h) x columns
// [c0, c0 + w), one prefetch per 128-byte line, spread over the CTA.
__device__ __forceinline__ void prefetch_block(const float *A, int64_t lda, int64_t r0, int64_t h, int64_t c0,
                                               int64_t w) {
    if (h <= 0 || w <= 0) return;
    const int64_t l0 = c0 / 32, l1 = (c0 + w - 1) / 32;  // 32 floats per line
    const int64_t nl = l1 - l0 + 1;
    for (int64_t e = threadIdx.x; e < h * nl; e += blockDim.x) {
        const int64_t r = e / nl, l = e - r * nl;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(A + (r0 + r) * lda + (l0 + l) * 32));
    }
}

struct BatchSys {
    int64_t m, n, lda;
    int64_t a_off;   // element offset of A_i in the matrix pools
    int64_t mrow;    // first row of the system's m-sized arrays (rows of kR values)
    int64_t nrow;    // first row of the system's n-sized arrays
    int64_t tr, tc;  // offsets in the row / column table pools
    int s, t, fb_r, fb_c;
    double alpha;
};

struct InnerArgs {
    const BatchSys *sys;
    const int *order;          // systems in queue order
    int count;
    int *queue;                // next queue position (zeroed before launch)
    const float *A32;
    const double *cdf_r, *cdf_c;
    const float *coef_r, *coef_c;
    int tau;
    uint64_t seed;
    // per-system pass inputs/outputs
    const float *F32, *G32;    // f, g in FP32 (rows of kR)
    float *dZ, *dX, *S, *Vd;   // corrections and duals (rows of kR), zeroed per pass
    const double *Xb;          // x at the pass start (FP64 rows of kR)
    const double *Xref;        // NULL = no test
    const double *thr2;        // per system and RHS: squared error threshold
    int check_every;
    int prefetch;              // L2 prefetch of the next blocks (the FP32 pool exceeds L2)
    int64_t iters;             // per-system iteration budget of this pass
    int64_t *iters_done;       // per system, accumulated over passes
    const int64_t *iter_cap;   // per system: total iterations allowed
    const int *active;         // per system: 0 = converged, skip
    int col_path;              // blocks of 16 / 32 columns: 0 = a row's 16-byte vectors over tau/4 lanes,
                               // 1 = one lane per column (the wide blocks' layout)
    int32_t *idx_out;          // NULL, or per system idx_cap pairs (j_k, i_k) of iterations 1..idx_cap
    int64_t idx_cap;
    unsigned long long timeout_ns;
    int njoint;                // order[0 .. njoint) run on a whole cluster each (cluster launches only)
    int *queue_joint;          // next joint queue position (zeroed before launch)
};

// Sum over the 32 lanes of 8 per-lane values v[0..7], every shuffle a useful
// one (exchange halves, keep the other half): afterwards lane L holds the
// total of value ((L >> 4) & 1) * 4 + ((L >> 3) & 1) * 2 + ((L >> 2) & 1).
__device__ __forceinline__ float warp_sum8f(const float (&v)[8], int lane) {
    const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0, h2 = (lane & 4) != 0;
    float a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float keep = h4 ? v[i + 4] : v[i], send = h4 ? v[i] : v[i + 4];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = h3 ? a[i + 2] : a[i], send = h3 ? a[i] : a[i + 2];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c = (h2 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h2 ? b[0] : b[1], 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// Thread-block cluster helpers: rank and size of the cluster, a cluster-wide
// barrier (release / acquire at cluster scope, every thread of every CTA), and
// loads from another CTA's shared memory (distributed shared memory).
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the object at p in the CTA of the given rank
__device__ __forceinline__ uint32_t cluster_map(const void *p, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(a)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return a;
}
__device__ __forceinline__ float ld_cluster_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double ld_cluster_f64(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int ld_cluster_s32(uint32_t a) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void load8(const float *p, float (&v)[kR]) {
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// One CTA per system; CPL = columns per lane in the column step (tau <= 32 CPL).
//
// Cluster launches (cluster of CS CTAs): the systems order[0 .. njoint), the
// ones predicted to run longest, are each run by a whole cluster.  CTA rank q
// of the cluster owns rows [m q / CS, m (q+1) / CS) in the column step and
// columns [n q / CS, n (q+1) / CS) in the row step; the two block products of
// an iteration (W = A_J^T dZ and R = A_I dX) are per-CTA partial sums, which
// every CTA adds up in rank order from the others' shared memory after a
// cluster barrier (double-buffered by iteration parity, so one barrier per
// product), and each CTA then updates its own rows of dZ / columns of dX.
// Rank 0 alone writes the duals S, V and the recorded indices.  Once the joint
// queue is empty, the CTAs of a cluster take the other systems one each.

template <int CPL, bool CL>
__global__ void __launch_bounds__(kBT, 1) batch_inner_kernel(const InnerArgs a) {
    extern __shared__ __align__(16) float bsm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *Wpart = bsm;                                 // [kBW][32*CPL][kR]
    float *W = Wpart + kBW * 32 * CPL * kR;             // [32*CPL][kR]
    float *Rr = W + 32 * CPL * kR;                      // [tau][kR]
    int *draws = reinterpret_cast<int *>(Rr + 256 * kR);  // [kDraws]
    // cluster launches (CL): this CTA's partial products, two buffers each
    // ([2][tau][kR] for W, then for R), then the test sums ([2][kR] doubles)
    auto wc_buf = [&](int par) { return reinterpret_cast<float *>(draws + kDraws) + (size_t)par * a.tau * kR; };
    auto rc_buf = [&](int par) { return wc_buf(2) + (size_t)par * a.tau * kR; };
    auto ec_buf = [&](int par) { return reinterpret_cast<double *>(wc_buf(4)) + par * kR; };
    __shared__ int s_item, s_stop;
    __shared__ double s_err[kBW][kR];
    bool joint = CL && a.njoint > 0;

    for (;;) {
        int item;
        if (CL && joint) {  // rank 0 takes the next joint system for the whole cluster
            if (cluster_rank() == 0 && tid == 0) s_item = atomicAdd(a.queue_joint, 1);
            cluster_sync();
            item = ld_cluster_s32(cluster_map(&s_item, 0));
            cluster_sync();  // read by every CTA before rank 0 takes another
            if (item >= a.njoint) {
                joint = false;
                continue;
            }
        } else {
            if (tid == 0) s_item = a.njoint + atomicAdd(a.queue, 1);
            __syncthreads();
            item = s_item;
            __syncthreads();
            if (item >= a.count) break;
        }
        // ranks sharing this system: the cluster (joint systems) or this CTA alone
        const int NRK = (CL && joint) ? (int)cluster_size() : 1, rk = (CL && joint) ? (int)cluster_rank() : 0;
        const int id = a.order[item];
        if (!a.active[id]) continue;
        const BatchSys d = a.sys[id];
        const int64_t left = a.iter_cap[id] - a.iters_done[id];
        const int64_t K = a.iters < left ? a.iters : left;
        if (K <= 0) continue;
        const float *A = a.A32 + d.a_off;
        const int64_t m = d.m, n = d.n, lda = d.lda;
        float *dZ = a.dZ + d.mrow * kR, *Vd = a.Vd + d.mrow * kR;
        float *dX = a.dX + d.nrow * kR, *S = a.S + d.nrow * kR;
        const float *F = a.F32 + d.mrow * kR, *G = a.G32 + d.nrow * kR;
        // this rank's rows (column step) and columns (row step)
        const int rbeg = (int)(m * rk / NRK), rend = (int)(m * (rk + 1) / NRK);
        const int cbeg = (int)(n * rk / NRK), cend = (int)(n * (rk + 1) / NRK);
        const uint64_t k0 = (uint64_t)a.iters_done[id];
        int64_t k = 0;
        bool stopped = false;
        while (k < K && !stopped) {
            // ---- draws for the next (up to) 16 iterations ----
            if (warp == kBW - 1) {
                const uint64_t it = k0 + (uint64_t)k + (uint64_t)(lane >> 1);  // iteration index - 1
                const uint64_t dd = 2 * it + (uint64_t)(lane & 1);
                const double u = draw_uniform(a.seed, (uint64_t)id, dd);
                const int pick = (lane & 1) ? pick_block(a.cdf_r + d.tr, d.s, u, d.fb_r)
                                            : pick_block(a.cdf_c + d.tc, d.t, u, d.fb_c);
                draws[lane] = pick;
                // record the draws of iterations this pass runs (entry it of the system's row)
                if (a.idx_out && rk == 0 && (int64_t)it < a.idx_cap && k + (int64_t)(lane >> 1) < K)
                    a.idx_out[((int64_t)id * a.idx_cap + (int64_t)it) * 2 + (lane & 1)] = pick;
            }
            __syncthreads();
            const int64_t kend = (K - k < kDraws / 2) ? K : k + kDraws / 2;
            for (; k < kend; ++k) {
                const int slot = (int)((k % (kDraws / 2)) * 2);
                const int j = draws[slot], i = draws[slot + 1];
                const int par = (int)(k & 1);  // reduction buffers of this iteration (cluster launches)
                if (a.prefetch) {  // the row block of this iteration streams into L2 during the column step
                    const int64_t pi0 = (int64_t)i * a.tau;
                    prefetch_block(A, lda, pi0, pi0 + a.tau <= m ? a.tau : m - pi0, cbeg, cend - cbeg);
                }
                // ================= column step =================
                const int64_t j0 = (int64_t)j * a.tau;
                const int wc = (int)((j0 + a.tau <= n ? a.tau : n - j0));
                const float cJ = a.coef_c[d.tc + j];
                // full, 16-byte aligned blocks of 16 or 32 columns: tau/4 lanes per row, one
                // 16-byte load per lane, 32/(tau/4) rows per warp instruction (wider blocks
                // run faster on the lane-per-column path: tau 128 on 8192 x 2048, 607 against
                // 722 us per iteration)
                const bool fast = a.col_path == 0 && wc == a.tau && (j0 & 3) == 0 && wc >= 16 && wc <= 32 &&
                                  (wc & (wc - 1)) == 0;
                const int lpr = wc >> 2, rpw = fast ? 32 / lpr : 1, sub = lane % lpr, rrow = lane / lpr;
                if (fast) {
                    constexpr int UR = kColRowsInFlight;
                    float acc[4][kR];
#pragma unroll
                    for (int e = 0; e < 4; ++e)
#pragma unroll
                        for (int r = 0; r < kR; ++r) acc[e][r] = 0.f;
                    for (int64_t row0 = rbeg + (int64_t)warp * rpw * UR; row0 < rend;
                         row0 += (int64_t)kBW * rpw * UR) {
                        float4 av[UR];
                        float z[UR][kR];
#pragma unroll
                        for (int u = 0; u < UR; ++u) {
                            const int64_t row = row0 + (int64_t)u * rpw + rrow;
                            if (row < rend) {
                                av[u] = __ldg(reinterpret_cast<const float4 *>(A + row * lda + j0) + sub);
                                load8(dZ + row * kR, z[u]);
                            } else {
                                av[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                                for (int r = 0; r < kR; ++r) z[u][r] = 0.f;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < UR; ++u) {
                            const float ae[4] = {av[u].x, av[u].y, av[u].z, av[u].w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
#pragma unroll
                                for (int r = 0; r < kR; ++r) acc[e][r] = fmaf(ae[e], z[u][r], acc[e][r]);
                        }
                    }
                    // add the warp's row lanes (same sub), then one lane per column quad writes
                    for (int o = lpr; o < 32; o <<= 1)
#pragma unroll
                        for (int e = 0; e < 4; ++e)
#pragma unroll
                            for (int r = 0; r < kR; ++r) acc[e][r] += __shfl_xor_sync(0xffffffffu, acc[e][r], o);
                    if (rrow == 0) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float *dst = Wpart + ((size_t)warp * 32 * CPL + 4 * sub + e) * kR;
                            *reinterpret_cast<float4 *>(dst) = make_float4(acc[e][0], acc[e][1], acc[e][2], acc[e][3]);
                            *reinterpret_cast<float4 *>(dst + 4) =
                                make_float4(acc[e][4], acc[e][5], acc[e][6], acc[e][7]);
                        }
                    }
                } else {
                    constexpr int UR = CPL >= 8 ? 2 : 4;  // rows in flight per warp
                    float acc[CPL][kR];
#pragma unroll
                    for (int q = 0; q < CPL; ++q)
#pragma unroll
                        for (int r = 0; r < kR; ++r) acc[q][r] = 0.f;
                    for (int64_t row0 = rbeg + warp; row0 < rend; row0 += (int64_t)kBW * UR) {
                        float z[UR][kR], av[UR][CPL];
#pragma unroll
                        for (int u = 0; u < UR; ++u) {
                            const int64_t row = row0 + (int64_t)u * kBW;
                            if (row < rend) {
                                load8(dZ + row * kR, z[u]);
                                const float *Ar = A + row * lda + j0;
#pragma unroll
                                for (int q = 0; q < CPL; ++q) {
                                    const int c = lane + 32 * q;
                                    av[u][q] = c < wc ? __ldg(Ar + c) : 0.f;
                                }
                            } else {
#pragma unroll
                                for (int r = 0; r < kR; ++r) z[u][r] = 0.f;
#pragma unroll
                                for (int q = 0; q < CPL; ++q) av[u][q] = 0.f;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < UR; ++u)
#pragma unroll
                            for (int q = 0; q < CPL; ++q)
#pragma unroll
                                for (int r = 0; r < kR; ++r) acc[q][r] = fmaf(av[u][q], z[u][r], acc[q][r]);
                    }
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        float *dst = Wpart + ((size_t)warp * 32 * CPL + lane + 32 * q) * kR;
                        *reinterpret_cast<float4 *>(dst) = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
                        *reinterpret_cast<float4 *>(dst + 4) = make_float4(acc[q][4], acc[q][5], acc[q][6], acc[q][7]);
                    }
                }
                __syncthreads();
                if (!CL || NRK == 1) {
                    for (int e = tid; e < wc * kR; e += kBT) {
                        float sum = G[(j0 + e / kR) * kR + e % kR];
                        for (int w2 = 0; w2 < kBW; ++w2) sum += Wpart[(size_t)w2 * 32 * CPL * kR + e];
                        W[e] = sum;
                        S[(j0 + e / kR) * kR + e % kR] += cJ * sum;
                    }
                } else {  // this CTA's rows, then every rank's partial in rank order
                    float *wmine = wc_buf(par);
                    for (int e = tid; e < wc * kR; e += kBT) {
                        float sum = 0.f;
                        for (int w2 = 0; w2 < kBW; ++w2) sum += Wpart[(size_t)w2 * 32 * CPL * kR + e];
                        wmine[e] = sum;
                    }
                    cluster_sync();
                    for (int e = tid; e < wc * kR; e += kBT) {
                        float sum = G[(j0 + e / kR) * kR + e % kR];
                        for (int q = 0; q < NRK; ++q) sum += ld_cluster_f32(cluster_map(wmine + e, (uint32_t)q));
                        W[e] = sum;
                        if (rk == 0) S[(j0 + e / kR) * kR + e % kR] += cJ * sum;
                    }
                }
                __syncthreads();
                if (fast) {
                    // z update: the lane's 4 columns of W stay in registers; each row's dot is
                    // added over its tau/4 lanes
                    constexpr int UR = kColRowsInFlight;
                    float wv[4][kR];
#pragma unroll
                    for (int e = 0; e < 4; ++e) load8(W + (4 * sub + e) * kR, wv[e]);
                    for (int64_t row0 = rbeg + (int64_t)warp * rpw * UR; row0 < rend;
                         row0 += (int64_t)kBW * rpw * UR) {
                        float4 av[UR];
#pragma unroll
                        for (int u = 0; u < UR; ++u) {
                            const int64_t row = row0 + (int64_t)u * rpw + rrow;
                            av[u] = row < rend ? __ldg(reinterpret_cast<const float4 *>(A + row * lda + j0) + sub)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < UR; ++u) {
                            const float ae[4] = {av[u].x, av[u].y, av[u].z, av[u].w};
                            float t8[kR];
#pragma unroll
                            for (int r = 0; r < kR; ++r) {
                                float t = 0.f;
#pragma unroll
                                for (int e = 0; e < 4; ++e) t = fmaf(ae[e], wv[e][r], t);
                                t8[r] = t;
                            }
                            for (int o = 1; o < lpr; o <<= 1)
#pragma unroll
                                for (int r = 0; r < kR; ++r) t8[r] += __shfl_xor_sync(0xffffffffu, t8[r], o);
                            const int64_t row = row0 + (int64_t)u * rpw + rrow;
                            if (sub == 0 && row < rend) {
                                float *zr = dZ + row * kR;
#pragma unroll
                                for (int r = 0; r < kR; ++r) zr[r] -= cJ * t8[r];
                            }
                        }
                    }
                }
                // wide blocks (more than 32 columns): warps over rows, lanes over the columns
                // lane + 32 q (the column partial's layout, coalesced 128-byte loads), W of the
                // lane's columns in registers, the 8 sums of a row added over the warp by one
                // transposed butterfly; rows of UR in flight
                const bool wide = !fast && CPL >= 2 && wc > 32;
                if constexpr (CPL >= 2) {
                    if (wide) {
                        constexpr int UR = CPL >= 8 ? 2 : 4;
                        float wv[CPL][kR];
#pragma unroll
                        for (int q = 0; q < CPL; ++q) {
                            const int c = lane + 32 * q;
                            if (c < wc) {
                                load8(W + c * kR, wv[q]);
                            } else {
#pragma unroll
                                for (int r = 0; r < kR; ++r) wv[q][r] = 0.f;
                            }
                        }
                        const int ridx = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                        for (int64_t row0 = rbeg + (int64_t)warp * UR; row0 < rend; row0 += (int64_t)kBW * UR) {
                            float av[UR][CPL];
#pragma unroll
                            for (int u = 0; u < UR; ++u) {
                                const int64_t row = row0 + u;
                                const float *Ar = A + row * lda + j0;
#pragma unroll
                                for (int q = 0; q < CPL; ++q) {
                                    const int c = lane + 32 * q;
                                    av[u][q] = (row < rend && c < wc) ? __ldg(Ar + c) : 0.f;
                                }
                            }
#pragma unroll
                            for (int u = 0; u < UR; ++u) {
                                float t8[kR];
#pragma unroll
                                for (int r = 0; r < kR; ++r) {
                                    float t = 0.f;
#pragma unroll
                                    for (int q = 0; q < CPL; ++q) t = fmaf(av[u][q], wv[q][r], t);
                                    t8[r] = t;
                                }
                                const float v = warp_sum8f(t8, lane);
                                const int64_t row = row0 + u;
                                if ((lane & 3) == 0 && row < rend) dZ[row * kR + ridx] -= cJ * v;
                            }
                        }
                    }
                }
                const bool vec4 = ((j0 & 3) == 0) && ((wc & 3) == 0);
                for (int64_t row = (fast || wide) ? rend : rbeg + tid; row < rend; row += kBT) {
                    float t8[kR] = {0, 0, 0, 0, 0, 0, 0, 0};
                    const float *Ar = A + row * lda + j0;
                    if (vec4) {
                        for (int c0 = 0; c0 < wc; c0 += 16) {  // up to four 16-byte loads in flight
                            float4 a4[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                a4[u] = (c0 + 4 * u < wc) ? __ldg(reinterpret_cast<const float4 *>(Ar + c0 + 4 * u))
                                                          : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                if (c0 + 4 * u >= wc) break;
                                const float ae[4] = {a4[u].x, a4[u].y, a4[u].z, a4[u].w};
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    float wv[kR];
                                    load8(W + (c0 + 4 * u + e) * kR, wv);
#pragma unroll
                                    for (int r = 0; r < kR; ++r) t8[r] = fmaf(ae[e], wv[r], t8[r]);
                                }
                            }
                        }
                    } else {
                        for (int c = 0; c < wc; ++c) {
                            const float av = __ldg(Ar + c);
                            float wv[kR];
                            load8(W + c * kR, wv);
#pragma unroll
                            for (int r = 0; r < kR; ++r) t8[r] = fmaf(av, wv[r], t8[r]);
                        }
                    }
                    float *zr = dZ + row * kR;
#pragma unroll
                    for (int r = 0; r < kR; ++r) zr[r] -= cJ * t8[r];
                }
                __syncthreads();
                // ================= row step =================
                if (a.prefetch && k + 1 < kend) {  // the next column block streams into L2 during the row step
                    const int64_t pj0 = (int64_t)draws[slot + 2] * a.tau;
                    prefetch_block(A, lda, rbeg, rend - rbeg, pj0, pj0 + a.tau <= n ? a.tau : n - pj0);
                }
                const int64_t i0 = (int64_t)i * a.tau;
                const int hr = (int)((i0 + a.tau <= m ? a.tau : m - i0));
                const float cI = a.coef_r[d.tr + i];
                for (int l = warp; l < hr; l += kBW) {
                    float acc[kR] = {0, 0, 0, 0, 0, 0, 0, 0};
                    const float *Ar = A + (i0 + l) * lda;
                    constexpr int CU = 8;  // columns in flight per lane
                    for (int64_t col0 = cbeg + lane; col0 < cend; col0 += 32 * CU) {
                        float av[CU], xv[CU][kR];
#pragma unroll
                        for (int u = 0; u < CU; ++u) {
                            const int64_t col = col0 + 32 * u;
                            if (col < cend) {
                                av[u] = __ldg(Ar + col);
                                load8(dX + col * kR, xv[u]);
                            } else {
                                av[u] = 0.f;
#pragma unroll
                                for (int r = 0; r < kR; ++r) xv[u][r] = 0.f;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < CU; ++u)
#pragma unroll
                            for (int r = 0; r < kR; ++r) acc[r] = fmaf(av[u], xv[u][r], acc[r]);
                    }
#pragma unroll
                    for (int r = 0; r < kR; ++r) acc[r] = warp_sum(acc[r]);
                    if (lane < kR) {
                        float v = acc[0];
#pragma unroll
                        for (int r = 1; r < kR; ++r)
                            if (lane == r) v = acc[r];
                        if (!CL || NRK == 1) Rr[l * kR + lane] = v - F[(i0 + l) * kR + lane] + dZ[(i0 + l) * kR + lane];
                        else rc_buf(par)[l * kR + lane] = v;
                    }
                }
                if (!CL || NRK == 1) {
                    __syncthreads();
                } else {  // every rank's partial in rank order; dZ_I rows of other ranks through L2
                    cluster_sync();
                    const float *rmine = rc_buf(par);
                    for (int e = tid; e < hr * kR; e += kBT) {
                        float sum = 0.f;
                        for (int q = 0; q < NRK; ++q) sum += ld_cluster_f32(cluster_map(rmine + e, (uint32_t)q));
                        Rr[e] = sum - F[i0 * kR + e] + __ldcg(dZ + i0 * kR + e);
                    }
                    __syncthreads();
                }
                for (int64_t col = cbeg + tid; col < cend; col += kBT) {
                    float t8[kR] = {0, 0, 0, 0, 0, 0, 0, 0};
                    for (int l0 = 0; l0 < hr; l0 += 8) {  // eight rows in flight
                        float av[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            av[u] = (l0 + u < hr) ? __ldg(A + (i0 + l0 + u) * lda + col) : 0.f;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            if (l0 + u >= hr) break;
                            float rv[kR];
                            load8(Rr + (l0 + u) * kR, rv);
#pragma unroll
                            for (int r = 0; r < kR; ++r) t8[r] = fmaf(av[u], rv[r], t8[r]);
                        }
                    }
                    float *xr = dX + col * kR;
#pragma unroll
                    for (int r = 0; r < kR; ++r) xr[r] -= cI * t8[r];
                }
                if (rk == 0)
                    for (int e = tid; e < hr * kR; e += kBT) Vd[i0 * kR + e] -= cI * Rr[e];
                __syncthreads();
                // ================= stopping test =================
                if (a.Xref && a.check_every > 0 && ((int64_t)k0 + k + 1) % a.check_every == 0) {
                    double e2[kR] = {0, 0, 0, 0, 0, 0, 0, 0};
                    const double *xb = a.Xb + d.nrow * kR, *xr = a.Xref + d.nrow * kR;
                    for (int64_t col = cbeg + tid; col < cend; col += kBT) {
#pragma unroll
                        for (int r = 0; r < kR; ++r) {
                            const double df = xb[col * kR + r] + (double)dX[col * kR + r] - xr[col * kR + r];
                            e2[r] = fma(df, df, e2[r]);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < kR; ++r) e2[r] = warp_sum(e2[r]);
                    if (lane == 0)
#pragma unroll
                        for (int r = 0; r < kR; ++r) s_err[warp][r] = e2[r];
                    __syncthreads();
                    if (!CL || NRK == 1) {
                        if (tid == 0) {
                            int ok = 1;
                            for (int r = 0; r < kR; ++r) {
                                double t = 0.0;
                                for (int w2 = 0; w2 < kBW; ++w2) t += s_err[w2][r];
                                if (!(t <= a.thr2[(int64_t)id * kR + r])) ok = 0;
                            }
                            s_stop = ok;
                        }
                    } else {  // this CTA's columns, then every rank's sum in rank order
                        double *emine = ec_buf((int)(((int64_t)k0 + k + 1) / a.check_every & 1));
                        if (tid < kR) {
                            double t = 0.0;
                            for (int w2 = 0; w2 < kBW; ++w2) t += s_err[w2][tid];
                            emine[tid] = t;
                        }
                        cluster_sync();
                        if (tid == 0) {
                            int ok = 1;
                            for (int r = 0; r < kR; ++r) {
                                double t = 0.0;
                                for (int q = 0; q < NRK; ++q) t += ld_cluster_f64(cluster_map(emine + r, (uint32_t)q));
                                if (!(t <= a.thr2[(int64_t)id * kR + r])) ok = 0;
                            }
                            s_stop = ok;
                        }
                    }
                    __syncthreads();
                    if (s_stop) {
                        stopped = true;
                        ++k;
                        break;
                    }
                }
            }
        }
        if (tid == 0 && rk == 0) a.iters_done[id] += k;
        __syncthreads();
    }
    // no CTA leaves while another may still read its shared memory
    if (CL) cluster_sync();
}

// ---------------------------------------------------------------------------
// Batched FP64 sweep: for each system, ym = A P (m x 8) and yn = A^T Q
// (n x 8) over FP64 A; work items are (system, chunk of kSweepRows rows).
// ---------------------------------------------------------------------------
constexpr int kSR = 32;

struct SweepArgs {
    const BatchSys *sys;
    const int2 *items;   // (system, first row)
    int nitems;
    const double *A64;
    const double *P;     // n-rows (nrow offsets), may be NULL
    const float *Pf;     // alternatively FP32 P
    const double *Q;     // m-rows (mrow offsets), may be NULL
    const float *Qf;
    double *ym, *yn;     // outputs (zeroed before)
    const int *active;
};

__global__ void __launch_bounds__(256) batch_sweep_kernel(const SweepArgs a) {
    const int item = blockIdx.x;
    if (item >= a.nitems) return;
    const int2 it = a.items[item];
    const BatchSys d = a.sys[it.x];
    if (a.active && !a.active[it.x]) return;
    const int64_t r0 = it.y, r1 = (r0 + kSR < d.m) ? r0 + kSR : d.m;
    const double *A = a.A64 + d.a_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool hasP = a.P || a.Pf, hasQ = a.Q || a.Qf;
    // A P: warp per row, lanes over columns
    if (hasP) {
        for (int64_t row = r0 + warp; row < r1; row += 8) {
            double acc[kR] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int64_t col = lane; col < d.n; col += 32) {
                const double av = A[row * d.lda + col];
                const int64_t pr = (d.nrow + col) * kR;
#pragma unroll
                for (int r = 0; r < kR; ++r) acc[r] = fma(av, a.P ? a.P[pr + r] : (double)a.Pf[pr + r], acc[r]);
            }
#pragma unroll
            for (int r = 0; r < kR; ++r) acc[r] = warp_sum(acc[r]);
            if (lane < kR) {
                double v = acc[0];
#pragma unroll
                for (int r = 1; r < kR; ++r)
                    if (lane == r) v = acc[r];
                a.ym[(d.mrow + row) * kR + lane] = v;
            }
        }
    }
    // A^T Q: thread per column, sum over the chunk's rows, atomically added
    if (hasQ) {
        for (int64_t col = tid; col < d.n; col += 256) {
            double acc[kR] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int64_t row = r0; row < r1; ++row) {
                const double av = A[row * d.lda + col];
                const int64_t qr = (d.mrow + row) * kR;
#pragma unroll
                for (int r = 0; r < kR; ++r) acc[r] = fma(av, a.Q ? a.Q[qr + r] : (double)a.Qf[qr + r], acc[r]);
            }
#pragma unroll
            for (int r = 0; r < kR; ++r) atomicAdd(a.yn + (d.nrow + col) * kR + r, acc[r]);
        }
    }
}

// Elementwise pass kernels over all systems' rows (rows of kR values).
// f = b - z - ym ; F32 = f ; zero corrections.
__global__ void batch_prepare_kernel(int64_t mrows, int64_t nrows, const double *B, const double *Z,
                                     const double *YM, double *F, float *F32, const double *G, float *G32,
                                     float *dZ, float *Vd, float *dX, float *S) {
    const int64_t tot_m = mrows * kR, tot_n = nrows * kR;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot_m + tot_n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < tot_m) {
            const double f = (B[e] - Z[e]) - YM[e];
            F[e] = f;
            F32[e] = (float)f;
            dZ[e] = 0.f;
            Vd[e] = 0.f;
        } else {
            const int64_t q = e - tot_m;
            G32[q] = (float)G[q];
            dX[q] = 0.f;
            S[q] = 0.f;
        }
    }
}

// x += yn, z -= ym for active systems (all rows; inactive systems have zero duals).
__global__ void batch_update_kernel(int64_t mrows, int64_t nrows, double *X, const double *YN, double *Z,
                                    const double *YM) {
    const int64_t tot_m = mrows * kR, tot_n = nrows * kR;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot_m + tot_n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < tot_n) X[e] += YN[e];
        else Z[e - tot_n] -= YM[e - tot_n];
    }
}

// Per system and RHS: e2 = ||x - xref||^2, r2 = ||xref||^2 (one CTA per system).
__global__ void batch_error_kernel(const BatchSys *sys, const double *X, const double *Xref, double *e2,
                                   double *r2) {
    const BatchSys d = sys[blockIdx.x];
    __shared__ double se[kR][8], sr[kR][8];
    double a[kR] = {0, 0, 0, 0, 0, 0, 0, 0}, b[kR] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t col = threadIdx.x; col < d.n; col += blockDim.x) {
        const int64_t q = (d.nrow + col) * kR;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const double df = X[q + r] - Xref[q + r];
            a[r] = fma(df, df, a[r]);
            b[r] = fma(Xref[q + r], Xref[q + r], b[r]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        a[r] = warp_sum(a[r]);
        b[r] = warp_sum(b[r]);
    }
    if (lane == 0)
        for (int r = 0; r < kR; ++r) {
            se[r][warp] = a[r];
            sr[r][warp] = b[r];
        }
    __syncthreads();
    if (threadIdx.x < kR) {
        double x = 0, y = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            x += se[threadIdx.x][w];
            y += sr[threadIdx.x][w];
        }
        e2[(int64_t)blockIdx.x * kR + threadIdx.x] = x;
        r2[(int64_t)blockIdx.x * kR + threadIdx.x] = y;
    }
}

// Pass bookkeeping on the device (one thread per system): a system is active
// while some RHS error exceeds tol; its pass threshold is
// max(tol ||xref||, red * err)^2 per RHS.  Converged systems are counted.
__global__ void batch_pass_kernel(int count, int nrhs, const double *e2, const double *r2, double tol,
                                  double red, int *active, double *thr2, int *status, int *converged,
                                  const int64_t *iter_cap) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= count) return;
    if (iter_cap[id] == 0) {  // left out of this solve
        active[id] = 0;
        return;
    }
    int ok = 1;
    for (int r = 0; r < kR; ++r) {
        const double e = e2[(int64_t)id * kR + r], x2 = r2[(int64_t)id * kR + r];
        if (r < nrhs && !(e <= tol * tol * x2)) ok = 0;
        const double t1 = tol * tol * x2, t2 = red * red * e;
        thr2[(int64_t)id * kR + r] = r < nrhs ? (t1 > t2 ? t1 : t2) : 1e300;
    }
    active[id] = ok ? 0 : 1;
    status[id] = ok ? 0 : 4;
    if (ok) atomicAdd(converged, 1);
}

// Copy between the caller's (nrhs-strided) and the internal (kR-strided) layout.
__global__ void batch_pack_kernel(int64_t rows, int nrhs, const double *src, double *dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * kR;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / kR;
        const int r = (int)(e % kR);
        dst[e] = r < nrhs ? src[row * nrhs + r] : 0.0;
    }
}

__global__ void batch_unpack_kernel(int64_t rows, int nrhs, const double *src, double *dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * nrhs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / nrhs;
        const int r = (int)(e % nrhs);
        dst[e] = src[row * kR + r];
    }
}

int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 4096));
}

}  // namespace
}  // namespace rebk

using namespace rebk;

struct rebk_batch_s {
    cudaStream_t stream = nullptr;
    bool own_stream = false;  // created here: the legacy default stream cannot be captured
    int count = 0, nrhs = 1, tau = 0, max_outer = 6, check_every = 10;
    int col_path = 0;  // tile shape of the column step for blocks of 16 / 32 columns (autotuned with tau)
    int cluster = 1;   // CTAs per cluster for the longest systems (1 = every system on one CTA)
    bool top_tier = false;  // library choice: the few longest systems on clusters of kTopCluster,
                            // in a launch of their own beside the main one (second stream)
    int ntop = 0, grid_top = 0;
    cudaStream_t stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double joint_frac = 0.0;  // joint when predicted time >= joint_frac x the mean load per CTA
                              // (0: kDefaultJointFrac, and no clusters when every system qualifies)
    int njoint = 0;           // systems at the front of the queue order run jointly in this solve
    int grid = 0;             // CTAs of the main cluster launch in this solve
    std::vector<int64_t> hist_it;  // the previous solve's iterations per system (empty: none)
    double red = 1e-4;
    std::vector<int64_t> m, n, lda, a_off, mrow, nrow;
    int64_t Mrows = 0, Nrows = 0, Apool = 0;
    std::vector<double> alpha_given;  // <= 0: 1.75 / beta_max
    double *A64 = nullptr;
    float *A32 = nullptr;
    // tables for the current tau
    int tables_tau = 0;
    double *nr = nullptr, *nc = nullptr, *cdf_r = nullptr, *cdf_c = nullptr, *c64r = nullptr, *c64c = nullptr;
    float *c32r = nullptr, *c32c = nullptr;
    BatchSys *d_sys = nullptr;
    std::vector<BatchSys> sys;
    int *d_order = nullptr;
    // state (rows of kR)
    double *Z = nullptr, *F = nullptr, *YM = nullptr, *G = nullptr, *YN = nullptr, *Xi = nullptr, *Bi = nullptr,
           *Xr = nullptr;
    double *X0i = nullptr, *Z0i = nullptr;  // starting points (warm start), allocated on first use
    bool warm_x = false, warm_z = false;    // start from X0i / Z0i instead of x = 0 / z = b
    float *F32 = nullptr, *G32 = nullptr, *dZ = nullptr, *dX = nullptr, *S = nullptr, *Vd = nullptr;
    // per system
    int64_t *iters_done = nullptr, *iter_cap = nullptr;
    int *active = nullptr, *status = nullptr, *counters = nullptr;  // counters: [0] queue, [1] converged
    double *thr2 = nullptr, *e2 = nullptr, *r2 = nullptr;
    int2 *items = nullptr;
    int nitems = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> evs;
    // recording (rebk_batch_record): block indices and the final z of the next solves
    int32_t *rec_idx = nullptr;
    int64_t rec_cap = 0;
    double *rec_z = nullptr;
};

namespace {

rebk_status bfail(rebk_status s, const std::string &msg) {
    set_last_error(msg);
    return s;
}

#define BCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess) return bfail(e__ == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA, \
                                             std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

void free_batch(rebk_batch h) {
    if (!h) return;
    void *ptrs[] = {h->A64, h->A32, h->nr, h->nc, h->cdf_r, h->cdf_c, h->c64r, h->c64c, h->c32r, h->c32c,
                    h->d_sys, h->d_order, h->Z, h->F, h->YM, h->G, h->YN, h->Xi, h->Bi, h->Xr, h->F32,
                    h->G32, h->dZ, h->dX, h->S, h->Vd, h->iters_done, h->iter_cap, h->active, h->status,
                    h->counters, h->thr2, h->e2, h->r2, h->items, h->X0i, h->Z0i};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (cudaEvent_t e : h->evs) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->stream2) cudaStreamDestroy(h->stream2);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
}

// Block tables, step coefficients and descriptors for block size tau.
rebk_status build_tables(rebk_batch h, int tau, const std::vector<char> *only = nullptr) {
    if (h->tables_tau == tau && !only) return REBK_OK;
    const cudaStream_t st = h->stream;
    int64_t S = 0, T = 0, maxscr = 0;
    std::vector<int64_t> so(h->count), to(h->count);
    for (int i = 0; i < h->count; ++i) {
        so[i] = S;
        to[i] = T;
        S += (h->m[i] + tau - 1) / tau;
        T += (h->n[i] + tau - 1) / tau;
        maxscr = std::max(maxscr, h->m[i] + h->n[i] + 64 * h->n[i]);
    }
    double *ptr64[] = {h->nr, h->nc, h->cdf_r, h->cdf_c, h->c64r, h->c64c};
    for (double *p : ptr64)
        if (p) cudaFree(p);
    if (h->c32r) cudaFree(h->c32r);
    if (h->c32c) cudaFree(h->c32c);
    h->nr = h->nc = h->cdf_r = h->cdf_c = h->c64r = h->c64c = nullptr;
    h->c32r = h->c32c = nullptr;
    BCK(cudaMalloc(&h->nr, sizeof(double) * S));
    BCK(cudaMalloc(&h->cdf_r, sizeof(double) * S));
    BCK(cudaMalloc(&h->c64r, sizeof(double) * S));
    BCK(cudaMalloc(&h->c32r, sizeof(float) * S));
    BCK(cudaMalloc(&h->nc, sizeof(double) * T));
    BCK(cudaMalloc(&h->cdf_c, sizeof(double) * T));
    BCK(cudaMalloc(&h->c64c, sizeof(double) * T));
    BCK(cudaMalloc(&h->c32c, sizeof(float) * T));
    double *scratch = nullptr;
    int *fb = nullptr;
    BCK(cudaMalloc(&scratch, sizeof(double) * maxscr));
    BCK(cudaMalloc(&fb, sizeof(int) * 2 * h->count));
    // beta_max needs Gram scratch per system
    int64_t gmax = 0;
    for (int i = 0; i < h->count; ++i)
        gmax = std::max<int64_t>(gmax, std::max((h->m[i] + tau - 1) / tau, (h->n[i] + tau - 1) / tau) *
                                           (int64_t)tau * tau);
    double *gram = nullptr, *br = nullptr, *bc = nullptr;
    BCK(cudaMalloc(&gram, sizeof(double) * gmax));
    BCK(cudaMalloc(&br, sizeof(double) * S));
    BCK(cudaMalloc(&bc, sizeof(double) * T));
    h->sys.resize(h->count);
    std::vector<double> hb(std::max(S, T));
    std::vector<int> hfb(2 * h->count);
    std::vector<double> alpha(h->count);
    for (int i = 0; i < h->count; ++i) {
        const int s = (int)((h->m[i] + tau - 1) / tau), t = (int)((h->n[i] + tau - 1) / tau);
        if (only && !(*only)[i]) continue;
        BCK(block_tables(h->A64 + h->a_off[i], h->lda[i], h->m[i], h->n[i], tau, tau, s, t, h->nr + so[i],
                         h->nc + to[i], h->cdf_r + so[i], h->cdf_c + to[i], fb + 2 * i, scratch, st));
        if (!(h->alpha_given[i] > 0)) {
            BCK(beta_max_device(h->A64 + h->a_off[i], h->lda[i], h->m[i], h->n[i], tau, tau, s, t,
                                h->nr + so[i], h->nc + to[i], gram, br + so[i], bc + to[i], st));
        }
    }
    BCK(cudaMemcpyAsync(hfb.data(), fb, sizeof(int) * 2 * h->count, cudaMemcpyDeviceToHost, st));
    std::vector<double> hbr(S), hbc(T), hnr(S);
    BCK(cudaMemcpyAsync(hbr.data(), br, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
    BCK(cudaMemcpyAsync(hbc.data(), bc, sizeof(double) * T, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    for (int i = 0; i < h->count; ++i) {
        const int s = (int)((h->m[i] + tau - 1) / tau), t = (int)((h->n[i] + tau - 1) / tau);
        double a = h->alpha_given[i];
        if (only && !(*only)[i]) a = 1.0;  // tables not built: the system is skipped
        else if (!(a > 0)) {
            double bmax = 0.0;
            for (int q = 0; q < s; ++q) bmax = std::max(bmax, hbr[so[i] + q]);
            for (int q = 0; q < t; ++q) bmax = std::max(bmax, hbc[to[i] + q]);
            a = bmax > 0 ? 1.75 / bmax : 1.0;
        }
        alpha[i] = a;
        if (!only || (*only)[i]) {
            BCK(step_coefficients(h->nr + so[i], s, a, h->c64r + so[i], h->c32r + so[i], st));
            BCK(step_coefficients(h->nc + to[i], t, a, h->c64c + to[i], h->c32c + to[i], st));
        }
        BatchSys &d = h->sys[i];
        d.m = h->m[i];
        d.n = h->n[i];
        d.lda = h->lda[i];
        d.a_off = h->a_off[i];
        d.mrow = h->mrow[i];
        d.nrow = h->nrow[i];
        d.tr = so[i];
        d.tc = to[i];
        d.s = s;
        d.t = t;
        d.fb_r = hfb[2 * i];
        d.fb_c = hfb[2 * i + 1];
        d.alpha = a;
    }
    if (!h->d_sys) BCK(cudaMalloc(&h->d_sys, sizeof(BatchSys) * h->count));
    BCK(cudaMemcpyAsync(h->d_sys, h->sys.data(), sizeof(BatchSys) * h->count, cudaMemcpyHostToDevice, st));
    BCK(cudaStreamSynchronize(st));
    cudaFree(scratch);
    cudaFree(fb);
    cudaFree(gram);
    cudaFree(br);
    cudaFree(bc);
    h->tables_tau = only ? -1 : tau;  // a partial build must be redone for a full solve
    return REBK_OK;
}

int cpl_for(int tau) { return tau <= 32 ? 1 : tau <= 64 ? 2 : tau <= 128 ? 4 : 8; }

// Dynamic shared memory of the inner kernel.  Kept to what the phases need: the rest
// of the SM's 256 KB serves as L1, which holds the dZ / dX rows that the lanes of a
// row and the warps of a row block re-read (reserving it for a system's dZ / dX
// instead made the systems that do not fit slower).
size_t inner_smem(int cpl, int tau, int cluster) {
    size_t b = sizeof(float) * ((size_t)kBW * 32 * cpl * kR + 32 * cpl * kR + 256 * kR) + sizeof(int) * kDraws;
    if (cluster > 1)  // the partial products and test sums read by the other CTAs of the cluster
        b += sizeof(float) * 4 * (size_t)tau * kR + sizeof(double) * 2 * kR;
    return b;
}

void *inner_kernel(int cpl, bool cl) {
    if (cl)
        return cpl == 1 ? (void *)&batch_inner_kernel<1, true>
               : cpl == 2 ? (void *)&batch_inner_kernel<2, true>
               : cpl == 4 ? (void *)&batch_inner_kernel<4, true> : (void *)&batch_inner_kernel<8, true>;
    return cpl == 1 ? (void *)&batch_inner_kernel<1, false>
           : cpl == 2 ? (void *)&batch_inner_kernel<2, false>
           : cpl == 4 ? (void *)&batch_inner_kernel<4, false> : (void *)&batch_inner_kernel<8, false>;
}

// CTAs of a persistent launch: one per SM, or for clusters of cs CTAs as many
// whole clusters as can be resident at once (cs CTAs each).
int inner_grid(int tau, int cs, int sms, int avail) {
    if (cs <= 1) return avail;
    const int cpl = cpl_for(tau);
    const size_t smem = inner_smem(cpl, tau, cs);
    void *k = inner_kernel(cpl, true);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(sms / cs * cs);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = cs;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return std::min(nc * cs, avail / cs * cs);
}

cudaError_t launch_inner(const InnerArgs &a, int grid, int cs, cudaStream_t st) {
    const int cpl = cpl_for(a.tau);
    const size_t smem = inner_smem(cpl, a.tau, cs);
    void *k = inner_kernel(cpl, cs > 1);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    InnerArgs c = a;
    void *params[] = {&c};
    if (cs <= 1) return cudaLaunchKernel(k, dim3(grid), dim3(kBT), params, smem, st);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = cs;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, k, params);
}

// Queues the kernels of one batched solve (graph-capturable: no host syncs).
rebk_status enqueue_solve(rebk_batch h, int tau, double tol, int64_t inner_iters, uint64_t seed,
                          bool use_ref, int passes, int *launches) {
    const cudaStream_t st = h->stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t totm = h->Mrows, totn = h->Nrows;
    auto sweep = [&](const double *P, const float *Pf, const double *Q, const float *Qf, double *ym,
                     double *yn) -> cudaError_t {
        if (ym) cudaMemsetAsync(ym, 0, sizeof(double) * totm * kR, st);
        if (yn) cudaMemsetAsync(yn, 0, sizeof(double) * totn * kR, st);
        SweepArgs s;
        s.sys = h->d_sys;
        s.items = h->items;
        s.nitems = h->nitems;
        s.A64 = h->A64;
        s.P = P;
        s.Pf = Pf;
        s.Q = Q;
        s.Qf = Qf;
        s.ym = ym;
        s.yn = yn;
        s.active = use_ref ? h->active : nullptr;
        batch_sweep_kernel<<<h->nitems, 256, 0, st>>>(s);
        ++*launches;
        return cudaGetLastError();
    };
    for (int pass = 0; pass < passes; ++pass) {
        // f = b - z - A x, g = A^T z
        BCK(sweep(h->Xi, nullptr, h->Z, nullptr, h->YM, h->G));
        batch_prepare_kernel<<<blocks_for((totm + totn) * kR, 256), 256, 0, st>>>(
            totm, totn, h->Bi, h->Z, h->YM, h->F, h->F32, h->G, h->G32, h->dZ, h->Vd, h->dX, h->S);
        ++*launches;
        if (use_ref) {
            BCK(cudaMemsetAsync(h->counters + 1, 0, sizeof(int), st));
            batch_error_kernel<<<h->count, 256, 0, st>>>(h->d_sys, h->Xi, h->Xr, h->e2, h->r2);
            batch_pass_kernel<<<(h->count + 127) / 128, 128, 0, st>>>(h->count, h->nrhs, h->e2, h->r2, tol,
                                                                   h->red, h->active, h->thr2, h->status,
                                                                   h->counters + 1, h->iter_cap);
            *launches += 2;
        }
        BCK(cudaMemsetAsync(h->counters, 0, sizeof(int), st));
        BCK(cudaMemsetAsync(h->counters + 2, 0, sizeof(int), st));
        InnerArgs a;
        memset(&a, 0, sizeof(a));
        a.sys = h->d_sys;
        a.order = h->d_order;
        a.count = h->count;
        a.queue = h->counters;
        a.A32 = h->A32;
        // prefetching pays only when the blocks come from HBM: a pool that fits in L2
        // (one shared matrix, small systems) is read from L2 anyway
        a.prefetch = (int64_t)sizeof(float) * h->Apool > kPrefetchPoolBytes;
        a.cdf_r = h->cdf_r;
        a.cdf_c = h->cdf_c;
        a.coef_r = h->c32r;
        a.coef_c = h->c32c;
        a.tau = tau;
        a.seed = seed;
        a.F32 = h->F32;
        a.G32 = h->G32;
        a.dZ = h->dZ;
        a.dX = h->dX;
        a.S = h->S;
        a.Vd = h->Vd;
        a.Xb = h->Xi;
        a.Xref = use_ref ? h->Xr : nullptr;
        a.thr2 = h->thr2;
        a.check_every = h->check_every;
        a.iters = inner_iters;
        a.iters_done = h->iters_done;
        a.iter_cap = h->iter_cap;
        a.active = h->active;
        a.col_path = h->col_path;
        a.idx_out = h->rec_idx;
        a.idx_cap = h->rec_cap;
        a.timeout_ns = kBarrierTimeoutNs;
        a.queue_joint = h->counters + 2;
        const bool clus = h->cluster > 1 && h->grid >= h->cluster && h->njoint > 0;
        a.njoint = clus ? h->njoint : 0;
        if (h->ntop > 0) {
            // the longest systems, order[0 .. ntop), each on a cluster of kTopCluster CTAs in a
            // launch of their own on the second stream; the main launch takes the rest
            BCK(cudaMemsetAsync(h->counters + 3, 0, sizeof(int) * 2, st));
            BCK(cudaEventRecord(h->ev_fork, st));
            BCK(cudaStreamWaitEvent(h->stream2, h->ev_fork, 0));
            InnerArgs t = a;
            t.count = h->ntop;
            t.njoint = h->ntop;
            t.queue = h->counters + 4;
            t.queue_joint = h->counters + 3;
            BCK(launch_inner(t, h->grid_top, kTopCluster, h->stream2));
            BCK(cudaEventRecord(h->ev_join, h->stream2));
            ++*launches;
            a.order = h->d_order + h->ntop;
            a.count = h->count - h->ntop;
        }
        BCK(launch_inner(a, clus ? h->grid : sms - h->grid_top, clus ? h->cluster : 1, st));
        ++*launches;
        if (h->ntop > 0) BCK(cudaStreamWaitEvent(st, h->ev_join, 0));
        // z <- z - A s, x <- x + A^T v; the FP32 duals are widened once into G and F
        // (free until the next pass) so the FP64 sweep converts nothing in its loops
        BCK(widen_f32(h->S, h->G, totn * kR, st));
        BCK(widen_f32(h->Vd, h->F, totm * kR, st));
        *launches += 2;
        BCK(sweep(h->G, nullptr, h->F, nullptr, h->YM, h->YN));
        batch_update_kernel<<<blocks_for((totm + totn) * kR, 256), 256, 0, st>>>(totm, totn, h->Xi, h->YN, h->Z,
                                                                                h->YM);
        ++*launches;
    }
    if (use_ref) {
        BCK(cudaMemsetAsync(h->counters + 1, 0, sizeof(int), st));
        batch_error_kernel<<<h->count, 256, 0, st>>>(h->d_sys, h->Xi, h->Xr, h->e2, h->r2);
        batch_pass_kernel<<<(h->count + 127) / 128, 128, 0, st>>>(h->count, h->nrhs, h->e2, h->r2, tol, h->red,
                                                               h->active, h->thr2, h->status, h->counters + 1, h->iter_cap);
        *launches += 2;
    }
    return REBK_OK;
}

}  // namespace

extern "C" {

rebk_status rebk_batch_create(rebk_batch *out, int32_t count, const int64_t *m, const int64_t *n,
                              const double *const *A, int A_on_device, const double *alpha,
                              const rebk_batch_options *opt) {
    set_last_error("");
    if (!out) return bfail(REBK_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !m || !n || !A) return bfail(REBK_EINVAL, "count >= 1 and m, n, A arrays required");
    rebk_batch_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.tau < 0 || o.tau > 256) return bfail(REBK_EINVAL, "tau must be 0 (auto) or 1..256");
    if (o.nrhs < 0 || o.nrhs > 8) return bfail(REBK_EINVAL, "nrhs must be 1..8");
    if (o.max_outer < 0 || o.check_every < 0 || o.inner_reduction < 0) return bfail(REBK_EINVAL, "negative option");
    if (o.col_path != 0 && o.col_path != 1) return bfail(REBK_EINVAL, "col_path must be 0 or 1");
    if (o.cluster != 0 && o.cluster != 1 && o.cluster != 2 && o.cluster != 4 && o.cluster != 8)
        return bfail(REBK_EINVAL, "cluster must be 0 (library choice), 1, 2, 4 or 8");
    if (!(o.joint_frac >= 0.0) || !std::isfinite(o.joint_frac)) return bfail(REBK_EINVAL, "joint_frac must be >= 0");
    for (int i = 0; i < count; ++i) {
        if (m[i] < 1 || n[i] < 1) return bfail(REBK_EINVAL, "every system needs m, n >= 1");
        if (!A[i]) return bfail(REBK_EINVAL, "NULL matrix pointer");
        if (m[i] > (1 << 24) || n[i] > (1 << 24)) return bfail(REBK_EUNSUPPORTED, "system too large for a batch");
    }
    rebk_batch h = new rebk_batch_s();
    h->stream = static_cast<cudaStream_t>(o.stream);
    h->count = count;
    h->nrhs = o.nrhs > 0 ? o.nrhs : 1;
    h->tau = o.tau;
    h->max_outer = o.max_outer > 0 ? o.max_outer : 6;
    h->check_every = o.check_every > 0 ? o.check_every : 10;
    h->red = o.inner_reduction > 0 ? o.inner_reduction : 1e-4;
    h->col_path = o.col_path;
    h->cluster = o.cluster > 0 ? o.cluster : kDefaultCluster;
    h->top_tier = o.cluster == 0;
    h->joint_frac = o.joint_frac;
    h->m.assign(m, m + count);
    h->n.assign(n, n + count);
    h->alpha_given.assign(count, 0.0);
    if (alpha)
        for (int i = 0; i < count; ++i) h->alpha_given[i] = alpha[i];
    int64_t mo = 0, no = 0, ao = 0;
    std::vector<int> first(count);  // first system holding the same matrix (equal pointer and shape)
    for (int i = 0; i < count; ++i) {
        const int64_t ld = (n[i] + 63) / 64 * 64;
        first[i] = i;
        for (int k = 0; k < i; ++k)
            if (first[k] == k && A[k] == A[i] && m[k] == m[i] && n[k] == n[i]) {
                first[i] = k;
                break;
            }
        h->lda.push_back(ld);
        h->a_off.push_back(first[i] == i ? ao : h->a_off[first[i]]);
        h->mrow.push_back(mo);
        h->nrow.push_back(no);
        if (first[i] == i) ao += m[i] * ld;
        mo += m[i];
        no += n[i];
    }
    h->Apool = ao;
    h->Mrows = mo;
    h->Nrows = no;
    auto fin = [&](rebk_status s) {
        if (s != REBK_OK) free_batch(h);
        return s;
    };
#define BCKH(call)                                                                                 \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess)                                                                    \
            return fin(bfail(e__ == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA,          \
                             std::string(#call) + ": " + cudaGetErrorString(e__)));                \
    } while (0)
    BCKH(cudaEventCreate(&h->ev0));
    BCKH(cudaEventCreate(&h->ev1));
    if (!h->stream) {
        BCKH(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    const cudaStream_t st = h->stream;
    BCKH(cudaMalloc(&h->A64, sizeof(double) * ao));
    BCKH(cudaMalloc(&h->A32, sizeof(float) * ao));
    for (int i = 0; i < count; ++i) {
        if (first[i] != i) continue;  // stored once
        BCKH(cudaMemcpy2DAsync(h->A64 + h->a_off[i], h->lda[i] * sizeof(double), A[i], n[i] * sizeof(double),
                               n[i] * sizeof(double), m[i],
                               A_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        if (h->lda[i] > n[i])
            BCKH(cudaMemset2DAsync(h->A64 + h->a_off[i] + n[i], h->lda[i] * sizeof(double), 0,
                                   (h->lda[i] - n[i]) * sizeof(double), m[i], st));
    }
    BCKH(convert_storage(h->A64, ao, h->A32, ao, 1, ao, 1, st));  // the pool as one row of ao elements
    const size_t MR = (size_t)mo * kR, NR = (size_t)no * kR;
    double **d64[] = {&h->Z, &h->F, &h->YM, &h->Bi};
    for (double **p : d64) BCKH(cudaMalloc(p, sizeof(double) * MR));
    double **dn64[] = {&h->G, &h->YN, &h->Xi, &h->Xr};
    for (double **p : dn64) BCKH(cudaMalloc(p, sizeof(double) * NR));
    float **f32m[] = {&h->F32, &h->dZ, &h->Vd};
    for (float **p : f32m) BCKH(cudaMalloc(p, sizeof(float) * MR));
    float **f32n[] = {&h->G32, &h->dX, &h->S};
    for (float **p : f32n) BCKH(cudaMalloc(p, sizeof(float) * NR));
    BCKH(cudaMalloc(&h->iters_done, sizeof(int64_t) * count));
    BCKH(cudaMalloc(&h->iter_cap, sizeof(int64_t) * count));
    BCKH(cudaMalloc(&h->active, sizeof(int) * count));
    BCKH(cudaMalloc(&h->status, sizeof(int) * count));
    BCKH(cudaMalloc(&h->counters, sizeof(int) * 8));
    BCKH(cudaMalloc(&h->thr2, sizeof(double) * count * kR));
    BCKH(cudaMalloc(&h->e2, sizeof(double) * count * kR));
    BCKH(cudaMalloc(&h->r2, sizeof(double) * count * kR));
    // sweep work items and the first solve's queue order (largest m * n first; later
    // solves order by the previous solve's measured iterations, see run_batch)
    std::vector<int2> items;
    for (int i = 0; i < count; ++i)
        for (int64_t r = 0; r < m[i]; r += kSR) items.push_back(make_int2(i, (int)r));
    h->nitems = (int)items.size();
    BCKH(cudaMalloc(&h->items, sizeof(int2) * items.size()));
    BCKH(cudaMemcpy(h->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return m[a] * n[a] > m[b] * n[b]; });
    BCKH(cudaMalloc(&h->d_order, sizeof(int) * count));
    BCKH(cudaMemcpy(h->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
#undef BCKH
    if (h->tau > 0) {
        rebk_status s = build_tables(h, h->tau);
        if (s != REBK_OK) return fin(s);
    }
    *out = h;
    return REBK_OK;
}

void rebk_batch_destroy(rebk_batch h) { free_batch(h); }

rebk_status rebk_batch_record(rebk_batch h, int32_t *idx_out, int64_t idx_cap, double *Z_out) {
    if (!h) return bfail(REBK_EINVAL, "NULL handle");
    if (idx_cap < 0 || (idx_out && idx_cap == 0)) return bfail(REBK_EINVAL, "idx_cap must be >= 1 with idx_out");
    h->rec_idx = idx_out;
    h->rec_cap = idx_out ? idx_cap : 0;
    h->rec_z = Z_out;
    return REBK_OK;
}

rebk_status rebk_batch_info(rebk_batch h, int32_t *tau, int32_t *count) {
    if (!h) return bfail(REBK_EINVAL, "NULL handle");
    if (tau) *tau = h->tables_tau > 0 ? h->tables_tau : h->tau;
    if (count) *count = h->count;
    return REBK_OK;
}

}  // extern "C"

namespace {

// One solve of the loaded batch at block size tau (tables built).  Returns the
// stats; state buffers are reset from B.
rebk_status run_batch(rebk_batch h, int tau, double tol, int64_t max_iter, int64_t inner_iters,
                      uint64_t seed, bool use_ref, bool graph, rebk_batch_stats *stats,
                      const std::vector<char> *only = nullptr) {
    const cudaStream_t st = h->stream;
    const size_t MR = (size_t)h->Mrows * kR, NR = (size_t)h->Nrows * kR;
    {
        rebk_status ts = build_tables(h, tau, only);
        if (ts != REBK_OK) return ts;
    }
    // x0 = 0, z0 = b (or the caller's starting points); counters
    if (h->warm_x) BCK(cudaMemcpyAsync(h->Xi, h->X0i, sizeof(double) * NR, cudaMemcpyDeviceToDevice, st));
    else BCK(cudaMemsetAsync(h->Xi, 0, sizeof(double) * NR, st));
    BCK(cudaMemcpyAsync(h->Z, h->warm_z ? h->Z0i : h->Bi, sizeof(double) * MR, cudaMemcpyDeviceToDevice, st));
    BCK(cudaMemsetAsync(h->iters_done, 0, sizeof(int64_t) * h->count, st));
    std::vector<int64_t> cap(h->count, max_iter);
    std::vector<int> ones(h->count, 1), fours(h->count, REBK_MAX_ITER);
    if (only)
        for (int i = 0; i < h->count; ++i)
            if (!(*only)[i]) {
                cap[i] = 0;
                ones[i] = 0;
            }
    BCK(cudaMemcpyAsync(h->iter_cap, cap.data(), sizeof(int64_t) * h->count, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(h->active, ones.data(), sizeof(int) * h->count, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(h->status, fours.data(), sizeof(int) * h->count, cudaMemcpyHostToDevice, st));
    std::vector<double> big(h->count * kR, 1e300);
    BCK(cudaMemcpyAsync(h->thr2, big.data(), sizeof(double) * big.size(), cudaMemcpyHostToDevice, st));
    BCK(cudaMemsetAsync(h->counters, 0, sizeof(int) * 8, st));
    {
        // Queue plan: predicted time of each system on one CTA -- the previous solve's
        // iteration count (1 without one) times a per-iteration cost model fitted on
        // GB300 (a latency floor plus a term in the block elements: about 5.7 us +
        // 6.4 ns x tau / 16 x (m + n)) -- longest first.  With clusters, the systems
        // predicted at >= joint_frac (0.25 by default) x the mean load per CTA come
        // first and run on a whole cluster each.  The order changes no result: each
        // system's random stream is keyed by its index.
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        h->ntop = 0;
        h->grid_top = 0;
        const bool hist = (int)h->hist_it.size() == h->count;
        std::vector<double> cost(h->count, 0.0);
        double total = 0.0;
        for (int i = 0; i < h->count; ++i) {
            if (only && !(*only)[i]) continue;
            const double its = hist ? (double)std::max<int64_t>(h->hist_it[i], 1) : 1.0;
            cost[i] = its * (kIterFloorElems + (double)tau / 16.0 * (double)(h->m[i] + h->n[i]));
            total += cost[i];
        }
        std::vector<int> order(h->count);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        h->njoint = 0;
        int busy = 0;  // systems with work in this solve
        for (int i = 0; i < h->count; ++i) busy += cost[i] > 0.0;
        // library choice: the few systems predicted at >= kTopFrac x the mean load per SM
        // on clusters of kTopCluster, in a launch of their own beside the main one
        if (h->top_tier && h->cluster > 1) {
            int n1 = 0;
            while (n1 < kTopMax && n1 < busy && cost[order[n1]] >= kTopFrac * total / sms) ++n1;
            if (n1 > 0 && n1 < busy) {
                const int g1 = inner_grid(tau, kTopCluster, sms, n1 * kTopCluster);
                if (g1 >= kTopCluster) {
                    h->ntop = g1 / kTopCluster < n1 ? g1 / kTopCluster : n1;
                    h->grid_top = h->ntop * kTopCluster;
                    if (!h->stream2) BCK(cudaStreamCreateWithFlags(&h->stream2, cudaStreamNonBlocking));
                    if (!h->ev_fork) BCK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
                    if (!h->ev_join) BCK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
                }
            }
        }
        if (h->cluster > 1) {
            h->grid = inner_grid(tau, h->cluster, sms, sms - h->grid_top);
        }
        if (h->cluster > 1 && h->grid >= h->cluster) {
            const double frac = h->joint_frac > 0.0 ? h->joint_frac : kDefaultJointFrac;
            const double load = total / h->grid;
            while (h->ntop + h->njoint < h->count && cost[order[h->ntop + h->njoint]] > 0.0 &&
                   cost[order[h->ntop + h->njoint]] >= frac * load)
                ++h->njoint;
            // library choice: when every system qualifies none stands out, and a plain
            // launch (one CTA each) is faster (152 equal systems: 315 against 322 ms)
            if (h->joint_frac <= 0.0 && h->ntop == 0 && h->njoint == busy) h->njoint = 0;
        }
        BCK(cudaMemcpyAsync(h->d_order, order.data(), sizeof(int) * h->count, cudaMemcpyHostToDevice, st));
    }
    BCK(cudaStreamSynchronize(st));
    const int passes = h->max_outer;
    int launches = 0;
    BCK(cudaEventRecord(h->ev0, st));
    bool used_graph = false;
    if (graph) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        rebk_status rs = REBK_OK;
        if (e == cudaSuccess) {
            rs = enqueue_solve(h, tau, tol, inner_iters, seed, use_ref, passes, &launches);
            e = cudaStreamEndCapture(st, &g);
        }
        if (e == cudaSuccess && rs == REBK_OK) e = cudaGraphInstantiate(&ge, g, 0);
        if (e == cudaSuccess && rs == REBK_OK) {
            BCK(cudaEventRecord(h->ev0, st));
            e = cudaGraphLaunch(ge, st);
            used_graph = e == cudaSuccess;
        }
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (rs != REBK_OK) return rs;
        if (!used_graph) {
            cudaGetLastError();
            launches = 0;
        }
    }
    if (!used_graph) {
        rebk_status rs = enqueue_solve(h, tau, tol, inner_iters, seed, use_ref, passes, &launches);
        if (rs != REBK_OK) return rs;
    }
    BCK(cudaEventRecord(h->ev1, st));
    BCK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    std::vector<int64_t> it(h->count);
    int conv = 0;
    BCK(cudaMemcpy(it.data(), h->iters_done, sizeof(int64_t) * h->count, cudaMemcpyDeviceToHost));
    BCK(cudaMemcpy(&conv, h->counters + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (!only) h->hist_it = it;  // the next solve's queue plan
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->converged = use_ref ? conv : 0;
        stats->outer = passes;
        for (int64_t v : it) {
            stats->iterations += v;
            stats->max_iterations = std::max(stats->max_iterations, v);
        }
        stats->device_ms = ms;
        stats->launches = launches;
        stats->tau = tau;
        stats->graph = used_graph ? 1 : 0;
        stats->col_path = h->col_path;
        stats->cluster = h->cluster > 1 && h->grid >= h->cluster && h->njoint > 0 ? h->cluster : 1;
        stats->joint = h->njoint;
        stats->top_cluster = h->ntop > 0 ? kTopCluster : 0;
        stats->top_joint = h->ntop;
    }
    return REBK_OK;
}

}  // namespace

extern "C" rebk_status rebk_batch_solve_ex(rebk_batch h, const double *B, double *X, const double *X_ref,
                                           const double *X0, const double *Z0, double tol, int64_t max_iter,
                                           int64_t inner_iters, uint64_t seed, int32_t *status_out,
                                           rebk_batch_stats *stats) {
    set_last_error("");
    if (!h) return bfail(REBK_EINVAL, "NULL handle");
    if (!B || !X) return bfail(REBK_EINVAL, "B and X must be device pointers");
    if (max_iter < 0 || inner_iters < 0 || !std::isfinite(tol)) return bfail(REBK_EINVAL, "bad tol/max_iter");
    const cudaStream_t st = h->stream;
    if (h->own_stream) {  // order after the caller's work on the legacy default stream
        BCK(cudaEventRecord(h->ev0, 0));
        BCK(cudaStreamWaitEvent(st, h->ev0, 0));
    }
    h->warm_x = X0 != nullptr;
    h->warm_z = Z0 != nullptr;
    if (X0) {
        if (!h->X0i) BCK(cudaMalloc(&h->X0i, sizeof(double) * (size_t)h->Nrows * kR));
        batch_pack_kernel<<<blocks_for(h->Nrows * kR, 256), 256, 0, st>>>(h->Nrows, h->nrhs, X0, h->X0i);
    }
    if (Z0) {
        if (!h->Z0i) BCK(cudaMalloc(&h->Z0i, sizeof(double) * (size_t)h->Mrows * kR));
        batch_pack_kernel<<<blocks_for(h->Mrows * kR, 256), 256, 0, st>>>(h->Mrows, h->nrhs, Z0, h->Z0i);
    }
    const bool use_ref = X_ref != nullptr;
    if (inner_iters <= 0) inner_iters = use_ref ? max_iter : 2000;
    if (max_iter == 0) max_iter = (int64_t)1 << 40;
    // caller layout -> internal rows of kR values
    batch_pack_kernel<<<blocks_for(h->Mrows * kR, 256), 256, 0, st>>>(h->Mrows, h->nrhs, B, h->Bi);
    if (use_ref) batch_pack_kernel<<<blocks_for(h->Nrows * kR, 256), 256, 0, st>>>(h->Nrows, h->nrhs, X_ref, h->Xr);
    BCK(cudaGetLastError());
    int tau = h->tables_tau > 0 ? h->tables_tau : h->tau;
    if (tau <= 0) {
        if (!use_ref) {
            tau = 64;
        } else {
            // autotune: time a solve at each candidate block size on a sample of
            // (up to) 16 systems with a reduced iteration cap; keep the fastest
            // per converged system
            std::vector<char> sample(h->count, 0);
            const int stride = std::max(1, h->count / 16);
            for (int i = 0; i < h->count; i += stride) sample[i] = 1;
            // candidates: block size and, for blocks of 16 or 32 columns, the column step's tile
            // shape (16-byte vectors over tau/4 lanes of a row, or one lane per column)
            double best = 1e300;
            int best_tau = 64, best_path = 0;
            const int64_t trial_cap = std::min<int64_t>(max_iter, 20000);
            const int cands[][2] = {{16, 0}, {16, 1}, {32, 0}, {32, 1}, {64, 0}, {128, 0}, {256, 0}};
            for (const auto &cand : cands) {
                rebk_batch_stats s;
                h->col_path = cand[1];
                rebk_status rs = run_batch(h, cand[0], tol, trial_cap, inner_iters, seed, true, false, &s, &sample);
                if (rs != REBK_OK) return rs;
                const double score = s.device_ms / std::max(1, s.converged);
                if (score < best) {
                    best = score;
                    best_tau = cand[0];
                    best_path = cand[1];
                }
            }
            tau = best_tau;
            h->tau = tau;
            h->col_path = best_path;
        }
    }
    rebk_status rs = run_batch(h, tau, tol, max_iter, inner_iters, seed, use_ref, true, stats);
    if (rs != REBK_OK) return rs;
    batch_unpack_kernel<<<blocks_for(h->Nrows * h->nrhs, 256), 256, 0, st>>>(h->Nrows, h->nrhs, h->Xi, X);
    if (h->rec_z)
        batch_unpack_kernel<<<blocks_for(h->Mrows * h->nrhs, 256), 256, 0, st>>>(h->Mrows, h->nrhs, h->Z, h->rec_z);
    BCK(cudaGetLastError());
    if (status_out) BCK(cudaMemcpyAsync(status_out, h->status, sizeof(int) * h->count, cudaMemcpyDeviceToDevice, st));
    BCK(cudaStreamSynchronize(st));
    return REBK_OK;
}

extern "C" rebk_status rebk_batch_solve(rebk_batch h, const double *B, double *X, const double *X_ref,
                                        double tol, int64_t max_iter, int64_t inner_iters, uint64_t seed,
                                        int32_t *status_out, rebk_batch_stats *stats) {
    return rebk_batch_solve_ex(h, B, X, X_ref, nullptr, nullptr, tol, max_iter, inner_iters, seed, status_out,
                               stats);
}
