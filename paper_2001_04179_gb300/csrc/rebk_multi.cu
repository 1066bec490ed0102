// rebk_multi.cu -- Algorithm 1 for several right-hand sides of one matrix at once.
//
// Every right-hand side follows Algorithm 1 of Du, Si, Sun (arXiv:2001.04179),
// Section 2, in the correction form of the mixed-precision solve, and all of them
// use the same block sequence (the draws depend on the norms of A only).  For NR
// right-hand sides with FP32 corrections dZ (m x NR), dX (n x NR), duals S
// (n x NR), V (m x NR) and the FP32-rounded residuals F = B - Z - A X, G = A^T Z:
//   W  = A_J^T dZ + G_J,        dZ <- dZ - cJ A_J W,     S_J += cJ W,
//   Rr = A_I dX - F_I + dZ_I,   dX <- dX - cI A_I^T Rr,  V_I -= cI Rr,
// with cJ = alpha / ||A_J||_F^2 and cI = alpha / ||A_I||_F^2.  One read of a
// sampled block serves NR right-hand sides, so the device-wide reduction chain
// that bounds the one-right-hand-side kernel is shared by NR solves.
//
// GB300 mapping.  One cooperative launch, one CTA of 512 threads per SM.  CTA c
// owns the rows R_c (its dZ and V rows) and the 8-aligned columns C_c (its dX and
// S columns).  One device-wide barrier per iteration; round t, in three stages
// that each end in a CTA barrier,
//   A. reads Rr^{t-1} and W^t (one pass over the accumulators),
//   B. finishes iteration t-1's row step on the owned columns and does iteration
//      t's column step on the owned rows (independent of each other),
//   C. adds its partials of Rr^t (A_{I_t, C_c} dX, plus dZ_I - F_I on owned rows)
//      and of W^{t+1} (A_{R_c, J_{t+1}}^T dZ) into the next of three rotating
//      accumulator sets (2 replicas, red.global.add.v4.f32 over 4 right-hand
//      sides at a time), clears its share of the set after that, and arrives.
// Tiles of the sampled blocks (FP32 or BF16 storage) reach shared memory by 2-D
// TMA copies, two buffers per kind: a column tile serves the partial of W in one
// round and the column step of the next, a row tile the partial of Rr in one
// round and the row step of the next, so each tile is read from HBM once.
//
// With FP32 storage and groups of 8 the four products run on tensor cores:
// mma.sync m16n8k8 with three TF32 products per step (a_hi b_hi + a_hi b_lo +
// a_lo b_hi, hi = the top 19 bits, lo = the FP32 remainder), which keeps FP32
// accuracy to about 2^-20 relative; the (16-row tile, K step) pairs of a stage's
// two products are split evenly over the 16 warps, whose tile sums meet in two
// shared buffers.  Each product
// is 128 x 136 x 8 or smaller, too small for the asynchronous tcgen05 issue /
// commit / TMEM read-back to pay inside a step that a device-wide reduction
// bounds; the warp-level form cuts the instructions of a step about sixfold
// against the FP32 FMA form below.
//
// Otherwise products along tile rows (Rr partials, the column step) run a warp per row with
// the vector of each half-warp's NR/2 right-hand sides held in registers and a
// half-warp butterfly that ends with each sum on one lane; products along tile
// columns (the row step, W partials) run a thread per (column, 4 right-hand
// sides) with the rows split over spare threads through a shared scratch.
//
// The FP64 helpers of the refinement loop (A P and A^T Q for NR vectors, norms,
// the residual and update steps) follow the kernel.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {
namespace {

constexpr int kMT = 512, kMW = kMT / 32;
constexpr int kCMx = 9;  // 16-column chunks of dX a half-warp holds in registers (144 columns)
constexpr int kCMw = 8;  // 16-column chunks of w a half-warp holds in registers (128 columns)

__device__ __forceinline__ uint32_t m_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void m_mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(m_smem(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void m_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(m_smem(bar)), "r"(bytes)
                 : "memory");
}

// Waits for the phase with the given parity; false after timeout_ns.
__device__ __forceinline__ bool m_wait(uint64_t *bar, uint32_t parity, unsigned long long timeout_ns) {
    uint32_t done = 0;
    unsigned long long t0 = 0;
    for (uint32_t spins = 0;; ++spins) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(m_smem(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (spins == 0) t0 = globaltimer_ns();
        if ((spins & 63u) == 63u && globaltimer_ns() - t0 > timeout_ns) return false;
    }
}

__device__ __forceinline__ void m_tma_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(m_smem(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(m_smem(bar))
        : "memory");
}

__device__ __forceinline__ void m_red4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

template <typename TA> __device__ __forceinline__ float m_ld(const TA *p);
template <> __device__ __forceinline__ float m_ld<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float m_ld<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}

// Sums H values over the 16 lanes of each half-warp.  Afterwards lane L with
// (L & 15) % (16 / H) == 0 holds the sum of value (L & 15) / (16 / H).
template <int H> __device__ __forceinline__ float half_reduce(const float (&s)[H], int lane);

template <> __device__ __forceinline__ float half_reduce<4>(const float (&s)[4], int lane) {
    const bool b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
    const float a0 = (b3 ? s[2] : s[0]) + __shfl_xor_sync(0xffffffffu, b3 ? s[0] : s[2], 8);
    const float a1 = (b3 ? s[3] : s[1]) + __shfl_xor_sync(0xffffffffu, b3 ? s[1] : s[3], 8);
    float c = (b2 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, b2 ? a0 : a1, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

template <> __device__ __forceinline__ float half_reduce<2>(const float (&s)[2], int lane) {
    const bool b3 = (lane & 8) != 0;
    float c = (b3 ? s[1] : s[0]) + __shfl_xor_sync(0xffffffffu, b3 ? s[0] : s[1], 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// out_l[q] = sum_{c < width} T[l ld + c] u[q us + c] for rows l < rows: a warp per
// row; the 16 lanes of half h hold u for q in [H h, H h + H) over 16 CM columns in
// registers (wider rows run in segments).  deliver(l, v, first_segment) is called
// by every lane of the warp; v as half_reduce leaves it.
template <typename TA, int NR, int CM, typename Deliver>
__device__ __forceinline__ void row_products(const TA *T, int ld, int rows, int width, const float *u, int us,
                                             int warp, int lane, Deliver deliver) {
    constexpr int H = NR / 2;
    const int h = lane >> 4, cl = lane & 15;
    for (int seg = 0; seg == 0 || seg < width; seg += 16 * CM) {
        float ur[CM][H];
#pragma unroll
        for (int k = 0; k < CM; ++k) {
            const int c = seg + cl + 16 * k;
#pragma unroll
            for (int i = 0; i < H; ++i) ur[k][i] = c < width ? u[(H * h + i) * us + c] : 0.f;
        }
        for (int l = warp; l < rows; l += kMW) {
            float s[H];
#pragma unroll
            for (int i = 0; i < H; ++i) s[i] = 0.f;
            const TA *row = T + (size_t)l * ld;
#pragma unroll
            for (int k = 0; k < CM; ++k) {
                const int c = seg + cl + 16 * k;
                const float av = c < width ? m_ld<TA>(row + c) : 0.f;
#pragma unroll
                for (int i = 0; i < H; ++i) s[i] = fmaf(av, ur[k][i], s[i]);
            }
            deliver(l, half_reduce<H>(s, lane), seg == 0);
        }
    }
}

// out_c[q] = sum_{l < rows} T[l ld + c] v[l NR + q] for columns c < width: a
// thread per (column, group of 4 right-hand sides), the rows split RG ways over
// the spare threads when the scratch holds the RG partial results.
// deliver(c, g, s) receives the sums of right-hand sides 4 g .. 4 g + 3.
template <typename TA, int NR, typename Deliver>
__device__ __forceinline__ void col_products(const TA *T, int ld, int rows, int width, const float *v, float *scr,
                                             int scr_floats, int tid, Deliver deliver) {
    constexpr int NG = NR / 4;
    const int units = width * NG;
    if (units == 0 || rows == 0) return;
    int RG = kMT / units;
    if (RG > rows) RG = rows;
    if (RG > scr_floats / (width * NR)) RG = scr_floats / (width * NR);
    if (RG < 1) RG = 1;
    for (int e = tid; e < units * RG; e += kMT) {
        const int c = e % width, g = (e / width) % NG, rg = e / units;
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        for (int l = rg; l < rows; l += RG) {
            const float av = m_ld<TA>(T + (size_t)l * ld + c);
            const float4 vv = *reinterpret_cast<const float4 *>(v + l * NR + 4 * g);
            s[0] = fmaf(av, vv.x, s[0]);
            s[1] = fmaf(av, vv.y, s[1]);
            s[2] = fmaf(av, vv.z, s[2]);
            s[3] = fmaf(av, vv.w, s[3]);
        }
        if (RG == 1) {
            deliver(c, g, s);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) scr[((size_t)rg * NR + 4 * g + i) * width + c] = s[i];
        }
    }
    if (RG > 1) {
        __syncthreads();
        for (int e = tid; e < units; e += kMT) {
            const int c = e % width, g = e / width;
            float s[4] = {0.f, 0.f, 0.f, 0.f};
            for (int rg = 0; rg < RG; ++rg) {
#pragma unroll
                for (int i = 0; i < 4; ++i) s[i] += scr[((size_t)rg * NR + 4 * g + i) * width + c];
            }
            deliver(c, g, s);
        }
    }
}

__device__ __forceinline__ uint32_t tf32_hi(float a) { return __float_as_uint(a) & 0xffffe000u; }

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One product of mma_pair: Y (rows up to M rounded up to 16, 8 columns,
// row-major; zero on entry) += A B for the M x K matrix A(m, k) = A[m am + k ak]
// and the K x 8 matrix B(k, q) = B[k bk + q bq] in shared memory.  Reads A for
// rows up to M rounded up to 16 and columns up to K rounded up to 8, B for rows
// up to K rounded up to 8: B must be zero there, A finite and in bounds.
struct MmaProd {
    const float *A;
    int am, ak, M;
    const float *B;
    int bk, bq, K;
    float *Y;
};

// (16-row tile, K step) pairs lo .. hi - 1 (tile-major) of one product on one warp;
// each tile's sum goes to Y by shared-memory atomics when the warp leaves it.
__device__ __forceinline__ void mma_range(const MmaProd &p, int lo, int hi, int lane) {
    const int KS = (p.K + 7) >> 3;
    const int g = lane >> 2, t = lane & 3;
    const int am = p.am, ak = p.ak, bk = p.bk;
    int mt = lo / KS, ks = lo - mt * KS;
    const float *pb = p.B + t * bk + g * p.bq;
    // three accumulators (lo*hi, hi*lo, hi*hi): independent chains of tensor-core operations
    float d[4] = {0.f, 0.f, 0.f, 0.f}, e1[4] = {0.f, 0.f, 0.f, 0.f}, e2[4] = {0.f, 0.f, 0.f, 0.f};
    auto flush = [&]() {
        float *y = p.Y + (mt * 16 + g) * 8 + 2 * t;
        atomicAdd(y, d[0] + (e1[0] + e2[0]));
        atomicAdd(y + 1, d[1] + (e1[1] + e2[1]));
        atomicAdd(y + 64, d[2] + (e1[2] + e2[2]));
        atomicAdd(y + 65, d[3] + (e1[3] + e2[3]));
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = e1[i] = e2[i] = 0.f;
    };
    const float *pa = p.A + (mt * 16 + g) * am + t * ak;
#pragma unroll 2
    for (int idx = lo; idx < hi; ++idx) {
        if (ks == KS) {
            flush();
            ++mt;
            ks = 0;
            pa += 16 * am;
        }
        const int ko = ks * 8;
        const float af[4] = {pa[ko * ak], pa[ko * ak + 8 * am], pa[(ko + 4) * ak], pa[(ko + 4) * ak + 8 * am]};
        const float bf0 = pb[ko * bk], bf1 = pb[(ko + 4) * bk];
        uint32_t ah[4], al[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ah[i] = tf32_hi(af[i]);
            al[i] = __float_as_uint(af[i] - __uint_as_float(ah[i]));
        }
        const uint32_t bh0 = tf32_hi(bf0), bh1 = tf32_hi(bf1);
        const uint32_t bl0 = __float_as_uint(bf0 - __uint_as_float(bh0));
        const uint32_t bl1 = __float_as_uint(bf1 - __uint_as_float(bh1));
        mma_tf32(e1, al, bh0, bh1);
        mma_tf32(e2, ah, bl0, bl1);
        mma_tf32(d, ah, bh0, bh1);
        ++ks;
    }
    flush();
}

// Two independent products on tensor cores in one pass: the (tile, K step) pairs
// of both (the first product's first) are split into 16 equal shares, one per warp.
__device__ __forceinline__ void mma_pair(const MmaProd &p1, const MmaProd &p2, int warp, int lane) {
    const int T1 = (p1.M > 0 && p1.K > 0) ? ((p1.M + 15) >> 4) * ((p1.K + 7) >> 3) : 0;
    const int T2 = (p2.M > 0 && p2.K > 0) ? ((p2.M + 15) >> 4) * ((p2.K + 7) >> 3) : 0;
    const int T = T1 + T2;
    const int lo = warp * T / kMW, hi = (warp + 1) * T / kMW;
    if (lo < T1 && lo < hi) mma_range(p1, lo, hi < T1 ? hi : T1, lane);
    if (hi > T1 && lo < hi) mma_range(p2, (lo > T1 ? lo : T1) - T1, hi - T1, lane);
}

template <typename TA, int NR, bool MMA>
__global__ void __launch_bounds__(kMT, 1) rebk_multi_kernel(const __grid_constant__ MultiArgs M) {
    extern __shared__ __align__(128) unsigned char msm[];
    const GridArgs &a = M.geo;
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t m = a.m, n = a.n;
    const int64_t nu = (n + 7) / 8;
    const int64_t r0 = m * cta / G, r1 = m * (cta + 1) / G;
    const int64_t c0 = 8 * (nu * cta / G) < n ? 8 * (nu * cta / G) : n;
    const int64_t c1 = 8 * (nu * (cta + 1) / G) < n ? 8 * (nu * (cta + 1) / G) : n;
    const int nrow = (int)(r1 - r0), ncol = (int)(c1 - c0);
    const int64_t K = a.iters;
    const int tau_r = a.tau_r;
    const int xs = multi_xs(a.ncol_cap), ws = multi_ws(a.tau_c);
    const MultiSmem L = multi_smem_layout(a.nrow_cap, a.ncol_cap, a.tau_r, a.tau_c, NR, a.tile_c_bytes,
                                          a.tile_r_bytes, M.scr_floats);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(msm);    // [0, 1] column tiles, [2, 3] row tiles
    int *flags = reinterpret_cast<int *>(msm + 64);        // [0] non-finite, [1] a copy wait gave up, [2] barrier
    // ring of upcoming draws and step coefficients, slot u & 7 for iteration u:
    // J_u, I_u, alpha / ||A_{:,J_u}||_F^2, alpha / ||A_{I_u,:}||_F^2 (thread 0 fills it
    // three iterations ahead, so no dependent global load sits on a round's path)
    int *ring_j = reinterpret_cast<int *>(msm + 128), *ring_i = ring_j + 8;
    float *ring_cj = reinterpret_cast<float *>(msm + 192), *ring_ci = ring_cj + 8;
    TA *const tc0 = reinterpret_cast<TA *>(msm + L.tc0), *const tc1 = reinterpret_cast<TA *>(msm + L.tc1);
    TA *const tr0 = reinterpret_cast<TA *>(msm + L.tr0), *const tr1 = reinterpret_cast<TA *>(msm + L.tr1);
    auto tcb = [&](int64_t b) { return (b & 1) ? tc1 : tc0; };
    auto trb = [&](int64_t b) { return (b & 1) ? tr1 : tr0; };
    float *zeta = reinterpret_cast<float *>(msm + L.zeta);  // [nrow][NR]: dZ of the owned rows
    float *xi = reinterpret_cast<float *>(msm + L.xi);      // [NR][xs]: dX of the owned columns
    float *sw = reinterpret_cast<float *>(msm + L.w);       // [NR][ws]: W of the current column block
    float *sr = reinterpret_cast<float *>(msm + L.r);       // [tau_r][NR]: Rr of the previous row block
    float *scr = reinterpret_cast<float *>(msm + L.scr);
    const float *coef_r = static_cast<const float *>(a.coef_r);
    const float *coef_c = static_cast<const float *>(a.coef_c);
    const int aw = a.acc_w;
    const int64_t accset = (int64_t)kMultiReplicas * aw;
    float *acc = static_cast<float *>(a.acc);
    const int rep = cta % kMultiReplicas;
    const int64_t clr0 = accset * cta / G, clr1 = accset * (cta + 1) / G;

    auto col_range = [&](int j, int64_t *ja, int64_t *jb) {
        if (a.col_off) {
            *ja = __ldg(a.col_off + j);
            *jb = __ldg(a.col_off + j + 1);
        } else {
            *ja = (int64_t)j * a.tau_c;
            *jb = *ja + a.tau_c < n ? *ja + a.tau_c : n;
        }
    };
    auto row_range = [&](int i, int64_t *ia, int64_t *ib) {
        if (a.row_off) {
            *ia = __ldg(a.row_off + i);
            *ib = __ldg(a.row_off + i + 1);
        } else {
            *ia = (int64_t)i * tau_r;
            *ib = *ia + tau_r < m ? *ia + tau_r : m;
        }
    };
    auto jdraw = [&](int64_t t) { return ring_j[t & 7]; };
    auto idraw = [&](int64_t t) { return ring_i[t & 7]; };

    {  // zero everything after the header: tile slack, the padding of the vectors
        uint4 *p = reinterpret_cast<uint4 *>(msm + 512);
        const int words = (int)((L.total - 512) / 16);
        for (int e = tid; e < words; e += kMT) p[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    for (int e = tid; e < nrow * NR; e += kMT) zeta[e] = M.dZ[r0 * NR + e];
    for (int e = tid; e < ncol * NR; e += kMT) xi[(e % NR) * xs + e / NR] = M.dX[c0 * NR + e];
    // thread 0's draw pipeline: indices of iteration t + 4 load at the start of round
    // t, coefficients of iteration t + 3 at the start of round t, and the ring slot of
    // iteration t + 3 is written at the end of round t
    int nj = 0, ni = 0, wj = 0, wi = 0;
    float wcj = 0.f, wci = 0.f;
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) m_mbar_init(&mbar[i], 1);
        flags[0] = 0;
        flags[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int64_t u = 1; u <= 3 && u <= K; ++u) {
            const int j = __ldg(a.idx + 2 * (u - 1)), i = __ldg(a.idx + 2 * (u - 1) + 1);
            ring_j[u & 7] = j;
            ring_i[u & 7] = i;
            ring_cj[u & 7] = __ldg(coef_c + j);
            ring_ci[u & 7] = __ldg(coef_r + i);
        }
        if (K >= 4) {
            nj = __ldg(a.idx + 6);
            ni = __ldg(a.idx + 7);
        }
    }
    __syncthreads();
    // G_J of the next column block, read a round ahead (entry tid + k * kMT)
    float gpre[4] = {0.f, 0.f, 0.f, 0.f};
    auto prefetch_g = [&](int64_t u) {
        if (u > K) return;
        int64_t ja, jb;
        col_range(jdraw(u), &ja, &jb);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = tid + k * kMT;
            if (e < (int)(jb - ja) * NR) gpre[k] = __ldg(M.G + ja * NR + e);
        }
    };
    // duals of the owned rows (V) and columns (S): entry e = tid + k * kMT of the CTA's
    // slice stays in a register for the whole launch (the CTA is its only writer);
    // slices longer than 4 * kMT entries keep the rest in global memory
    float vreg[4], sreg[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int e = tid + k * kMT;
        vreg[k] = e < nrow * NR ? M.V[r0 * NR + e] : 0.f;
        sreg[k] = e < ncol * NR ? M.S[c0 * NR + e] : 0.f;
    }

    // Tiles: the column tile of J_t in column buffer t & 1, the row tile of I_t in
    // row buffer t & 1.  Every thread tracks the phases; thread 0 issues.
    // per buffer b: phase parity (bit b) and copy in flight (bit 2 + b), in registers
    uint32_t cst = 0u, rst = 0u;
    int64_t cxa = 0, cxb = 0;  // first column of the copied box, column buffers 0 and 1
    auto cx0 = [&](int64_t b) { return (b & 1) ? cxb : cxa; };
    auto issue_c = [&](int64_t t) {
        if (t < 1 || t > K || nrow == 0) return;
        const int b = (int)(t & 1);
        int64_t ja, jb;
        col_range(jdraw(t), &ja, &jb);
        const int x0 = (int)(ja & ~(int64_t)(a.tma_vx - 1));
        if (b) cxb = x0;
        else cxa = x0;
        cst |= 4u << b;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            m_expect_tx(&mbar[b], (uint32_t)a.tile_c_bytes_tx);
            for (int bx = 0; bx < a.nbox_c; ++bx)
                m_tma_2d(tcb(b) + (size_t)bx * a.bh_c * a.bw_c, &a.tmap_c, x0, (int)(r0 + (int64_t)bx * a.bh_c),
                         &mbar[b]);
        }
    };
    auto issue_r = [&](int64_t t) {
        if (t < 1 || t > K || ncol == 0) return;
        const int b = (int)(t & 1);
        rst |= 4u << b;
        if (tid == 0) {
            int64_t ia, ib;
            row_range(idraw(t), &ia, &ib);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            m_expect_tx(&mbar[2 + b], (uint32_t)a.tile_r_bytes_tx);
            m_tma_2d(trb(b), &a.tmap_r, (int)c0, (int)ia, &mbar[2 + b]);
        }
    };
    auto wait_c = [&](int64_t t) {
        const int b = (int)(t & 1);
        if (!(cst & (4u << b))) return;
        if (m_wait(&mbar[b], (cst >> b) & 1u, a.timeout_ns)) {
            cst ^= 1u << b;
            cst &= ~(4u << b);
        } else {
            flags[1] = 1;
        }
    };
    auto wait_r = [&](int64_t t) {
        const int b = (int)(t & 1);
        if (!(rst & (4u << b))) return;
        if (m_wait(&mbar[2 + b], (rst >> b) & 1u, a.timeout_ns)) {
            rst ^= 1u << b;
            rst &= ~(4u << b);
        } else {
            flags[1] = 1;
        }
    };
    // partial of W^t over the owned rows (column tile of J_t) into accumulator set dst
    // MMA scratch: the two products of a stage accumulate in two zeroed buffers
    float *Y1 = scr, *Y2x = scr + ((a.ncol_cap + 15) & ~15) * 8, *Y2w = scr + ((a.tau_r + 15) & ~15) * 8;
    // W partials (rows j < wc of Y) into accumulator set dst; Y zeroed for reuse
    auto deliver_w = [&](const float *Yc, int wc, float *dst) {
        float *base = dst + (int64_t)rep * aw + tau_r * NR;
        for (int e = tid; e < ((wc + 15) & ~15) * 2; e += kMT) {
            float4 *y = reinterpret_cast<float4 *>(const_cast<float *>(Yc)) + e;
            const float4 v = *y;
            *y = make_float4(0.f, 0.f, 0.f, 0.f);
            if ((e >> 1) < wc) m_red4(base + (e >> 1) * NR + 4 * (e & 1), v.x, v.y, v.z, v.w);
        }
    };
    // partial of W^t over the owned rows (column tile of J_t) into accumulator set dst
    auto partial_w = [&](int64_t t, float *dst) {
        int64_t ja, jb;
        col_range(jdraw(t), &ja, &jb);
        const TA *T = tcb(t) + (ja - cx0(t));
        const int wc = (int)(jb - ja);
        if constexpr (MMA) {
            const MmaProd none{nullptr, 0, 0, 0, nullptr, 0, 0, 0, nullptr};
            const MmaProd pw{reinterpret_cast<const float *>(T), 1, a.bw_c, wc, zeta, NR, 1, nrow, Y2w};
            mma_pair(none, pw, warp, lane);
            __syncthreads();
            deliver_w(Y2w, wc, dst);
        } else {
            float *base = dst + (int64_t)rep * aw + tau_r * NR;
            col_products<TA, NR>(T, a.bw_c, nrow, wc, zeta, scr, M.scr_floats, tid,
                                 [&](int j, int g, const float(&s)[4]) {
                                     m_red4(base + j * NR + 4 * g, s[0], s[1], s[2], s[3]);
                                 });
        }
    };

    int64_t done = K;
    bool alive = K >= 1;
    issue_c(1);
    issue_c(2);
    issue_r(1);
    if (alive) {
        wait_c(1);
        __syncthreads();
        if (flags[1]) {
            if (tid == 0) atomicExch(a.status, 6);
            alive = false;
            done = 0;
        } else {
            partial_w(1, acc);
        }
        prefetch_g(1);
    }
    grid_arrive(a.bar);
    for (int64_t t = 1; alive && t <= K + 1; ++t) {
        if (!grid_wait(a.bar, (unsigned)G * (unsigned)t, a.status, a.timeout_ns, flags + 2)) {
            done = t >= 2 ? t - 2 : 0;
            break;
        }
        const float *accS = acc + ((t - 1) % 3) * accset;
        if (tid == 0 && t + 3 <= K) {
            wj = nj;
            wi = ni;
            wcj = __ldg(coef_c + wj);
            wci = __ldg(coef_r + wi);
            if (t + 4 <= K) {
                nj = __ldg(a.idx + 2 * (t + 3));
                ni = __ldg(a.idx + 2 * (t + 3) + 1);
            }
        }
        // ---- A. Rr^{t-1} and W^t from the accumulators ----
        const bool rowstep = t >= 2, colstep = t <= K;
        int64_t ia = 0, ib = 0, ja = 0, jb = 0;
        if (rowstep) row_range(idraw(t - 1), &ia, &ib);
        if (colstep) col_range(jdraw(t), &ja, &jb);
        const int hr = (int)(ib - ia), wc = (int)(jb - ja);
        for (int e = tid; e < ((hr + 7) & ~7) * NR; e += kMT) {
            float v = 0.f;
            if (e < hr * NR) {
#pragma unroll
                for (int q = 0; q < kMultiReplicas; ++q) v += __ldcg(accS + (int64_t)q * aw + e);
            }
            sr[e] = v;
            if (!isfinite(v)) flags[0] = 1;
        }
        auto fill_w = [&](int e, float g) {
            float v = 0.f;
            if (e < wc * NR) {
                v = g;
#pragma unroll
                for (int q = 0; q < kMultiReplicas; ++q) v += __ldcg(accS + (int64_t)q * aw + tau_r * NR + e);
            }
            sw[(e % NR) * ws + e / NR] = v;
            if (!isfinite(v)) flags[0] = 1;
        };
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (tid + k * kMT < ((wc + 7) & ~7) * NR) fill_w(tid + k * kMT, gpre[k]);
        for (int e = tid + 4 * kMT; e < ((wc + 7) & ~7) * NR; e += kMT)
            fill_w(e, e < wc * NR ? __ldg(M.G + ja * NR + e) : 0.f);
        __syncthreads();
        if (flags[0]) {
            if (tid == 0) atomicExch(a.status, 5);
            done = t >= 2 ? t - 2 : 0;
            break;
        }
        const float cI = rowstep ? ring_ci[(t - 1) & 7] : 0.f, cJ = colstep ? ring_cj[t & 7] : 0.f;
        // ---- B. row step of iteration t-1 (owned columns), column step of iteration t (owned rows) ----
        if constexpr (MMA) {
            const MmaProd px{reinterpret_cast<const float *>(trb(t - 1)), 1, a.bw_r, rowstep ? ncol : 0, sr, NR, 1,
                             hr, Y1};
            const MmaProd pz{reinterpret_cast<const float *>(tcb(t) + (ja - cx0(t))), a.bw_c, 1, colstep ? nrow : 0,
                             sw, 1, ws, wc, Y2x};
            mma_pair(px, pz, warp, lane);
            __syncthreads();
            if (rowstep) {
                for (int e = tid; e < ((ncol + 15) & ~15) * NR; e += kMT) {
                    const float v = Y1[e];
                    Y1[e] = 0.f;
                    if ((e >> 3) < ncol) xi[(e & 7) * xs + (e >> 3)] -= cI * v;
                }
            }
            if (colstep) {
                for (int e = tid; e < ((nrow + 15) & ~15) * NR; e += kMT) {
                    const float v = Y2x[e];
                    Y2x[e] = 0.f;
                    if (e < nrow * NR) zeta[e] -= cJ * v;
                }
            }
        } else {
            if (rowstep)
                col_products<TA, NR>(trb(t - 1), a.bw_r, hr, ncol, sr, scr, M.scr_floats, tid,
                                     [&](int c, int g, const float(&s)[4]) {
#pragma unroll
                                         for (int i = 0; i < 4; ++i) xi[(4 * g + i) * xs + c] -= cI * s[i];
                                     });
            if (colstep) {
                constexpr int SP = 16 / (NR / 2);
                row_products<TA, NR, kCMw>(tcb(t) + (ja - cx0(t)), a.bw_c, nrow, wc, sw, ws, warp, lane,
                                           [&](int rl, float v, bool) {
                                               if ((lane & (SP - 1)) == 0)
                                                   zeta[rl * NR + (NR / 2) * (lane >> 4) + (lane & 15) / SP] -=
                                                       cJ * v;
                                           });
            }
        }
        if (rowstep) {  // dual V on the owned rows of I_{t-1}
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = tid + k * kMT;
                const int64_t row = r0 + e / NR;
                if (e < nrow * NR && row >= ia && row < ib) vreg[k] -= cI * sr[(row - ia) * NR + e % NR];
            }
            for (int e = tid + 4 * kMT; e < nrow * NR; e += kMT) {
                const int64_t row = r0 + e / NR;
                if (row >= ia && row < ib) M.V[r0 * NR + e] -= cI * sr[(row - ia) * NR + e % NR];
            }
        }
        if (colstep) {  // dual S on the owned columns of J_t
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = tid + k * kMT;
                const int64_t c = c0 + e / NR;
                if (e < ncol * NR && c >= ja && c < jb) sreg[k] += cJ * sw[(e % NR) * ws + (c - ja)];
            }
            for (int e = tid + 4 * kMT; e < ncol * NR; e += kMT) {
                const int64_t c = c0 + e / NR;
                if (c >= ja && c < jb) M.S[c0 * NR + e] += cJ * sw[(e % NR) * ws + (c - ja)];
            }
        }
        __syncthreads();
        issue_r(t + 1);  // the buffer of I_{t-1} takes I_{t+1}
        if (!colstep) break;  // t = K + 1: the last row step is done
        issue_c(t + 2);       // the buffer of J_t takes J_{t+2}
        // ---- C. partials of Rr^t and W^{t+1} into set t % 3 ----
        float *accT = acc + (t % 3) * accset;
        const bool wnext = t + 1 <= K;
        wait_r(t);
        if (wnext) wait_c(t + 1);
        __syncthreads();
        if (flags[1]) {
            if (tid == 0) atomicExch(a.status, 6);
            done = t - 1;
            break;
        }
        int64_t ia2, ib2, ja2 = 0, jb2 = 0;
        row_range(idraw(t), &ia2, &ib2);
        if (wnext) col_range(jdraw(t + 1), &ja2, &jb2);
        const int hr2 = (int)(ib2 - ia2), wc2 = (int)(jb2 - ja2);
        float *rbase = accT + (int64_t)rep * aw;
        // Rr^t = A_{I_t, C_c} dX^{t-1} (+ dZ^t_I - F_I on the owned rows), 4 right-hand sides per red
        auto deliver_r = [&](int l, int q0, float (&o)[4], bool first) {
            const int64_t row = ia2 + l;
            const bool own = first && row >= r0 && row < r1;
            if (ncol == 0 && !own) return;
            if (own) {
#pragma unroll
                for (int i = 0; i < 4; ++i) o[i] += zeta[(row - r0) * NR + q0 + i] - M.F[row * NR + q0 + i];
            }
            m_red4(rbase + l * NR + q0, o[0], o[1], o[2], o[3]);
        };
        if constexpr (MMA) {
            const MmaProd pr{reinterpret_cast<const float *>(trb(t)), a.bw_r, 1, hr2, xi, 1, xs, ncol, Y1};
            const MmaProd pw{reinterpret_cast<const float *>(tcb(t + 1) + (ja2 - cx0(t + 1))), 1, a.bw_c, wc2, zeta, NR,
                             1, nrow, Y2w};
            mma_pair(pr, pw, warp, lane);
            __syncthreads();
            for (int e = tid; e < ((hr2 + 15) & ~15) * 2; e += kMT) {
                float4 *y = reinterpret_cast<float4 *>(Y1) + e;
                const float4 v = *y;
                *y = make_float4(0.f, 0.f, 0.f, 0.f);
                float o[4] = {v.x, v.y, v.z, v.w};
                if ((e >> 1) < hr2) deliver_r(e >> 1, 4 * (e & 1), o, true);
            }
            if (wnext) deliver_w(Y2w, wc2, accT);
        } else {
            const int src0 = NR == 8 ? (lane & 16) : 0, step = NR == 8 ? 4 : 8;
            const bool writer = NR == 8 ? (lane & 15) == 0 : lane == 0;
            const int q0 = NR == 8 ? 4 * (lane >> 4) : 0;
            row_products<TA, NR, kCMx>(trb(t), a.bw_r, hr2, ncol, xi, xs, warp, lane,
                                       [&](int l, float v, bool first) {
                                           float o[4];
#pragma unroll
                                           for (int i = 0; i < 4; ++i) o[i] = __shfl_sync(0xffffffffu, v, src0 + step * i);
                                           if (writer) deliver_r(l, q0, o, first);
                                       });
            if (wnext) partial_w(t + 1, accT);
        }
        {  // this CTA's share of the set that round t + 1 fills
            float *accN = acc + ((t + 1) % 3) * accset;
            for (int64_t e = clr0 + tid; e < clr1; e += kMT) accN[e] = 0.f;
        }
        prefetch_g(t + 1);
        if (tid == 0 && t + 3 <= K) {
            const int u = (int)((t + 3) & 7);
            ring_j[u] = wj;
            ring_i[u] = wi;
            ring_cj[u] = wcj;
            ring_ci[u] = wci;
        }
        grid_arrive(a.bar);
    }
    // no tensor copy may still be writing shared memory when the CTA leaves
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            if (cst & (4u << b)) m_wait(&mbar[b], (cst >> b) & 1u, a.timeout_ns);
            if (rst & (4u << b)) m_wait(&mbar[2 + b], (rst >> b) & 1u, a.timeout_ns);
        }
    }
    __syncthreads();
    for (int e = tid; e < nrow * NR; e += kMT) M.dZ[r0 * NR + e] = zeta[e];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int e = tid + k * kMT;
        if (e < nrow * NR) M.V[r0 * NR + e] = vreg[k];
        if (e < ncol * NR) M.S[c0 * NR + e] = sreg[k];
    }
    for (int e = tid; e < ncol * NR; e += kMT) M.dX[c0 * NR + e] = xi[(e % NR) * xs + e / NR];
    if (cta == 0 && tid == 0) *a.iters_done = done;
}

template <typename TA, int NR, bool MMA> void *multi_ptr() {
    return reinterpret_cast<void *>(&rebk_multi_kernel<TA, NR, MMA>);
}

void *multi_kernel(bool bf16, int nr, bool mma) {
    if (bf16) return nr == 8 ? multi_ptr<__nv_bfloat16, 8, false>() : multi_ptr<__nv_bfloat16, 4, false>();
    if (nr == 8) return mma ? multi_ptr<float, 8, true>() : multi_ptr<float, 8, false>();
    return multi_ptr<float, 4, false>();
}

// ---------------------------------------------------------------------------
// FP64 helpers of the refinement loop.  On GB300 the FP64 pipe, not memory,
// bounds these products (2 NR FMAs per matrix entry), so each is laid out to
// spend FP64 instructions on the products alone: no cross-lane FP64 sums.
// ---------------------------------------------------------------------------
constexpr int kApSeg = 1024;  // columns per warp in multi_ap

template <typename T> __device__ __forceinline__ double ldd(const T *p) { return (double)__ldg(p); }

// Y[i][q] += sum over one column segment of A[i][c] P[c][q]: a lane per row, the
// vector entries of a column broadcast to the warp.
template <typename TP, int NR>
__global__ void __launch_bounds__(256) multi_ap_kernel(const double *__restrict__ A, int64_t lda, int64_t m,
                                                       int64_t n, const TP *__restrict__ P, double *Y) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int64_t segs = (n + kApSeg - 1) / kApSeg;
    const int64_t rg = wid / segs, sg = wid % segs;
    const int64_t i = rg * 32 + lane;
    if (rg * 32 >= m) return;
    const int64_t ca = sg * kApSeg, cb = ca + kApSeg < n ? ca + kApSeg : n;
    const bool ok = i < m;
    const double *row = A + (ok ? i : 0) * lda;
    double s[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) s[q] = 0.0;
    for (int64_t c = ca; c < cb; ++c) {
        const double av = ok ? __ldg(row + c) : 0.0;
#pragma unroll
        for (int q = 0; q < NR; ++q) s[q] = fma(av, ldd(P + c * NR + q), s[q]);
    }
    if (ok) {
#pragma unroll
        for (int q = 0; q < NR; ++q) atomicAdd(Y + i * NR + q, s[q]);
    }
}

// Y[c][q] += sum over one row range of A[i][c] Q[i][q]: a thread per column.
template <typename TQ, int NR>
__global__ void __launch_bounds__(256) multi_atq_kernel(const double *__restrict__ A, int64_t lda, int64_t m,
                                                        int64_t n, const TQ *__restrict__ Q, double *Y) {
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t ra = m * blockIdx.y / gridDim.y, rb = m * (blockIdx.y + 1) / gridDim.y;
    if (c >= n) return;
    double s[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) s[q] = 0.0;
    for (int64_t i = ra; i < rb; ++i) {
        const double av = __ldg(A + i * lda + c);
#pragma unroll
        for (int q = 0; q < NR; ++q) s[q] = fma(av, ldd(Q + i * NR + q), s[q]);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) atomicAdd(Y + c * NR + q, s[q]);
}

__global__ void multi_norms_kernel(const double *a, const float *b, const double *r, int64_t len, int nr,
                                   double *out) {
    __shared__ double red[2][32];
    const int q = blockIdx.x;
    double e2 = 0.0, r2 = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        const int64_t k = i * nr + q;
        const double rv = r ? r[k] : 0.0;
        const double d = (a ? a[k] : 0.0) + (b ? (double)b[k] : 0.0) - rv;
        e2 += d * d;
        r2 += rv * rv;
    }
    e2 = warp_sum(e2);
    r2 = warp_sum(r2);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][w] = e2;
        red[1][w] = r2;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        e2 = lane < nw ? red[0][lane] : 0.0;
        r2 = lane < nw ? red[1][lane] : 0.0;
        e2 = warp_sum(e2);
        r2 = warp_sum(r2);
        if (lane == 0) {
            out[q] = e2;
            out[nr + q] = r2;
        }
    }
}

__global__ void multi_gather_kernel(const double *src, int64_t ld, int64_t cnt, int64_t len, int nr, double *dst) {
    const int64_t tot = len * nr;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nr, j = e % nr;
        dst[e] = j < cnt ? src[j * ld + i] : 0.0;
    }
}

__global__ void multi_scatter_kernel(const double *src, int64_t cnt, int64_t len, int nr, double *dst, int64_t ld) {
    const int64_t tot = len * cnt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / len, i = e % len;
        dst[j * ld + i] = src[i * nr + j];
    }
}

__global__ void multi_form_kernel(const double *B, const double *Z, const double *Ym, float *F, int64_t mm,
                                  const double *Yn, float *Gv, int64_t nn) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mm + nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < mm) F[e] = (float)(B[e] - Z[e] - Ym[e]);
        else Gv[e - mm] = (float)Yn[e - mm];
    }
}

__global__ void multi_apply_kernel(double *X, const double *Yn, int64_t nn, double *Z, const double *Ym, int64_t mm) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mm + nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nn) X[e] += Yn[e];
        else Z[e - nn] -= Ym[e - nn];
    }
}

unsigned grid_for(int64_t tot) {
    int64_t b = (tot + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

size_t multi_smem_bytes(const MultiArgs &M, int nr) {
    const GridArgs &a = M.geo;
    return multi_smem_layout(a.nrow_cap, a.ncol_cap, a.tau_r, a.tau_c, nr, a.tile_c_bytes, a.tile_r_bytes,
                             M.scr_floats)
        .total;
}

int multi_max_ctas(bool bf16, int nr, bool mma, size_t smem) {
    void *k = multi_kernel(bf16, nr, mma);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kMT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm >= 1 ? sms : 0;
}

cudaError_t launch_multi(const MultiArgs &M, bool bf16, int nr, int G, cudaStream_t st) {
    const size_t smem = multi_smem_bytes(M, nr);
    void *k = multi_kernel(bf16, nr, M.mma != 0);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    MultiArgs copy = M;
    void *params[] = {&copy};
    return cudaLaunchCooperativeKernel(k, dim3(G), dim3(kMT), params, smem, st);
}

cudaError_t multi_ap(const double *A, int64_t lda, int64_t m, int64_t n, int nr, const void *P, bool p_f32,
                     double *Y, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(Y, 0, sizeof(double) * m * nr, st);
    if (e != cudaSuccess || m == 0 || n == 0) return e;
    const int64_t warps = (m + 31) / 32 * ((n + kApSeg - 1) / kApSeg);
    const int64_t blocks = (warps + 7) / 8;
    if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
#define REBK_AP(T, R) \
    multi_ap_kernel<T, R><<<(unsigned)blocks, 256, 0, st>>>(A, lda, m, n, static_cast<const T *>(P), Y)
    if (nr == 8) {
        if (p_f32) REBK_AP(float, 8);
        else REBK_AP(double, 8);
    } else if (nr == 4) {
        if (p_f32) REBK_AP(float, 4);
        else REBK_AP(double, 4);
    } else {
        return cudaErrorInvalidValue;
    }
#undef REBK_AP
    return cudaGetLastError();
}

cudaError_t multi_atq(const double *A, int64_t lda, int64_t m, int64_t n, int nr, const void *Q, bool q_f32,
                      double *Y, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(Y, 0, sizeof(double) * n * nr, st);
    if (e != cudaSuccess || m == 0 || n == 0) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cb = (n + 255) / 256;
    int64_t ranges = (8 * (int64_t)sms + cb - 1) / cb;
    if (ranges > m) ranges = m;
    if (ranges > 65535) ranges = 65535;
    if (ranges < 1) ranges = 1;
    if (cb > 0x7fffffff) return cudaErrorInvalidConfiguration;
    dim3 g((unsigned)cb, (unsigned)ranges);
#define REBK_ATQ(T, R) multi_atq_kernel<T, R><<<g, 256, 0, st>>>(A, lda, m, n, static_cast<const T *>(Q), Y)
    if (nr == 8) {
        if (q_f32) REBK_ATQ(float, 8);
        else REBK_ATQ(double, 8);
    } else if (nr == 4) {
        if (q_f32) REBK_ATQ(float, 4);
        else REBK_ATQ(double, 4);
    } else {
        return cudaErrorInvalidValue;
    }
#undef REBK_ATQ
    return cudaGetLastError();
}

cudaError_t multi_norms(const double *a, const float *b, const double *r, int64_t len, int nr, double *out,
                        cudaStream_t st) {
    multi_norms_kernel<<<nr, 512, 0, st>>>(a, b, r, len, nr, out);
    return cudaGetLastError();
}

cudaError_t multi_gather(const double *src, int64_t ld, int64_t cnt, int64_t len, int nr, double *dst,
                         cudaStream_t st) {
    multi_gather_kernel<<<grid_for(len * nr), 256, 0, st>>>(src, ld, cnt, len, nr, dst);
    return cudaGetLastError();
}

cudaError_t multi_scatter(const double *src, int64_t cnt, int64_t len, int nr, double *dst, int64_t ld,
                          cudaStream_t st) {
    multi_scatter_kernel<<<grid_for(len * cnt), 256, 0, st>>>(src, cnt, len, nr, dst, ld);
    return cudaGetLastError();
}

cudaError_t multi_form(const double *B, const double *Z, const double *Ym, float *F, int64_t m, const double *Yn,
                       float *G, int64_t n, int nr, cudaStream_t st) {
    multi_form_kernel<<<grid_for((m + n) * nr), 256, 0, st>>>(B, Z, Ym, F, m * nr, Yn, G, n * nr);
    return cudaGetLastError();
}

cudaError_t multi_apply(double *X, const double *Yn, int64_t n, double *Z, const double *Ym, int64_t m, int nr,
                        cudaStream_t st) {
    multi_apply_kernel<<<grid_for((m + n) * nr), 256, 0, st>>>(X, Yn, n * nr, Z, Ym, m * nr);
    return cudaGetLastError();
}

}  // namespace rebk
