// rebk_mlp.cu -- the learned warm start: a small network y = W3 relu(W2 relu(W1 b))
// (output scale s: y = s W3 relu(W2 relu(W1 b))) whose output gives the starting
// point x^0 = A^T y, z^0 = b - A x^0 of REBK.
//
// Theorem main of Du, Si, Sun (arXiv:2001.04179) needs x^0 in range(A^T) and
// z^0 in b + range(A); x^0 = A^T y satisfies the first for any y and z^0 =
// b - A x^0 the second, so the solve still converges to A^+ b while its error
// bound starts from ||x^0 - A^+ b|| and ||z^0 - b_perp|| = ||A (A^+ b - x^0)||,
// both small when the network is good.  The network is trained on
// solver-generated pairs with either the loss mean ||A^T y - A^+ b||^2 or the
// y-space loss mean ||y - y*||^2 / ||y*||^2, y* = (A^T)^+ A^+ b (the minimum-norm
// solution of A^T y = A^+ b, also a solver output).  The y-space loss weighs the
// error of x^0 in the direction of singular value sigma by 1 / sigma^2, the
// directions the iteration converges slowest in; the x-space loss shrinks their
// gradient by sigma^2 instead.
//
// Arithmetic: BF16 operands, FP32 accumulation on the tensor cores, FP32
// master weights and Adam moments.  Every product of the forward and backward
// passes is written C = A B^T with both operands K-contiguous, so that one
// tcgen05 GEMM (rebk_umma.cu: TMA-staged 128-byte-swizzled tiles, TMEM
// accumulator) serves them all; the epilogues and the Adam step keep the
// transposed BF16 copies (activations, output gradients, weights) that the
// next product reads as its K-major operand.  Shapes the TMA tiles cannot
// describe (a K or leading dimension off a 16-byte multiple) run on a small
// mma.sync kernel with strided operands instead.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "rebk.h"
#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;

// C[i, j] = alpha * sum_k A(i, k) B(k, j) (+ beta * C[i, j]), A(i, k) =
// A[i * a_rs + k * a_cs], B(k, j) = B[k * b_rs + j * b_cs]; optional ReLU,
// optional multiply by (mask[i, j] > 0), FP32 output (ldc) and BF16 copy (ldcb).
struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16 *A;
    int64_t a_rs, a_cs;
    const __nv_bfloat16 *B;
    int64_t b_rs, b_cs;
    float *C;
    int64_t ldc;
    __nv_bfloat16 *Cb;
    int64_t ldcb;
    __nv_bfloat16 *CbT;
    int64_t ldcbt;
    float alpha, beta;
    int relu;
    const float *mask;
    int64_t ldm;
};

__device__ __forceinline__ uint32_t pack2(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

__global__ void __launch_bounds__(128) mlp_gemm_kernel(const GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];  // stored [n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // warp tile 32 x 32
    const int gid = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < g.K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 128) {
            const int i = e / BK, k = e % BK;
            const int gi = bm + i, gk = k0 + k;
            As[i][k] = (gi < g.M && gk < g.K) ? g.A[(int64_t)gi * g.a_rs + (int64_t)gk * g.a_cs] : zero;
        }
        for (int e = tid; e < BN * BK; e += 128) {
            const int j = e / BK, k = e % BK;
            const int gj = bn + j, gk = k0 + k;
            Bs[j][k] = (gj < g.N && gk < g.K) ? g.B[(int64_t)gk * g.b_rs + (int64_t)gj * g.b_cs] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int r = wm + a * 16 + gid;
                af[a][0] = pack2(&As[r][kk + tig * 2]);
                af[a][1] = pack2(&As[r + 8][kk + tig * 2]);
                af[a][2] = pack2(&As[r][kk + 8 + tig * 2]);
                af[a][3] = pack2(&As[r + 8][kk + 8 + tig * 2]);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int c = wn + b * 8 + gid;
                bf[b][0] = pack2(&Bs[c][kk + tig * 2]);
                bf[b][1] = pack2(&Bs[c][kk + 8 + tig * 2]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};"
                        : "+f"(acc[a][b][0]), "+f"(acc[a][b][1]), "+f"(acc[a][b][2]), "+f"(acc[a][b][3])
                        : "r"(af[a][0]), "r"(af[a][1]), "r"(af[a][2]), "r"(af[a][3]), "r"(bf[b][0]),
                          "r"(bf[b][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int i = bm + wm + a * 16 + gid + (h >= 2 ? 8 : 0);
                const int j = bn + wn + b * 8 + tig * 2 + (h & 1);
                if (i >= g.M || j >= g.N) continue;
                float v = g.alpha * acc[a][b][h];
                if (g.beta != 0.f) v += g.beta * g.C[(int64_t)i * g.ldc + j];
                if (g.relu) v = fmaxf(v, 0.f);
                if (g.mask && !(g.mask[(int64_t)i * g.ldm + j] > 0.f)) v = 0.f;
                if (g.C) g.C[(int64_t)i * g.ldc + j] = v;
                if (g.Cb) g.Cb[(int64_t)i * g.ldcb + j] = __float2bfloat16_rn(v);
                if (g.CbT) g.CbT[(int64_t)j * g.ldcbt + i] = __float2bfloat16_rn(v);
            }
}

__global__ void f64_to_bf16_kernel(const double *src, __nv_bfloat16 *dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = __float2bfloat16_rn(__double2float_rn(src[e]));
}

__global__ void f32_to_bf16_kernel(const float *src, __nv_bfloat16 *dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = __float2bfloat16_rn(src[e]);
}

// dst[c * ldd + r] = src[r * lds + c] for a rows x cols BF16 matrix, through
// 32 x 32 shared-memory tiles (both sides coalesced).  Block 32 x 8 threads.
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *__restrict__ src, int64_t lds, int64_t rows, int64_t cols,
                                      __nv_bfloat16 *__restrict__ dst, int64_t ldd) {
    __shared__ __nv_bfloat16 t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[k][threadIdx.x] = src[r * lds + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[c * ldd + r] = t[threadIdx.x][k];
    }
}

cudaError_t transpose_bf16(const __nv_bfloat16 *src, int64_t lds, int64_t rows, int64_t cols, __nv_bfloat16 *dst,
                           int64_t ldd, cudaStream_t st) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    transpose_bf16_kernel<<<grid, dim3(32, 8), 0, st>>>(src, lds, rows, cols, dst, ldd);
    return cudaGetLastError();
}

__global__ void f32_to_f64_kernel(const float *src, double *dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (double)src[e];
}

// R = P - X (FP32 P, FP64 X), BF16 copy; out[0] += sum R^2 (atomic).
__global__ void residual_kernel(const float *P, const double *X, float *R, __nv_bfloat16 *Rb, int64_t n,
                                double *loss) {
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float r = (float)((double)P[e] - X[e]);
        R[e] = r;
        Rb[e] = __float2bfloat16_rn(r);
        s += (double)r * r;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

// y-space relative loss, one CTA (256 threads) per batch row b:
// dY[b] = coef (Y[b] - T[b]) / ||T[b]||^2 (0 for a zero target), BF16 copy;
// loss[0] += ||Y[b] - T[b]||^2 / ||T[b]||^2.
__global__ void __launch_bounds__(256) yrel_kernel(const float *Y, const double *T, int64_t m, double coef,
                                                   float *dY, __nv_bfloat16 *dYb, double *loss) {
    __shared__ double red[2][8];
    const int64_t off = (int64_t)blockIdx.x * m;
    double st = 0.0, sd = 0.0;
    for (int64_t e = threadIdx.x; e < m; e += blockDim.x) {
        const double tv = T[off + e], d = (double)Y[off + e] - tv;
        st += tv * tv;
        sd += d * d;
    }
    st = warp_sum(st);
    sd = warp_sum(sd);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = st;
        red[1][threadIdx.x >> 5] = sd;
    }
    __syncthreads();
    double nt = 0.0, nd = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        nt += red[0][w];
        nd += red[1][w];
    }
    const double inv = nt > 0.0 ? 1.0 / nt : 0.0;
    for (int64_t e = threadIdx.x; e < m; e += blockDim.x) {
        const float g = (float)(coef * ((double)Y[off + e] - T[off + e]) * inv);
        dY[off + e] = g;
        dYb[off + e] = __float2bfloat16_rn(g);
    }
    if (threadIdx.x == 0) atomicAdd(loss, nd * inv);
}

// Adam on FP32 master weights; refreshes the BF16 copy (the transpose follows
// by transpose_bf16).
__global__ void adam_kernel(float *w, const float *grad, float *m1, float *m2, __nv_bfloat16 *wb, int64_t n,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float gv = grad[e];
        const float a = b1 * m1[e] + (1.f - b1) * gv, b = b2 * m2[e] + (1.f - b2) * gv * gv;
        m1[e] = a;
        m2[e] = b;
        const float v = w[e] - lr * (a / c1) / (sqrtf(b / c2) + eps);
        w[e] = v;
        wb[e] = __float2bfloat16_rn(v);
    }
}

int eblocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t gemm(const GemmArgs &g, cudaStream_t st) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
    mlp_gemm_kernel<<<grid, 128, 0, st>>>(g);
    return cudaGetLastError();
}

GemmArgs gemm_args(int M, int N, int K, const __nv_bfloat16 *A, int64_t a_rs, int64_t a_cs,
                   const __nv_bfloat16 *B, int64_t b_rs, int64_t b_cs, float *C, int64_t ldc,
                   __nv_bfloat16 *Cb, int64_t ldcb) {
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.a_rs = a_rs; g.a_cs = a_cs;
    g.B = B; g.b_rs = b_rs; g.b_cs = b_cs;
    g.C = C; g.ldc = ldc; g.Cb = Cb; g.ldcb = ldcb;
    g.alpha = 1.f;
    return g;
}

}  // namespace
}  // namespace rebk

using namespace rebk;

struct rebk_mlp_s {
    cudaStream_t stream = nullptr;
    int64_t m = 0, n = 0, hidden = 0, cap = 0;  // input / output size m, A columns n, batch capacity
    // weights: W1 (hidden x m), W2 (hidden x hidden), W3 (m x hidden)
    float *w[3] = {nullptr, nullptr, nullptr}, *g[3] = {nullptr, nullptr, nullptr};
    float *m1[3] = {nullptr, nullptr, nullptr}, *m2[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16 *wb[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16 *wbT[3] = {nullptr, nullptr, nullptr};  // transposed BF16 copies
    int64_t wsize[3] = {0, 0, 0}, wrows[3] = {0, 0, 0}, wcols[3] = {0, 0, 0};
    __nv_bfloat16 *Ab = nullptr;   // BF16 copy of A (m x n, row-major, ld n)
    __nv_bfloat16 *AbT = nullptr;  // its transpose (n x m)
    // transposed BF16 activations and gradients (feature x capacity): the K-major
    // operands of the weight-gradient products
    __nv_bfloat16 *XbT = nullptr, *H1T = nullptr, *H2T = nullptr, *dYT = nullptr, *dH2T = nullptr,
                  *dH1T = nullptr;
    int *gemm_err = nullptr;       // device word set by a tensor-core GEMM whose wait gave up
    float *gemm_ws = nullptr;      // split-K partial sums of the tensor-core GEMM
    size_t gemm_ws_floats = 0;
    int64_t umma_calls = 0, legacy_calls = 0;
    // activations (cap rows)
    __nv_bfloat16 *Xb = nullptr, *H1b = nullptr, *H2b = nullptr, *Yb = nullptr, *Rb = nullptr, *dYb = nullptr,
                  *dH2b = nullptr, *dH1b = nullptr;
    float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *P = nullptr, *R = nullptr, *dY = nullptr, *dH2 = nullptr,
          *dH1 = nullptr;
    double *loss = nullptr;
    int64_t step = 0;
    int32_t loss_kind = REBK_MLP_LOSS_X;
    float out_scale = 1.f;  // y = out_scale * W3 relu(W2 relu(W1 b))
};

namespace rebk {
int64_t mlp_batch_capacity(::rebk_mlp_s *h) { return h ? h->cap : 0; }
}  // namespace rebk

namespace {

rebk_status mfail(rebk_status s, const std::string &msg) {
    set_last_error(msg);
    return s;
}

#define MCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess) return mfail(e__ == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA, \
                                             std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

void free_mlp(rebk_mlp h) {
    if (!h) return;
    for (int l = 0; l < 3; ++l) {
        void *p[] = {h->w[l], h->g[l], h->m1[l], h->m2[l], h->wb[l], h->wbT[l]};
        for (void *q : p)
            if (q) cudaFree(q);
    }
    void *p[] = {h->Ab, h->AbT, h->Xb, h->H1b, h->H2b, h->Yb, h->Rb, h->dYb, h->dH2b, h->dH1b, h->H1, h->H2, h->Y,
                 h->P, h->R, h->dY, h->dH2, h->dH1, h->loss, h->XbT, h->H1T, h->H2T, h->dYT, h->dH2T, h->dH1T,
                 h->gemm_err, h->gemm_ws};
    for (void *q : p)
        if (q) cudaFree(q);
    delete h;
}

// C (M x N) = alpha * sum_k A[i * lda + k] B[j * ldb + k] (both operands
// K-contiguous), epilogue as umma_gemm: the tensor-core GEMM when the TMA tiles
// can describe the operands, else the mma.sync kernel with the same strides.
rebk_status mm(rebk_mlp h, int64_t M, int64_t N, int64_t K, const __nv_bfloat16 *A, int64_t lda,
               const __nv_bfloat16 *B, int64_t ldb, float alpha, float *C, int64_t ldc, __nv_bfloat16 *Cb,
               int64_t ldcb, __nv_bfloat16 *CbT, int64_t ldcbt, int relu = 0, const float *mask = nullptr,
               int64_t ldm = 0) {
    const cudaStream_t st = h->stream;
    if (umma_gemm_supported((int)M, (int)N, (int)K, A, lda, B, ldb) && (C != nullptr || Cb != nullptr)) {
        ++h->umma_calls;
        MCK(umma_gemm((int)M, (int)N, (int)K, A, lda, B, ldb, alpha, C, ldc, Cb, ldcb, CbT, ldcbt, relu, mask, ldm,
                      h->gemm_ws, h->gemm_ws_floats, h->gemm_err, st));
        return REBK_OK;
    }
    ++h->legacy_calls;
    GemmArgs g = gemm_args((int)M, (int)N, (int)K, A, lda, 1, B, 1, ldb, C, ldc, Cb, ldcb);
    g.CbT = CbT;
    g.ldcbt = ldcbt;
    g.alpha = alpha;
    g.relu = relu;
    g.mask = mask;
    g.ldm = ldm;
    MCK(gemm(g, st));
    return REBK_OK;
}

// Forward pass for `batch` inputs (rows of Xb, columns of XbT): H1, H2 (FP32,
// BF16 and transposed BF16), Y (FP32 + BF16).
rebk_status forward(rebk_mlp h, int64_t batch) {
    const int64_t m = h->m, H = h->hidden, cap = h->cap;
    rebk_status s = mm(h, batch, H, m, h->Xb, m, h->wb[0], m, 1.f, h->H1, H, h->H1b, H, h->H1T, cap, 1);
    if (s == REBK_OK) s = mm(h, batch, H, H, h->H1b, H, h->wb[1], H, 1.f, h->H2, H, h->H2b, H, h->H2T, cap, 1);
    if (s == REBK_OK) s = mm(h, batch, m, H, h->H2b, H, h->wb[2], H, h->out_scale, h->Y, m, h->Yb, m, nullptr, 0);
    return s;
}

// Reads and clears the tensor-core GEMM's error word (after a stream sync).
rebk_status gemm_status(rebk_mlp h) {
    int e = 0;
    MCK(cudaMemcpy(&e, h->gemm_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        MCK(cudaMemset(h->gemm_err, 0, sizeof(int)));
        return mfail(REBK_ECUDA, "tensor-core GEMM: a bounded wait gave up");
    }
    return REBK_OK;
}

rebk_status check_batch(rebk_mlp h, int64_t batch) {
    if (batch < 1 || batch > h->cap) return mfail(REBK_EINVAL, "batch must be 1..capacity");
    return REBK_OK;
}

}  // namespace

extern "C" {

rebk_status rebk_mlp_create(rebk_mlp *out, const double *A, int64_t m, int64_t n, int A_on_device,
                            int64_t hidden, int64_t batch_capacity, const float *const *init_weights,
                            uint64_t seed, void *stream) {
    set_last_error("");
    if (!out) return mfail(REBK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!A || m < 1 || n < 1 || hidden < 1 || batch_capacity < 1)
        return mfail(REBK_EINVAL, "A, m, n, hidden, batch_capacity required");
    rebk_mlp h = new rebk_mlp_s();
    h->stream = static_cast<cudaStream_t>(stream);
    h->m = m;
    h->n = n;
    h->hidden = hidden;
    h->cap = batch_capacity;
    h->wsize[0] = hidden * m;
    h->wsize[1] = hidden * hidden;
    h->wsize[2] = m * hidden;
    h->wrows[0] = hidden; h->wcols[0] = m;
    h->wrows[1] = hidden; h->wcols[1] = hidden;
    h->wrows[2] = m;      h->wcols[2] = hidden;
    const cudaStream_t st = h->stream;
    auto fin = [&](rebk_status s) {
        if (s != REBK_OK) free_mlp(h);
        return s;
    };
#define MCKH(call)                                                                                 \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess)                                                                    \
            return fin(mfail(e__ == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA,          \
                             std::string(#call) + ": " + cudaGetErrorString(e__)));                \
    } while (0)
    const int64_t fan_in[3] = {m, hidden, hidden};
    for (int l = 0; l < 3; ++l) {
        const int64_t sz = h->wsize[l];
        MCKH(cudaMalloc(&h->w[l], sizeof(float) * sz));
        MCKH(cudaMalloc(&h->g[l], sizeof(float) * sz));
        MCKH(cudaMalloc(&h->m1[l], sizeof(float) * sz));
        MCKH(cudaMalloc(&h->m2[l], sizeof(float) * sz));
        MCKH(cudaMalloc(&h->wb[l], sizeof(__nv_bfloat16) * sz));
        MCKH(cudaMalloc(&h->wbT[l], sizeof(__nv_bfloat16) * sz));
        MCKH(cudaMemsetAsync(h->m1[l], 0, sizeof(float) * sz, st));
        MCKH(cudaMemsetAsync(h->m2[l], 0, sizeof(float) * sz, st));
        if (init_weights && init_weights[l]) {
            MCKH(cudaMemcpyAsync(h->w[l], init_weights[l], sizeof(float) * sz, cudaMemcpyHostToDevice, st));
        } else {
            // He initialisation N(0, 2 / fan_in), drawn on the host from a fixed seed
            std::vector<float> hw(sz);
            uint64_t sstate = seed * 0x9E3779B97F4A7C15ull + (uint64_t)l + 1;
            auto next = [&]() {  // splitmix64
                uint64_t z = (sstate += 0x9E3779B97F4A7C15ull);
                z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                return z ^ (z >> 31);
            };
            const double sd = std::sqrt(2.0 / (double)fan_in[l]);
            for (int64_t e = 0; e < sz; e += 2) {
                const double u1 = ((next() >> 11) + 1.0) * 0x1.0p-53, u2 = (next() >> 11) * 0x1.0p-53;
                const double r = std::sqrt(-2.0 * std::log(u1));
                hw[e] = (float)(sd * r * std::cos(2 * M_PI * u2));
                if (e + 1 < sz) hw[e + 1] = (float)(sd * r * std::sin(2 * M_PI * u2));
            }
            MCKH(cudaMemcpyAsync(h->w[l], hw.data(), sizeof(float) * sz, cudaMemcpyHostToDevice, st));
            MCKH(cudaStreamSynchronize(st));
        }
        f32_to_bf16_kernel<<<eblocks(sz), 256, 0, st>>>(h->w[l], h->wb[l], sz);
        MCKH(cudaGetLastError());
        MCKH(transpose_bf16(h->wb[l], h->wcols[l], h->wrows[l], h->wcols[l], h->wbT[l], h->wrows[l], st));
    }
    // BF16 copy of A (m x n) for the loss-gradient products
    double *Ad = nullptr;
    if (!A_on_device) {
        MCKH(cudaMalloc(&Ad, sizeof(double) * m * n));
        MCKH(cudaMemcpyAsync(Ad, A, sizeof(double) * m * n, cudaMemcpyHostToDevice, st));
    }
    MCKH(cudaMalloc(&h->Ab, sizeof(__nv_bfloat16) * m * n));
    MCKH(cudaMalloc(&h->AbT, sizeof(__nv_bfloat16) * m * n));
    f64_to_bf16_kernel<<<eblocks(m * n), 256, 0, st>>>(A_on_device ? A : Ad, h->Ab, m * n);
    MCKH(cudaGetLastError());
    MCKH(transpose_bf16(h->Ab, n, m, n, h->AbT, m, st));
    MCKH(cudaGetLastError());
    MCKH(cudaStreamSynchronize(st));
    if (Ad) cudaFree(Ad);
    const int64_t C = batch_capacity;
    MCKH(cudaMalloc(&h->Xb, sizeof(__nv_bfloat16) * C * m));
    MCKH(cudaMalloc(&h->H1b, sizeof(__nv_bfloat16) * C * hidden));
    MCKH(cudaMalloc(&h->H2b, sizeof(__nv_bfloat16) * C * hidden));
    MCKH(cudaMalloc(&h->Yb, sizeof(__nv_bfloat16) * C * m));
    MCKH(cudaMalloc(&h->Rb, sizeof(__nv_bfloat16) * C * n));
    MCKH(cudaMalloc(&h->dYb, sizeof(__nv_bfloat16) * C * m));
    MCKH(cudaMalloc(&h->dH2b, sizeof(__nv_bfloat16) * C * hidden));
    MCKH(cudaMalloc(&h->dH1b, sizeof(__nv_bfloat16) * C * hidden));
    MCKH(cudaMalloc(&h->H1, sizeof(float) * C * hidden));
    MCKH(cudaMalloc(&h->H2, sizeof(float) * C * hidden));
    MCKH(cudaMalloc(&h->Y, sizeof(float) * C * m));
    MCKH(cudaMalloc(&h->P, sizeof(float) * C * n));
    MCKH(cudaMalloc(&h->R, sizeof(float) * C * n));
    MCKH(cudaMalloc(&h->dY, sizeof(float) * C * m));
    MCKH(cudaMalloc(&h->dH2, sizeof(float) * C * hidden));
    MCKH(cudaMalloc(&h->dH1, sizeof(float) * C * hidden));
    MCKH(cudaMalloc(&h->loss, sizeof(double)));
    MCKH(cudaMalloc(&h->XbT, sizeof(__nv_bfloat16) * C * m));
    MCKH(cudaMalloc(&h->H1T, sizeof(__nv_bfloat16) * C * hidden));
    MCKH(cudaMalloc(&h->H2T, sizeof(__nv_bfloat16) * C * hidden));
    MCKH(cudaMalloc(&h->dYT, sizeof(__nv_bfloat16) * C * m));
    MCKH(cudaMalloc(&h->dH2T, sizeof(__nv_bfloat16) * C * hidden));
    MCKH(cudaMalloc(&h->dH1T, sizeof(__nv_bfloat16) * C * hidden));
    MCKH(cudaMalloc(&h->gemm_err, sizeof(int)));
    MCKH(cudaMemset(h->gemm_err, 0, sizeof(int)));
    h->gemm_ws_floats = umma_workspace_floats();
    MCKH(cudaMalloc(&h->gemm_ws, sizeof(float) * h->gemm_ws_floats));
#undef MCKH
    *out = h;
    return REBK_OK;
}

void rebk_mlp_destroy(rebk_mlp h) { free_mlp(h); }

rebk_status rebk_mlp_forward(rebk_mlp h, const double *Bm, int64_t batch, double *Y) {
    if (!h || !Bm || !Y) return mfail(REBK_EINVAL, "NULL argument");
    rebk_status s = check_batch(h, batch);
    if (s != REBK_OK) return s;
    const cudaStream_t st = h->stream;
    f64_to_bf16_kernel<<<eblocks(batch * h->m), 256, 0, st>>>(Bm, h->Xb, batch * h->m);
    MCK(cudaGetLastError());
    s = forward(h, batch);
    if (s != REBK_OK) return s;
    f32_to_f64_kernel<<<eblocks(batch * h->m), 256, 0, st>>>(h->Y, Y, batch * h->m);
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(st));
    return gemm_status(h);
}

rebk_status rebk_mlp_gradients(rebk_mlp h, const double *Bm, const double *Xls, int64_t batch, double *loss,
                               float *const *grads_host) {
    if (!h || !Bm || !Xls) return mfail(REBK_EINVAL, "NULL argument");
    rebk_status s = check_batch(h, batch);
    if (s != REBK_OK) return s;
    const cudaStream_t st = h->stream;
    const int64_t m = h->m, n = h->n, H = h->hidden, cap = h->cap;
    f64_to_bf16_kernel<<<eblocks(batch * m), 256, 0, st>>>(Bm, h->Xb, batch * m);
    MCK(cudaGetLastError());
    MCK(transpose_bf16(h->Xb, m, batch, m, h->XbT, cap, st));
    s = forward(h, batch);
    if (s != REBK_OK) return s;
    MCK(cudaMemsetAsync(h->loss, 0, sizeof(double), st));
    // dY: gradient w.r.t. the last layer's unscaled output (the loss gradient in y times out_scale)
    if (h->loss_kind == REBK_MLP_LOSS_X) {
        // P = Y A (batch x n): A^T y for every sample; R = P - X_ls
        s = mm(h, batch, n, m, h->Yb, m, h->AbT, m, 1.f, h->P, n, nullptr, 0, nullptr, 0);
        if (s != REBK_OK) return s;
        residual_kernel<<<eblocks(batch * n), 256, 0, st>>>(h->P, Xls, h->R, h->Rb, batch * n, h->loss);
        MCK(cudaGetLastError());
        // dY = (2 s / batch) R A^T (batch x m)
        s = mm(h, batch, m, n, h->Rb, n, h->Ab, n, 2.f * h->out_scale / (float)batch, h->dY, m, h->dYb, m, h->dYT,
               cap);
        if (s != REBK_OK) return s;
    } else {
        // dY = (2 s / batch) (Y - Y*) / ||Y*||^2 per row
        yrel_kernel<<<(unsigned)batch, 256, 0, st>>>(h->Y, Xls, m, 2.0 * h->out_scale / (double)batch, h->dY,
                                                     h->dYb, h->loss);
        MCK(cudaGetLastError());
        MCK(transpose_bf16(h->dYb, m, batch, m, h->dYT, cap, st));
    }
    // dW3 = dY^T H2 (m x H)
    s = mm(h, m, H, batch, h->dYT, cap, h->H2T, cap, 1.f, h->g[2], H, nullptr, 0, nullptr, 0);
    // dH2 = (dY W3) * [H2 > 0]
    if (s == REBK_OK)
        s = mm(h, batch, H, m, h->dYb, m, h->wbT[2], m, 1.f, h->dH2, H, h->dH2b, H, h->dH2T, cap, 0, h->H2, H);
    // dW2 = dH2^T H1 (H x H)
    if (s == REBK_OK) s = mm(h, H, H, batch, h->dH2T, cap, h->H1T, cap, 1.f, h->g[1], H, nullptr, 0, nullptr, 0);
    // dH1 = (dH2 W2) * [H1 > 0]
    if (s == REBK_OK)
        s = mm(h, batch, H, H, h->dH2b, H, h->wbT[1], H, 1.f, h->dH1, H, h->dH1b, H, h->dH1T, cap, 0, h->H1, H);
    // dW1 = dH1^T X (H x m)
    if (s == REBK_OK) s = mm(h, H, m, batch, h->dH1T, cap, h->XbT, cap, 1.f, h->g[0], m, nullptr, 0, nullptr, 0);
    if (s != REBK_OK) return s;
    double lsum = 0.0;
    MCK(cudaMemcpyAsync(&lsum, h->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    s = gemm_status(h);
    if (s != REBK_OK) return s;
    if (loss) *loss = lsum / (double)batch;
    if (grads_host)
        for (int l = 0; l < 3; ++l)
            if (grads_host[l]) MCK(cudaMemcpy(grads_host[l], h->g[l], sizeof(float) * h->wsize[l], cudaMemcpyDeviceToHost));
    return REBK_OK;
}

rebk_status rebk_mlp_train_step(rebk_mlp h, const double *Bm, const double *Xls, int64_t batch, double lr,
                                double *loss) {
    rebk_status s = rebk_mlp_gradients(h, Bm, Xls, batch, loss, nullptr);
    if (s != REBK_OK) return s;
    const cudaStream_t st = h->stream;
    ++h->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)h->step), c2 = 1.f - std::pow(b2, (float)h->step);
    for (int l = 0; l < 3; ++l) {
        adam_kernel<<<eblocks(h->wsize[l]), 256, 0, st>>>(h->w[l], h->g[l], h->m1[l], h->m2[l], h->wb[l], h->wsize[l],
                                                          (float)lr, b1, b2, 1e-8f, c1, c2);
        MCK(cudaGetLastError());
        MCK(transpose_bf16(h->wb[l], h->wcols[l], h->wrows[l], h->wcols[l], h->wbT[l], h->wrows[l], st));
    }
    MCK(cudaStreamSynchronize(st));
    return REBK_OK;
}

rebk_status rebk_mlp_set_loss(rebk_mlp h, int32_t loss, double out_scale) {
    if (!h) return mfail(REBK_EINVAL, "NULL network");
    if (loss != REBK_MLP_LOSS_X && loss != REBK_MLP_LOSS_Y_REL) return mfail(REBK_EINVAL, "unknown loss");
    if (!(out_scale > 0.0) || !std::isfinite(out_scale)) return mfail(REBK_EINVAL, "out_scale must be > 0");
    h->loss_kind = loss;
    h->out_scale = (float)out_scale;
    return REBK_OK;
}

rebk_status rebk_mlp_shape(rebk_mlp h, int64_t *m, int64_t *n) {
    if (!h) return mfail(REBK_EINVAL, "NULL network");
    if (m) *m = h->m;
    if (n) *n = h->n;
    return REBK_OK;
}

rebk_status rebk_mlp_get_weights(rebk_mlp h, float *const *weights_host) {
    if (!h || !weights_host) return mfail(REBK_EINVAL, "NULL argument");
    for (int l = 0; l < 3; ++l)
        if (weights_host[l]) MCK(cudaMemcpy(weights_host[l], h->w[l], sizeof(float) * h->wsize[l], cudaMemcpyDeviceToHost));
    return REBK_OK;
}

rebk_status rebk_gemm_bf16(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B, int64_t ldb,
                           float alpha, float *C, int64_t ldc, void *stream, int32_t *path) {
    set_last_error("");
    if (!A || !B || !C) return mfail(REBK_EINVAL, "A, B and C must be device pointers");
    if (M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N) return mfail(REBK_EINVAL, "bad shape");
    if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return mfail(REBK_EUNSUPPORTED, "dimension above 2^31");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const __nv_bfloat16 *a = static_cast<const __nv_bfloat16 *>(A), *b = static_cast<const __nv_bfloat16 *>(B);
    const bool tc = umma_gemm_supported((int)M, (int)N, (int)K, A, lda, B, ldb);
    if (path) *path = tc ? 1 : 0;
    if (tc) {
        int *err = nullptr;
        float *ws = nullptr;
        const size_t wsf = umma_workspace_floats();
        MCK(cudaMalloc(&err, sizeof(int)));
        cudaError_t e = cudaMalloc(&ws, sizeof(float) * wsf);
        if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
        if (e == cudaSuccess)
            e = umma_gemm((int)M, (int)N, (int)K, a, lda, b, ldb, alpha, C, ldc, nullptr, 0, nullptr, 0, 0, nullptr, 0,
                          ws, wsf, err, st);
        int herr = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(err);
        if (ws) cudaFree(ws);
        MCK(e);
        if (herr) return mfail(REBK_ECUDA, "tensor-core GEMM: a bounded wait gave up");
        return REBK_OK;
    }
    GemmArgs g = gemm_args((int)M, (int)N, (int)K, a, lda, 1, b, 1, ldb, C, ldc, nullptr, 0);
    g.alpha = alpha;
    MCK(gemm(g, st));
    MCK(cudaStreamSynchronize(st));
    return REBK_OK;
}

}  // extern "C"
