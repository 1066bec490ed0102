// rebk_umma.cu -- BF16 GEMM on the fifth-generation tensor cores (tcgen05) for
// the warm-start network: C = alpha * A B^T with A (M x K) and B (N x K) both
// K-contiguous ("K-major") BF16, FP32 accumulation in tensor memory.
//
// One CTA computes one 128 x 128 tile of C over a range of K (split-K over
// blockIdx.z).  Warp roles inside the 128-thread CTA:
//   thread 0   TMA producer: 64-wide K slices of A and B (128 B rows, 128-byte
//              swizzle) into a 4-stage shared-memory ring, completion counted
//              on a "full" mbarrier per stage;
//   thread 32  MMA issuer: per stage four tcgen05.mma (M 128, N 128, K 16) into
//              one TMEM accumulator of 128 lanes x 128 FP32 columns, then
//              tcgen05.commit on the stage's "empty" mbarrier (frees the slot)
//              and, after the last slice, on the "done" mbarrier;
//   warp 2     allocates and frees the 128 TMEM columns;
//   all warps  epilogue: warp w reads TMEM lanes 32w..32w+31 (rows of the tile)
//              with tcgen05.ld 32x32b, 32 columns at a time, stages them in
//              shared memory and writes FP32 C, a BF16 copy and a BF16
//              transposed copy (the backward pass needs both layouts as K-major
//              operands) with coalesced accesses, ReLU / a mask applied; under
//              split-K it stores alpha * acc into its slice of a workspace, and a
//              second kernel adds the slices in a fixed order (deterministic).
// Every mbarrier wait is bounded by the global timer; a wait that gives up sets
// the caller's error word, the producer then waits (bounded) for the copies it
// issued, and TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {
namespace {

constexpr int UM_BM = 128, UM_BN = 128, UM_BK = 64, UM_STAGES = 4, UM_THREADS = 128;
constexpr uint32_t UM_TILE_A = UM_BM * UM_BK * 2, UM_TILE_B = UM_BN * UM_BK * 2;  // 16 KB each
constexpr uint32_t UM_STAGE_BYTES = UM_TILE_A + UM_TILE_B;
constexpr uint32_t UM_TMEM_COLS = UM_BN;  // FP32 accumulator columns
constexpr size_t UM_SMEM = 1024 /* alignment slack */ + (size_t)UM_STAGES * UM_STAGE_BYTES + 256;

struct UmmaArgs {
    CUtensorMap ta;  // A: inner dimension K, outer M; box 64 x 128, 128-byte swizzle
    CUtensorMap tb;  // B: inner dimension K, outer N
    int M, N, K;
    int kb_per_split;      // 64-wide K slices per blockIdx.z
    float alpha;
    float *C;              // FP32 output (row-major, ldc) or NULL
    int64_t ldc;
    __nv_bfloat16 *Cb;     // BF16 copy (row-major, ldcb) or NULL
    int64_t ldcb;
    __nv_bfloat16 *CbT;    // BF16 transposed copy: CbT[j * ldcbt + i] or NULL
    int64_t ldcbt;
    int relu;
    const float *mask;     // multiply by (mask[i * ldm + j] > 0) or NULL
    int64_t ldm;
    float *ws;             // split-K: partial tile sums, ws[z][i][j] (M x N each), or NULL
    int *error;            // device word: 1 once a wait gave up
    unsigned long long timeout_ns;
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void um_mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void um_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase of the given parity; false once timeout_ns passed.
__device__ __forceinline__ bool um_wait(uint32_t bar, uint32_t parity, unsigned long long timeout_ns) {
    uint32_t done = 0;
    unsigned long long t0 = 0;
    for (uint32_t spins = 0;; ++spins) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (spins == 0) t0 = globaltimer_ns();
        if ((spins & 63u) == 63u && globaltimer_ns() - t0 > timeout_ns) return false;
    }
}

__device__ __forceinline__ void um_tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 B, 8-row groups 1024 B apart (stride byte
// offset), leading byte offset unused for this layout, descriptor version 1,
// layout type 2 (128-byte swizzle).  The tile base is 1024-byte aligned.
__device__ __forceinline__ uint64_t um_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = UM_BN, M = UM_BM.
constexpr uint32_t kUmmaIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UM_BN >> 3) << 17) |
                                ((uint32_t)(UM_BM >> 4) << 24);

__device__ __forceinline__ void um_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(kUmmaIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void um_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void um_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void um_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of the calling lane's TMEM row.
__device__ __forceinline__ void um_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(UM_THREADS, 1) umma_gemm_kernel(const __grid_constant__ UmmaArgs g) {
    extern __shared__ __align__(1024) unsigned char um_raw[];
    const uint32_t raw = su32(um_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned tiles (128-byte swizzle atoms)
    unsigned char *bp = um_raw + (base - raw);
    const uint32_t bar0 = base + UM_STAGES * UM_STAGE_BYTES;  // full[s], empty[s], done
    auto full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(UM_STAGES + s); };
    const uint32_t done = bar0 + 8u * (uint32_t)(2 * UM_STAGES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bp + UM_STAGES * UM_STAGE_BYTES + 8 * (2 * UM_STAGES + 1));
    int *s_err = reinterpret_cast<int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * UM_BM, n0 = blockIdx.x * UM_BN;
    const int kb_total = (g.K + UM_BK - 1) / UM_BK;
    const int kb0 = blockIdx.z * g.kb_per_split;
    const int kb1 = min(kb0 + g.kb_per_split, kb_total);
    const int nkb = kb1 - kb0;

    if (tid == 0) {
        for (int s = 0; s < UM_STAGES; ++s) {
            um_mbar_init(full(s), 1);
            um_mbar_init(empty(s), 1);
        }
        um_mbar_init(done, 1);
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(UM_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    um_fence_before();
    __syncthreads();
    um_fence_after();
    const uint32_t tmem = *tmem_slot;

    int issued[UM_STAGES];  // producer: copies issued per stage
#pragma unroll
    for (int s = 0; s < UM_STAGES; ++s) issued[s] = 0;
    if (tid == 0) {
        // ---- TMA producer ----
        for (int i = 0; i < nkb; ++i) {
            const int s = i % UM_STAGES;
            if (i >= UM_STAGES && !um_wait(empty(s), (uint32_t)((i / UM_STAGES - 1) & 1), g.timeout_ns)) {
                *s_err = 1;
                break;
            }
            const uint32_t sa = base + (uint32_t)s * UM_STAGE_BYTES, sb = sa + UM_TILE_A;
            um_expect_tx(full(s), UM_STAGE_BYTES);
            um_tma_2d(sa, &g.ta, (kb0 + i) * UM_BK, m0, full(s));
            um_tma_2d(sb, &g.tb, (kb0 + i) * UM_BK, n0, full(s));
            ++issued[s];
        }
    } else if (tid == 32) {
        // ---- MMA issuer ----
        for (int i = 0; i < nkb; ++i) {
            const int s = i % UM_STAGES;
            if (!um_wait(full(s), (uint32_t)((i / UM_STAGES) & 1), g.timeout_ns)) {
                *s_err = 1;
                break;
            }
            um_fence_after();
            const uint32_t sa = base + (uint32_t)s * UM_STAGE_BYTES, sb = sa + UM_TILE_A;
            const uint64_t ad = um_desc(sa), bd = um_desc(sb);
#pragma unroll
            for (int k = 0; k < UM_BK / 16; ++k)  // K = 16 per instruction: 32 bytes along the swizzled row
                um_mma(tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), (i > 0 || k > 0) ? 1u : 0u);
            um_commit(empty(s));
        }
        um_commit(done);  // arrives once every MMA issued above has completed
    }
    // ---- epilogue: every warp, its 32 TMEM lanes ----
    __syncwarp();
    const bool ok_done = um_wait(done, 0u, g.timeout_ns);
    um_fence_after();
    if (!ok_done) *s_err = 1;
    __syncthreads();
    const bool ok = *s_err == 0 && nkb > 0;
    // Each warp stages its 32 rows x 32 columns through shared memory (the
    // pipeline buffers: every copy has landed and every MMA has read them), so
    // that every global access below covers consecutive columns of one row
    // (C, Cb, mask, workspace slice) or consecutive rows of one column (CbT).
    float *stile = reinterpret_cast<float *>(bp) + warp * (32 * 33);
    const int rbase = m0 + warp * 32;
#pragma unroll 1
    for (int c = 0; c < UM_BN; c += 32) {
        float v[32];
        um_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        if (!ok) continue;  // uniform over the CTA
        const int j0 = n0 + c;
        const int jc = j0 + lane;  // this lane's column in the row-wise passes
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            float x = g.alpha * v[e];
            if (!g.ws && g.relu) x = fmaxf(x, 0.f);
            stile[lane * 33 + e] = x;
        }
        __syncwarp();
        if (g.ws) {
            float *slice = g.ws + (int64_t)blockIdx.z * g.M * g.N;
            for (int r = 0; r < 32; ++r) {
                const int i = rbase + r;
                if (i < g.M && jc < g.N) slice[(int64_t)i * g.N + jc] = stile[r * 33 + lane];
            }
            __syncwarp();
            continue;
        }
        if (g.mask) {
            for (int r = 0; r < 32; ++r) {
                const int i = rbase + r;
                if (i < g.M && jc < g.N && !(g.mask[(int64_t)i * g.ldm + jc] > 0.f)) stile[r * 33 + lane] = 0.f;
            }
            __syncwarp();
        }
        for (int r = 0; r < 32; ++r) {
            const int i = rbase + r;
            if (i >= g.M || jc >= g.N) continue;
            const float x = stile[r * 33 + lane];
            if (g.C) g.C[(int64_t)i * g.ldc + jc] = x;
            if (g.Cb) g.Cb[(int64_t)i * g.ldcb + jc] = __float2bfloat16_rn(x);
        }
        if (g.CbT) {
            const int i = rbase + lane;
            for (int e = 0; e < 32; ++e) {
                const int j = j0 + e;
                if (j < g.N && i < g.M) g.CbT[(int64_t)j * g.ldcbt + i] = __float2bfloat16_rn(stile[lane * 33 + e]);
            }
        }
        __syncwarp();
    }
    // no copy may still be landing in shared memory when the CTA leaves
    if (tid == 0 && *s_err != 0) {
        for (int s = 0; s < UM_STAGES; ++s)
            if (issued[s] > 0) um_wait(full(s), (uint32_t)((issued[s] - 1) & 1), g.timeout_ns);
    }
    if (tid == 0 && *s_err != 0) atomicExch(g.error, 1);
    um_fence_before();
    __syncthreads();
    if (warp == 2) {
        um_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UM_TMEM_COLS)
                     : "memory");
    }
}

// Split-K finish: v = sum of the `split` partial slices in slice order (already
// alpha-scaled); ReLU, mask, FP32 and BF16 outputs.
__global__ void umma_finish_kernel(int M, int N, int split, const float *ws, float *C, int64_t ldc,
                                   __nv_bfloat16 *Cb, int64_t ldcb, __nv_bfloat16 *CbT, int64_t ldcbt, int relu,
                                   const float *mask, int64_t ldm) {
    const int64_t MN = (int64_t)M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N, j = e - i * N;
        float x = 0.f;
        for (int z = 0; z < split; ++z) x += ws[z * MN + e];
        if (relu) x = fmaxf(x, 0.f);
        if (mask && !(mask[i * ldm + j] > 0.f)) x = 0.f;
        if (C) C[i * ldc + j] = x;
        const __nv_bfloat16 xb = __float2bfloat16_rn(x);
        if (Cb) Cb[i * ldcb + j] = xb;
        if (CbT) CbT[j * ldcbt + i] = xb;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 um_encode_fn() {
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

// rows x cols (cols contiguous, leading dimension ld) BF16 matrix, box 64 x 128, 128-byte swizzle.
bool um_map(CUtensorMap *map, const __nv_bfloat16 *p, int64_t rows, int64_t cols, int64_t ld) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = um_encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)UM_BK, (cuuint32_t)UM_BM};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(p), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool umma_gemm_supported(int M, int N, int K, const void *A, int64_t lda, const void *B, int64_t ldb) {
    auto al16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    return M > 0 && N > 0 && K > 0 && K % 8 == 0 && lda % 8 == 0 && ldb % 8 == 0 && lda >= K && ldb >= K &&
           al16(A) && al16(B) && um_encode_fn() != nullptr;
}

size_t umma_workspace_floats() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (size_t)sms * UM_BM * UM_BN;  // split x tiles <= SM count
}

cudaError_t umma_gemm(int M, int N, int K, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                      int64_t ldb, float alpha, float *C, int64_t ldc, __nv_bfloat16 *Cb, int64_t ldcb,
                      __nv_bfloat16 *CbT, int64_t ldcbt, int relu, const float *mask, int64_t ldm, float *ws,
                      size_t ws_floats, int *error, cudaStream_t st) {
    UmmaArgs g;
    memset(&g, 0, sizeof(g));
    if (!um_map(&g.ta, A, M, K, lda) || !um_map(&g.tb, B, N, K, ldb)) return cudaErrorInvalidValue;
    g.M = M;
    g.N = N;
    g.K = K;
    g.alpha = alpha;
    g.C = C;
    g.ldc = ldc;
    g.Cb = Cb;
    g.ldcb = ldcb;
    g.CbT = CbT;
    g.ldcbt = ldcbt;
    g.relu = relu;
    g.mask = mask;
    g.ldm = ldm;
    g.error = error;
    g.timeout_ns = 1000000000ull;  // 1 s per wait
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tm = (M + UM_BM - 1) / UM_BM, tn = (N + UM_BN - 1) / UM_BN;
    const int kb = (K + UM_BK - 1) / UM_BK;
    // split K when the tiles alone leave most SMs idle and the workspace holds the slices
    int split = 1;
    if (ws != nullptr && tm * tn < sms / 2) split = std::min(kb, std::max(1, sms / (tm * tn)));
    while (split > 1 && (size_t)split * M * N > ws_floats) --split;
    const int per = (kb + split - 1) / split;
    split = (kb + per - 1) / per;  // no empty split
    g.kb_per_split = per;
    g.ws = split > 1 ? ws : nullptr;
    cudaError_t e = cudaFuncSetAttribute(umma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UM_SMEM);
    if (e != cudaSuccess) return e;
    umma_gemm_kernel<<<dim3(tn, tm, split), UM_THREADS, UM_SMEM, st>>>(g);
    e = cudaGetLastError();
    if (e != cudaSuccess || split == 1) return e;
    const int64_t blocks = ((int64_t)M * N + 255) / 256;
    umma_finish_kernel<<<(unsigned)std::min<int64_t>(blocks, 4096), 256, 0, st>>>(M, N, split, ws, C, ldc, Cb, ldcb,
                                                                                 CbT, ldcbt, relu, mask, ldm);
    return cudaGetLastError();
}

}  // namespace rebk
