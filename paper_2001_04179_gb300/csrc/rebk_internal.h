// rebk_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

struct rebk_mlp_s;  // the warm-start network (rebk_mlp.cu)

namespace rebk {

constexpr int kThreads = 512;              // threads per CTA of the persistent kernel
constexpr int kWarps = kThreads / 32;
constexpr int kZWarps = 4;                 // warps of the column-step (z) chain
constexpr int kXWarps = kWarps - kZWarps;  // warps of the row-step (x) chain
constexpr int kZThreads = kZWarps * 32, kXThreads = kXWarps * 32;
constexpr int kZRing = 4;                  // z_I hand-over slots between the two chains
constexpr int kRing = 8;                   // block indices kept ahead / behind
constexpr size_t kSmemHeader = 512;        // index rings, flags, mbarriers, step coefficients
constexpr int kAccReplicas = 16;           // replicated accumulators (atomic contention)
constexpr int kAccReplicasF64 = 2;         // plain FP64: each CTA adds the replicas of every
                                           // entry in FP64, on the slow FP64 pipe
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s per wait
constexpr int64_t kMaxItersPerLaunch = 8000000;                 // barrier counter headroom

// Arguments of the persistent REBK kernel (Algorithm 1 on one system).
//
// State arrays z (length m) and x (length n) have the kernel's arithmetic type
// TS.  In the plain form (CORR = false) they are z and x of Algorithm 1,
// beta = b and gamma = NULL.  In the correction form (CORR = true) they are
// the corrections dz, dx, beta = f = b - z - A x, gamma = g = A^T z, and the
// duals s (length n) and v (length m) are accumulated (see rebk.h).
struct GridArgs {
    CUtensorMap tmap_c;     // TMA: column tiles (own rows x tau_c box)
    CUtensorMap tmap_r;     // TMA: row tiles (tau_r x own columns box)
    const void *A;          // stored copy, row-major, leading dimension lda (zero padded)
    int64_t lda, m, n;
    int tau_r, tau_c, s, t; // largest block sizes and block counts
    const int64_t *row_off; // device, s + 1 row-block offsets; NULL = blocks of tau_r rows
    const int64_t *col_off; // device, t + 1 column-block offsets; NULL = blocks of tau_c columns
    int col_align;          // with col_off: largest power of two (<= 16) dividing every column-block start
    const double *cdf_r, *cdf_c, *nr, *nc;
    const void *coef_r, *coef_c;  // TS: alpha / ||block||_F^2 (0 for blocks of zero norm)
    int fb_r, fb_c;         // fallback picks (last block of nonzero norm)
    double alpha;
    uint64_t seed, stream;
    int64_t k0, iters;      // iterations k0+1 .. k0+iters
    void *z, *x;            // TS, length m / n
    const double *beta;     // length m
    const double *gamma;    // length n (CORR) or NULL
    void *sdual, *vdual;    // TS, length n / m (CORR)
    const double *x_ref;    // NULL = no error test
    const double *x_base;   // CORR: the test uses x_base + x
    double tol2_abs;        // stop once ||(x_base +) x - x_ref||^2 <= tol2_abs
    int64_t check_every;    // test x^k when (check_offset + k) % check_every == 0
    int64_t check_offset;
    const int32_t *idx;     // 2 * iters entries: (j_k, i_k), from sample_blocks()
    void *acc;              // TS [2 chains][3 sets][acc_r][acc_w], zeroed before launch
    int acc_w, acc_r;
    int nrow_cap, ncol_cap; // shared-memory capacity for the owned slices
    int use_tma;            // tiles staged in shared memory by TMA
    int tma_vx;             // elements per 16 bytes
    int bw_c, bh_c, nbox_c; // column-tile box (width, height) and boxes per tile
    int bw_r;               // row-tile box width (height tau_r)
    int64_t tile_c_bytes, tile_r_bytes;        // shared-memory size of a tile (128-aligned)
    int64_t tile_c_bytes_tx, tile_r_bytes_tx;  // bytes a tile's copies deliver
    unsigned int *bar;      // barrier counter of the column-step chain, zeroed before launch
    unsigned int *bar_x;    // barrier counter of the row-step chain, zeroed before launch
    int *status;            // zeroed before launch
    int64_t *iters_done;
    unsigned long long timeout_ns;
};

enum class Mode { PlainF64, CorrF32, CorrBF16 };

inline int acc_replicas(Mode m) { return m == Mode::PlainF64 ? kAccReplicasF64 : kAccReplicas; }

// Shared-memory layout of the persistent kernel (byte offsets, 16-byte aligned).
struct SmemLayout {
    size_t zeta, beta, v, xi, s, w, r, zr, redz, redx, tc0, tc1, tr0, tr1, total;
};

__host__ __device__ inline SmemLayout smem_layout(int nrow_cap, int ncol_cap, int tau_r, int tau_c,
                                                  bool corr, int ts, int vec, int64_t tile_c_bytes,
                                                  int64_t tile_r_bytes) {
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    auto al128 = [](size_t x) { return (x + 127) & ~(size_t)127; };
    SmemLayout L;
    size_t o = kSmemHeader;
    L.tc0 = o; o = al128(o + (size_t)tile_c_bytes);
    L.tc1 = o; o = al128(o + (size_t)tile_c_bytes);
    L.tr0 = o; o = al128(o + (size_t)tile_r_bytes);
    L.tr1 = o; o = al128(o + (size_t)tile_r_bytes);
    L.zeta = o; o = al(o + (size_t)nrow_cap * ts);
    L.beta = o; o = al(o + (size_t)nrow_cap * ts);
    L.v = o;    if (corr) o = al(o + (size_t)nrow_cap * ts);
    // x and w are read over whole tile rows: room for the zero padding up to a multiple of 8
    L.xi = o;   o = al(o + (size_t)((ncol_cap + 7) / 8 * 8) * ts);
    L.s = o;    if (corr) o = al(o + (size_t)ncol_cap * ts);
    L.w = o;    o = al(o + (size_t)((tau_c + 7) / 8 * 8) * ts);
    L.r = o;    o = al(o + (size_t)tau_r * ts);
    L.zr = o;   o = al(o + (size_t)kZRing * tau_r * ts);
    size_t rz = (size_t)kZThreads * vec * ts, rx = (size_t)kXThreads * vec * ts;
    if (rz < (size_t)kZWarps * 8) rz = (size_t)kZWarps * 8;
    if (rx < (size_t)kXWarps * 8) rx = (size_t)kXWarps * 8;
    L.redz = o; o = al(o + rz);
    L.redx = o; o = al(o + rx);
    L.total = o;
    return L;
}

// Owned row / column slices of CTA c of G (rows [r0, r1), columns [c0, c1);
// column slices are aligned to 8 elements so every 16-byte vector load of a
// slice starts inside it or in the zero padding).
inline void host_slices(int64_t m, int64_t n, int G, int c, int64_t *r0, int64_t *r1,
                        int64_t *c0, int64_t *c1) {
    const int64_t nu = (n + 7) / 8;
    *r0 = m * c / G;
    *r1 = m * (c + 1) / G;
    int64_t a = 8 * (nu * c / G), b = 8 * (nu * (c + 1) / G);
    *c0 = a < n ? a : n;
    *c1 = b < n ? b : n;
}

size_t grid_smem_bytes(Mode mode, const GridArgs &a);
int storage_size(Mode mode);
bool tma_geometry(Mode mode, GridArgs &a);
cudaError_t tma_encode(Mode mode, GridArgs &a);
cudaError_t step_coefficients(const double *norms, int nb, double alpha, double *c64, float *c32,
                              cudaStream_t st);
// idx[2(k-1)] = j_k, idx[2(k-1)+1] = i_k for k = 1..K (draws of iterations k0+1..k0+K).
cudaError_t sample_blocks(uint64_t seed, uint64_t stream, int64_t k0, int64_t K, const double *cdf_r,
                          int s, const double *cdf_c, int t, int fb_r, int fb_c, int32_t *idx,
                          cudaStream_t st);
cudaError_t launch_grid(Mode mode, const GridArgs &a, int G, cudaStream_t st);
int grid_max_ctas(Mode mode, size_t smem);

// Setup and sweep kernels (rebk_setup.cu).
cudaError_t convert_storage(const double *src, int64_t lds, void *dst, int64_t ldd, int64_t m,
                            int64_t n, int storage, cudaStream_t st);
// Block norms, prefix sums and fallback picks.  row_off / col_off: device offset
// arrays of the partitions (s + 1, t + 1 entries), or NULL for blocks of tau_r / tau_c.
cudaError_t block_tables(const double *A, int64_t lda, int64_t m, int64_t n, int tau_r, int tau_c,
                         int s, int t, double *nr, double *nc, double *cdf_r, double *cdf_c,
                         int *fallback /* device int[2] */, double *scratch /* m + n + 64*n */,
                         cudaStream_t st, const int64_t *row_off = nullptr, const int64_t *col_off = nullptr);
// y_m = A p (length m), y_n = A^T q (length n); p or q may be NULL (skipped).
// TP/TQ: double or float inputs.
cudaError_t dual_sweep(const double *A, int64_t lda, int64_t m, int64_t n, const void *p,
                       bool p_f32, const void *q, bool q_f32, double *ym, double *yn,
                       cudaStream_t st);
// tau_r / tau_c: the largest block sizes; row_off / col_off as for block_tables.
cudaError_t beta_max_device(const double *A, int64_t lda, int64_t m, int64_t n, int tau_r, int tau_c,
                            int s, int t, const double *nr, const double *nc, double *gram_scratch,
                            double *beta_rows, double *beta_cols, cudaStream_t st,
                            const int64_t *row_off = nullptr, const int64_t *col_off = nullptr);
// out[0] = sum (a + x - r)^2 over n (a may be NULL), out[1] = sum r^2.
cudaError_t err_norms(const double *a, const double *x, const double *r, int64_t n, double *out,
                      cudaStream_t st);
// Grouped right-hand-side layout (right-hand side j = column j % g of block j / g,
// each block len x g row-major): gather cnt of them from j0 into rows of len;
// store x (n) and b - ax (m) of right-hand side j.
cudaError_t group_gather(const double *src, int64_t j0, int64_t cnt, int g, int64_t len, double *dst,
                         cudaStream_t st);
cudaError_t group_store_xz(const double *x, int64_t n, const double *b, const double *ax, int64_t m, int64_t j, int g,
                           double *X0, double *Z0, cudaStream_t st);
// C (M x N, ldc) = sum_k A[i a_rs + k a_cs] B[k b_rs + j b_cs] in FP64.
cudaError_t dgemm(int M, int N, int K, const double *A, int64_t a_rs, int64_t a_cs, const double *B, int64_t b_rs,
                  int64_t b_cs, double *C, int64_t ldc, cudaStream_t st);
// group_store_xz for right-hand sides j0 .. j0 + cnt - 1 (x: cnt rows of n; b, ax: cnt rows of m).
cudaError_t group_store_xz_many(const double *x, int64_t n, const double *b, const double *ax, int64_t m, int64_t j0,
                                int64_t cnt, int g, double *X0, double *Z0, cudaStream_t st);
// batch capacity of a warm-start network (rebk_mlp.cu)
int64_t mlp_batch_capacity(::rebk_mlp_s *h);
// the same with an FP32 x (a correction): out[0] = sum (a + x - r)^2, out[1] = sum r^2.
cudaError_t err_norms_f32(const double *a, const float *x, const double *r, int64_t n, double *out,
                          cudaStream_t st);
cudaError_t sum_sq(const double *v, int64_t n, double *out, cudaStream_t st);
// f = b - z - ym (length m); g = yn copy handled by caller
cudaError_t form_f(const double *b, const double *z, const double *ym, double *f, int64_t m,
                   cudaStream_t st);
// x += yn (n), z -= ym (m)
cudaError_t apply_update(double *x, const double *yn, int64_t n, double *z, const double *ym,
                         int64_t m, cudaStream_t st);
cudaError_t fill_zero_f32(float *p, int64_t n, cudaStream_t st);
// dst = (double) src, n entries
cudaError_t widen_f32(const float *src, double *dst, int64_t n, cudaStream_t st);
// out = a - b (length n)
cudaError_t vec_sub(const double *a, const double *b, double *out, int64_t n, cudaStream_t st);

// Extreme Ritz values of A^T A on range(A^T) after up to `steps` Golub-Kahan-Lanczos
// steps with full reorthogonalisation (rebk_spectral.cu): sigma_1^2 from below and
// sigma_r^2 from above.  Synchronises st.
cudaError_t lanczos_extremes(const double *A, int64_t lda, int64_t m, int64_t n, int steps, uint64_t seed,
                             cudaStream_t st, double *sigma1_sq, double *sigma_r_sq, int *steps_done);

// Arguments of the partition-free kernel (rebk_free.cu): Algorithm 1's step on
// index sets drawn independently per row / column (plain FP64).
struct FreeArgs {
    const double *A;        // FP64 copy, row-major, leading dimension lda
    const double *AT;       // FP64 copy of A^T, n rows of leading dimension ldt
    int64_t ldt;
    int64_t lda, m, n;
    int tau_r, tau_c;       // rows and columns drawn per iteration
    const double *rn, *cn;  // squared row / column norms
    double alpha;
    const int32_t *idx;     // [iters][tau_c + tau_r]: column draws, then row draws
    int64_t iters;
    double *z, *x;
    const double *b;
    double *acc;            // 3 sets of acc_w doubles (r, w, test partial), zeroed before launch
    int acc_w;
    unsigned int *bar;      // zeroed before launch
    int *status;            // zeroed before launch
    int64_t *iters_done;
    const double *x_ref;    // NULL = no error test
    double tol2_abs;
    int64_t check_every, check_offset;
    unsigned long long timeout_ns;
};
// idx[it][q]: draw q of iteration k0 + it + 1 (columns q < tau_c from the
// column draw's slots, rows after them from the row draw's slots).
cudaError_t free_sample(uint64_t seed, uint64_t stream, int64_t k0, int64_t K, const double *cdf_r, int64_t m,
                        const double *cdf_c, int64_t n, int tau_r, int tau_c, int fb_r, int fb_c, int32_t *idx,
                        cudaStream_t st);
cudaError_t launch_free(const FreeArgs &a, int G, cudaStream_t st);
// AT (n rows of ldt) = A^T (A: m rows of lda), FP64.
cudaError_t transpose_f64(const double *A, int64_t lda, int64_t m, int64_t n, double *AT, int64_t ldt,
                          cudaStream_t st);
size_t free_smem_bytes(int tau_r, int tau_c);
int free_max_ctas(int tau_r, int tau_c);

// Tensor-core BF16 GEMM (rebk_umma.cu): C (M x N) = alpha * A B^T with A (M x K)
// and B (N x K) K-contiguous BF16 rows (leading dimensions lda, ldb); FP32
// accumulation; epilogue writes FP32 C (ldc), a BF16 copy Cb and a transposed
// BF16 copy CbT (CbT[j * ldcbt + i]), each optional, after ReLU and a mask
// (mask[i * ldm + j] > 0).  Splits K when the output has few tiles and the
// workspace ws (ws_floats floats; umma_workspace_floats() always suffice) holds
// the partial slices, summed in a fixed order.  *error (device int) is set when
// a bounded wait gave up.
bool umma_gemm_supported(int M, int N, int K, const void *A, int64_t lda, const void *B, int64_t ldb);
size_t umma_workspace_floats();
cudaError_t umma_gemm(int M, int N, int K, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                      int64_t ldb, float alpha, float *C, int64_t ldc, __nv_bfloat16 *Cb, int64_t ldcb,
                      __nv_bfloat16 *CbT, int64_t ldcbt, int relu, const float *mask, int64_t ldm, float *ws,
                      size_t ws_floats, int *error, cudaStream_t st);

// Several right-hand sides of one matrix at once (rebk_multi.cu): Algorithm 1 in
// the correction form for NR right-hand sides sharing one block sequence.
// Vectors of NR right-hand sides are interleaved: entry (row i, right-hand side
// q) at [i * NR + q].
struct MultiArgs {
    // matrix copy (A, lda, m, n), blocks (tau_r, tau_c, s, t, row_off, col_off),
    // FP32 step coefficients (coef_r, coef_c), draws (idx, iters), tensor maps and
    // tile geometry (bw_c, bh_c, nbox_c, bw_r, tile bytes, tma_vx), owned-slice
    // capacities, FP32 accumulators (acc: 3 sets x kMultiReplicas x acc_w), barrier,
    // status, iters_done and timeout
    GridArgs geo;
    float *dZ, *dX, *S, *V;  // corrections and duals: [m][NR], [n][NR], [n][NR], [m][NR]
    const float *F, *G;      // f = b - z - A x ([m][NR]) and g = A^T z ([n][NR]), rounded to FP32
    int scr_floats;          // reduction scratch in shared memory (floats)
    int mma;                 // products on tensor cores (FP32 storage, NR = 8): tile strides and
                             // slack set for them (multi_setup)
};

constexpr int kMultiReplicas = 2;

struct MultiSmem {
    size_t tc0, tc1, tr0, tr1, zeta, xi, w, r, scr, total;
};

// Shared-memory layout of the multi kernel (byte offsets): 512-byte header
// (mbarriers, flags, step coefficients), two column tiles, two row tiles, dZ of
// the owned rows ([nrow_cap rounded up to 8][NR]), dX of the owned columns
// (q-major: [NR][xs]), w (q-major: [NR][ws]), r ([tau_r rounded up to 8][NR]) and
// the scratch.  Tile sizes include the slack the tensor-core products read past
// the copied box (zero-filled at launch).
__host__ __device__ inline int multi_xs(int ncol_cap) { return (ncol_cap + 31) / 32 * 32 + 4; }
__host__ __device__ inline int multi_ws(int tau_c) { return (tau_c + 31) / 32 * 32 + 4; }
__host__ __device__ inline MultiSmem multi_smem_layout(int nrow_cap, int ncol_cap, int tau_r, int tau_c, int nr,
                                                       int64_t tile_c_bytes, int64_t tile_r_bytes, int scr_floats) {
    auto al128 = [](size_t x) { return (x + 127) & ~(size_t)127; };
    MultiSmem L;
    size_t o = 512;
    L.tc0 = o; o = al128(o + (size_t)tile_c_bytes);
    L.tc1 = o; o = al128(o + (size_t)tile_c_bytes);
    L.tr0 = o; o = al128(o + (size_t)tile_r_bytes);
    L.tr1 = o; o = al128(o + (size_t)tile_r_bytes);
    L.zeta = o; o = al128(o + (size_t)((nrow_cap + 7) / 8 * 8) * nr * 4);
    L.xi = o;   o = al128(o + (size_t)nr * multi_xs(ncol_cap) * 4);
    L.w = o;    o = al128(o + (size_t)nr * multi_ws(tau_c) * 4);
    L.r = o;    o = al128(o + (size_t)((tau_r + 7) / 8 * 8) * nr * 4);
    L.scr = o;  o = al128(o + (size_t)scr_floats * 4);
    L.total = o;
    return L;
}
size_t multi_smem_bytes(const MultiArgs &M, int nr);
cudaError_t launch_multi(const MultiArgs &M, bool bf16, int nr, int G, cudaStream_t st);
int multi_max_ctas(bool bf16, int nr, bool mma, size_t smem);
// FP64 products with nr interleaved vectors: Y = A P (P: [n][nr], Y: [m][nr]) and
// Y = A^T Q (Q: [m][nr], Y: [n][nr]); P / Q FP64 or FP32 (p_f32); Y is overwritten.
cudaError_t multi_ap(const double *A, int64_t lda, int64_t m, int64_t n, int nr, const void *P, bool p_f32,
                     double *Y, cudaStream_t st);
cudaError_t multi_atq(const double *A, int64_t lda, int64_t m, int64_t n, int nr, const void *Q, bool q_f32,
                      double *Y, cudaStream_t st);
// out[q] = sum_i (a + b - r)^2 and out[nr + q] = sum_i r^2 over i < len for the
// interleaved vectors a (FP64), b (FP32), r (FP64); a, b may be NULL (zero).
cudaError_t multi_norms(const double *a, const float *b, const double *r, int64_t len, int nr, double *out,
                        cudaStream_t st);
// Interleave cnt vectors of length len (vector j at src + j * ld) into dst [len][nr]
// (vectors cnt .. nr - 1 zero), and back (the first cnt).
cudaError_t multi_gather(const double *src, int64_t ld, int64_t cnt, int64_t len, int nr, double *dst,
                         cudaStream_t st);
cudaError_t multi_scatter(const double *src, int64_t cnt, int64_t len, int nr, double *dst, int64_t ld,
                          cudaStream_t st);
// F = fp32(B - Z - Ym) (len m x nr), G = fp32(Yn) (len n x nr).
cudaError_t multi_form(const double *B, const double *Z, const double *Ym, float *F, int64_t m, const double *Yn,
                       float *G, int64_t n, int nr, cudaStream_t st);
// X += Yn (n x nr), Z -= Ym (m x nr).
cudaError_t multi_apply(double *X, const double *Yn, int64_t n, double *Z, const double *Ym, int64_t m, int nr,
                        cudaStream_t st);

// Sets the message rebk_last_error() returns on this thread (rebk_api.cu).
void set_last_error(const std::string &msg);

}  // namespace rebk
