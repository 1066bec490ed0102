/*
 * rebk.h -- C ABI of the GB300 (sm_103a) solver for the minimum-norm
 * least-squares solution A^+ b by randomized extended block Kaczmarz (REBK).
 *
 * Method: K. Du, W.-T. Si, X.-H. Sun, "Randomized extended block Kaczmarz for
 * solving least squares", arXiv:2001.04179.  The problem statement (Section 1)
 * is A x = b with A any real m x n matrix -- consistent or not, over- or
 * underdetermined, full rank or rank-deficient -- and the target is A^+ b.
 * The iteration is Algorithm 1 (Section 2) for any row and column partitions
 * (rebk_partition); the default is the contiguous equal-size blocks of
 * Section 3 (the last block may be shorter).
 *
 * Conventions for every call below:
 *  - Matrices are row-major FP64 with leading dimension lda >= n (elements).
 *  - "device" pointers are CUDA device addresses on the current device (for
 *    example torch tensor data_ptr()); "host" pointers are ordinary memory.
 *  - The caller owns every buffer it passes; the library never frees them and
 *    keeps no pointer to them after the call returns.  The library owns the
 *    handle and everything it allocated inside it (released by rebk_destroy).
 *  - Work is queued on the handle's stream (rebk_options.stream).  Solve calls
 *    synchronise that stream before returning (they read stopping results).
 *  - Errors: every call returns a rebk_status; on failure rebk_last_error()
 *    returns a message for the calling thread.  No C++ exception crosses the
 *    boundary.  Invalid arguments never reach a kernel.
 *  - Random draws (not specified by the paper): Philox4x64-10 with key
 *    (seed, stream_id) and counter (d, 0, 0, 0), d = 2(k-1) for the column
 *    draw and 2(k-1)+1 for the row draw of iteration k; u = (word0 >> 11) 2^-53;
 *    the block picked is the smallest index whose cumulative squared norm
 *    exceeds u ||A||_F^2 (Algorithm 1's sampling probabilities).
 */
#ifndef REBK_H
#define REBK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rebk_handle_s *rebk_handle;

typedef enum {
    REBK_OK = 0,
    REBK_EINVAL = 1,            /* invalid argument; nothing was launched            */
    REBK_ENOMEM = 2,            /* device or host allocation failed                  */
    REBK_ECUDA = 3,             /* a CUDA call failed (message in rebk_last_error)   */
    REBK_MAX_ITER = 4,          /* stopping test not met within max_iter; x is the
                                   last iterate                                      */
    REBK_DIVERGED = 5,          /* a reduced block product became Inf/NaN            */
    REBK_BARRIER_TIMEOUT = 6,   /* a device-wide wait gave up (bounded spin); x and z
                                   are not updated                                   */
    REBK_EUNSUPPORTED = 7       /* size or option outside what the library handles   */
} rebk_status;

/* Storage precision of the matrix copy used by the inner sweeps. */
typedef enum { REBK_FP64 = 0, REBK_FP32 = 1, REBK_BF16 = 2 } rebk_storage;

typedef struct {
    int64_t tau_row;       /* row block size tau >= 1 (Section 3 partition of [m]);
                              ignored when rebk_partition gives row offsets             */
    int64_t tau_col;       /* column block size >= 1 (partition of [n]); ignored when
                              rebk_partition gives column offsets                       */
    int32_t storage_mask;  /* extra copies to keep: (1<<REBK_FP32) | (1<<REBK_BF16);
                              the FP64 copy is always kept                              */
    int32_t num_ctas;      /* CTAs of the persistent solve kernel; 0 = library choice  */
    int64_t check_every;   /* iterations between stopping tests; 0 = library default   */
    void *stream;          /* cudaStream_t for all work; NULL = legacy default stream  */
} rebk_options;

typedef struct {
    int64_t iterations;    /* iterations of Algorithm 1 run (all passes for refinement) */
    int32_t outer;         /* refinement passes (0 for the plain solve)                 */
    int32_t status;        /* rebk_status of the solve                                  */
    double rel_err;        /* ||x - x_ref|| / ||x_ref|| at exit if x_ref given, else -1 */
    double resid_f;        /* ||b - z - A x|| / ||b|| at exit when computed, else -1    */
    double resid_g;        /* ||A^T z|| / (||A||_F ||b||) at exit when computed, else -1 */
    double device_ms;      /* device time from the first to the last queued work of the
                              solve (CUDA events on the handle's stream)                */
    double kernel_ms;      /* summed CUDA-event time of the persistent REBK launches    */
    double sweep_ms;       /* summed CUDA-event time of the FP64 sweeps over A          */
    int64_t launches;      /* kernels of this library launched by the solve             */
    int64_t grid_launches; /* of which persistent REBK launches                         */
} rebk_stats;

/* Optional inputs/outputs of a solve.  Zero-initialise and set what you need. */
typedef struct {
    const double *x_ref;   /* device, n: stop when ||x - x_ref||_2 <= tol ||x_ref||_2
                              (the paper's stop rule, Section 3); NULL = residual test  */
    const double *x0;      /* device, n: initial x (Theorem main needs x0 in range(A^T));
                              NULL = 0 (Section 3)                                      */
    const double *z0;      /* device, m: initial z (Theorem main needs z0 in b+range(A));
                              NULL = b (Section 3)                                      */
    double *z_out;         /* device, m: final z (NULL = not returned)                  */
    int32_t *idx_out;      /* device, 2*max_iter int32: (j_k, i_k) per iteration run    */
    int64_t k0;            /* first iteration is k0+1 (resume a random stream)          */
    uint64_t stream_id;    /* Philox key word 1                                         */
} rebk_solve_ext;

/* Options of the mixed-precision solve. */
typedef struct {
    int32_t storage;          /* REBK_FP32 or REBK_BF16 (must be in storage_mask)      */
    int32_t max_outer;        /* refinement passes at most; 0 = 30                      */
    int64_t inner_iters;      /* iterations per pass at most; 0 = library default       */
    double inner_reduction;   /* with x_ref: a pass ends once the error is below this
                                 fraction of its value at the pass start (0 = 1e-4 for
                                 FP32, 1e-2 for BF16)                                    */
} rebk_refine_opts;

/*
 * Partitions of the rows and columns for Algorithm 1 (Section 2: the row
 * blocks I_1..I_s partition [m], the column blocks J_1..J_t partition [n]).
 * Offsets are host arrays: block i of the rows is [row_off[i], row_off[i+1]),
 * with 0 = row_off[0] < row_off[1] < ... < row_off[s] = m (no empty block);
 * likewise col_off (t + 1 entries) for the columns.  A NULL offset array
 * selects the contiguous partition of Section 3's experiments: blocks of
 * rebk_options.tau_row (tau_col) consecutive rows (columns), the last one
 * shorter (s and t are then ignored).  Every block has at most 512 rows or
 * columns.  The library copies the offsets.
 */
typedef struct {
    const int64_t *row_off;  /* host, s + 1 entries, or NULL                      */
    int64_t s;               /* number of row blocks (with row_off)               */
    const int64_t *col_off;  /* host, t + 1 entries, or NULL                      */
    int64_t t;               /* number of column blocks (with col_off)            */
} rebk_partition;

/*
 * Creates a solver for the m x n matrix A (row-major, leading dimension lda,
 * host memory if A_on_device == 0, device memory otherwise; the library copies
 * it) with the block partitions *part (NULL = contiguous blocks of the sizes in
 * opt, see rebk_partition).  Builds the block squared Frobenius norm tables
 * and their prefix sums (Algorithm 1 sampling) in FP64 on the device, and the
 * reduced-precision copies named in opt->storage_mask.
 * alpha > 0 is the step size of Algorithm 1; alpha <= 0 picks 1.75 / beta_max
 * (Section 3's empirical choice) with beta_max from rebk_beta_max.
 * Errors: EINVAL (m, n, lda, tau out of range, NULL pointers, offsets not
 * strictly increasing from 0 to m / n), EUNSUPPORTED (a block above 512),
 * ENOMEM, ECUDA.  A matrix of all zeros is accepted (every solve returns
 * x = 0 = A^+ b).
 */
rebk_status rebk_create(rebk_handle *out, const double *A, int64_t m, int64_t n, int64_t lda,
                        int A_on_device, const rebk_partition *part, double alpha, const rebk_options *opt);

/* Releases everything the handle owns.  NULL is ignored. */
void rebk_destroy(rebk_handle h);

/*
 * Plain FP64 REBK (Algorithm 1) from z0 = b, x0 = 0 (Section 3).
 * b: device, m.  x: device, n (output).  Stops at the first multiple of
 * check_every iterations where the residual test holds:
 *   max(||b - z - A x|| / ||b||, ||A^T z|| / (||A||_F ||b||)) <= tol
 * (both vanish exactly at x = A^+ b, z = (I - A A^+) b), or after max_iter
 * iterations (REBK_MAX_ITER).  tol <= 0 runs exactly max_iter iterations.
 */
rebk_status rebk_solve(rebk_handle h, const double *b, double *x, double tol, int64_t max_iter,
                       uint64_t seed, rebk_stats *stats);

/*
 * As rebk_solve with the optional inputs/outputs of rebk_solve_ext (ext may be
 * NULL).  With ext->x_ref the stop rule is the relative error (checked every
 * check_every iterations; x returned is the iterate that passed).  With an
 * early stop, z_out holds z one iteration past the returned x (the column step
 * of the next iteration was already applied).  With idx_out, entries for the
 * iterations run are written.
 */
rebk_status rebk_solve_ex(rebk_handle h, const double *b, double *x, double tol, int64_t max_iter,
                          uint64_t seed, const rebk_solve_ext *ext, rebk_stats *stats);

/*
 * Mixed precision: Algorithm 1 applied to corrections with the FP32 or BF16
 * copy of A (FP32 arithmetic), inside an FP64 refinement loop on (x, z):
 *   f = b - z - A x,  g = A^T z                      (FP64 sweep over A)
 *   inner: dz <- dz - cJ A_J (A_J^T dz + g_J),  s_J += cJ (A_J^T dz + g_J)
 *          dx <- dx - cI A_I^T (A_I dx - f_I + dz_I),  v_I -= cI (same residual)
 *   z <- z - A s,  x <- x + A^T v                     (FP64 sweep over A)
 * so x stays in range(A^T) and z in b + range(A) to FP64 rounding (the
 * hypotheses of Theorem main), and A^+ b is a fixed point.  The random stream
 * continues across passes.  Stop: relative error <= tol with ext->x_ref, else
 * the residual test of rebk_solve after each pass.  max_iter bounds the total
 * inner iterations.  Sampling table and step sizes come from FP64 A.
 */
rebk_status rebk_solve_refined(rebk_handle h, const double *b, double *x, double tol,
                               int64_t max_iter, uint64_t seed, const rebk_refine_opts *ropt,
                               const rebk_solve_ext *ext, rebk_stats *stats);

/*
 * Algorithm 1 with index sets drawn without a partition (plain FP64).  Section 4
 * names variants of REBK whose random samplings do not depend on partitions;
 * the reading built here: iteration k draws tau_col column indices
 * independently, each with probability ||A_{:,j}||^2 / ||A||_F^2, and tau_row
 * row indices likewise with ||A_{i,:}||^2 / ||A||_F^2, and takes Algorithm 1's
 * step on the drawn columns A_J and rows A_I (a repeated draw repeats its
 * column or row; ||A_J||_F^2 sums the drawn columns' squared norms):
 *   z <- z - alpha / ||A_J||_F^2 A_J A_J^T z,
 *   x <- x - alpha / ||A_I||_F^2 A_I^T (A_I x - b_I + z_I).
 * Each step is non-expansive for 0 < alpha < 2.  At tau_row = tau_col = 1 it is
 * the randomized extended Kaczmarz method.  Draw q (0-based) of the column set
 * of iteration k uses Philox counter (2(k-1), q, 0, 0), of the row set
 * (2(k-1)+1, q, 0, 0), key (seed, ext->stream_id), word 0 as in rebk_solve.
 * h: any handle (its FP64 copy of A; the per-row and per-column norm tables and
 * an FP64 copy of A^T, n x m, from which the drawn columns are read as contiguous
 * rows, are built on the first call and kept with the handle).  alpha > 0: the
 * step; <= 0: the handle's alpha.
 * tau_row, tau_col in [1, 512].  ext as for rebk_solve_ex (x_ref stop rule
 * checked every check_every iterations, x0, z0, z_out, k0, stream_id), except
 * idx_out: device, (tau_col + tau_row) x max_iter int32 -- per iteration the
 * column draws, then the row draws.  Without x_ref (or tol <= 0) the solve runs
 * max_iter iterations.  Errors: EINVAL, EUNSUPPORTED (tau above 512), ENOMEM,
 * ECUDA, DIVERGED, BARRIER_TIMEOUT.
 */
rebk_status rebk_solve_free(rebk_handle h, int64_t tau_row, int64_t tau_col, double alpha, const double *b,
                            double *x, double tol, int64_t max_iter, uint64_t seed, const rebk_solve_ext *ext,
                            rebk_stats *stats);

/* Options of the multi-right-hand-side solve.  Zero-initialise and set what you need. */
typedef struct {
    int32_t storage;          /* REBK_FP32 or REBK_BF16 (must be in storage_mask)        */
    int32_t group;            /* right-hand sides per launch, 4 or 8; 0 = the largest
                                 whose tiles fit in shared memory                          */
    int32_t max_outer;        /* refinement passes per group at most; 0 = 30              */
    int32_t reserved;         /* 0                                                         */
    int64_t inner_iters;      /* iterations per pass at most; 0 = library default         */
    double inner_reduction;   /* as rebk_refine_opts.inner_reduction                      */
    int32_t *idx_out;         /* device, optional: (j_k, i_k) of the first group's
                                 iterations, 2 * max_iter int32                            */
    uint64_t stream_id;       /* Philox key word 1 of the first group; group g uses
                                 stream_id + g                                             */
} rebk_multi_opts;

/*
 * nrhs right-hand sides of one matrix.  Each one is solved as rebk_solve_refined
 * solves one (Algorithm 1 of Section 2 on corrections with the FP32 or BF16 copy
 * of A and FP32 arithmetic, inside the FP64 refinement loop on (x, z), x^0 = 0,
 * z^0 = b), and the right-hand sides run in groups of `group` that share one
 * block sequence: iteration k of every member draws the (J_k, I_k) that
 * rebk_solve_refined draws with the same seed and stream id, so one read of a
 * sampled block serves the whole group.  Group g (right-hand sides g*group ..
 * g*group + group - 1) uses Philox key (seed, opt->stream_id + g).
 * B: device, right-hand side j at B + j*ldb (m entries, ldb >= m).  X: device,
 * solution j written at X + j*ldx (n entries, ldx >= n).  X_ref: device or NULL,
 * reference j at X_ref + j*ldxr; with it a group stops once every member's
 * relative error ||x - x_ref|| / ||x_ref|| <= tol, without it once every member
 * passes the residual test of rebk_solve.  max_iter bounds each group's inner
 * iterations.  rel_out: host, nrhs doubles or NULL: per right-hand side the final
 * relative error (with X_ref) or max(resid_f, resid_g).  stats: totals over the
 * groups (iterations summed, outer the largest pass count, rel_err the largest
 * error).  Needs the tiles of the persistent kernel to fit a TMA box (tau_row,
 * tau_col and the owned column slice at most 256).  Errors: EINVAL, EUNSUPPORTED,
 * ENOMEM, ECUDA, DIVERGED, BARRIER_TIMEOUT; MAX_ITER when a group ends short of tol.
 */
rebk_status rebk_solve_multi(rebk_handle h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                             double tol, int64_t max_iter, uint64_t seed, const rebk_multi_opts *opt,
                             const double *X_ref, int64_t ldxr, double *rel_out, rebk_stats *stats);

/* The group size rebk_solve_multi picks for a storage (REBK_FP32 or REBK_BF16)
 * when rebk_multi_opts.group is 0: 8, or 4 when the tiles of 8 do not fit. */
rebk_status rebk_multi_group(rebk_handle h, int32_t storage, int32_t *group);

/*
 * beta^I_max and beta^J_max of Section 2.2 (largest ||block||_2^2 / ||block||_F^2
 * over the row blocks and over the column blocks), from FP64 block Gram
 * matrices and power iteration on the device.  Outputs are host doubles.
 */
rebk_status rebk_beta_max(rebk_handle h, double *beta_row, double *beta_col);

/* Step size alpha in use (host double). */
rebk_status rebk_get_alpha(rebk_handle h, double *alpha);

/*
 * Replaces the step size alpha of Algorithm 1 (Section 2.2 requires
 * 0 < alpha < 2 / max(beta^I_max, beta^J_max) for Theorem main) and rebuilds
 * the per-block coefficients alpha / ||block||_F^2 in FP64 and FP32 on the
 * handle's stream; the call synchronises that stream.  Any alpha > 0 is
 * accepted (a value past the bound may diverge: solves then return
 * REBK_DIVERGED or REBK_MAX_ITER).  Errors: EINVAL (NULL handle, alpha not
 * finite or <= 0), ECUDA.
 */
rebk_status rebk_set_alpha(rebk_handle h, double alpha);

/* Spectral quantities of Section 2's step-size results (rebk_spectral_estimates). */
typedef struct {
    double sigma1_sq;      /* largest Ritz value of A^T A: sigma_1(A)^2, approached from below  */
    double sigma_r_sq;     /* smallest Ritz value on range(A^T): sigma_r(A)^2 (smallest nonzero
                              singular value squared), approached from above                  */
    double fro2;           /* ||A||_F^2                                                         */
    double alpha_mean_opt; /* 2 ||A||_F^2 / (sigma1_sq + sigma_r_sq): Remark alpha's minimiser of
                              Theorem ner's rate delta (mean error only: far above 2 / beta_max
                              for most matrices, where single runs diverge)                     */
    double delta_opt;      /* (sigma1_sq - sigma_r_sq) / (sigma1_sq + sigma_r_sq), delta there    */
    double alpha;          /* the handle's alpha, at which the next four are evaluated          */
    double delta;          /* Theorem ner: max |1 - alpha sigma_i^2 / ||A||_F^2|                  */
    double eta;            /* Theorem main: 1 - (2 alpha - alpha^2 beta^I_max) sigma_r^2 / ||A||_F^2 */
    double rho;            /* Lemma estz: 1 - (2 alpha - alpha^2 beta^J_max) sigma_r^2 / ||A||_F^2   */
    double beta_row;       /* beta^I_max (Section 2.2)                                            */
    double beta_col;       /* beta^J_max                                                          */
    int32_t steps;         /* Lanczos steps taken (fewer than asked on an invariant subspace)     */
} rebk_spectrum;

/*
 * sigma_1^2 and sigma_r^2 of A (Section 2.1; r = rank A) by Golub-Kahan-Lanczos
 * bidiagonalisation in FP64 on the device with full reorthogonalisation
 * (steps in [1, 2048]; the start vector is a fixed function of seed), and the
 * step-size quantities of Remark alpha, Theorem ner and Theorem main built from
 * them (host struct *out).  The Ritz values bracket the spectrum from inside:
 * exact once steps reaches the rank (the iteration stops there), otherwise
 * sigma1_sq converges fast and sigma_r_sq slowly from above, so eta and rho
 * are optimistic until then.  Ritz values below 1e-12 sigma1_sq count as
 * zero (the numerical rank; on a rank-deficient A the last steps before the
 * rank can pick up a null-space direction, whose Ritz value is dropped).
 * Working memory (m + n) (steps + 1) doubles.
 * Errors: EINVAL (NULL, steps out of range), ENOMEM, ECUDA.  A = 0 gives zeros.
 */
rebk_status rebk_spectral_estimates(rebk_handle h, int32_t steps, uint64_t seed, rebk_spectrum *out);

/* Number of row blocks s and column blocks t (host int64). */
rebk_status rebk_get_blocks(rebk_handle h, int64_t *s, int64_t *t);

/*
 * Copies the partition in use to host arrays row_off (s + 1 entries) and
 * col_off (t + 1 entries), either may be NULL; *tau_row / *tau_col (may be
 * NULL) receive the largest block size of each.
 */
rebk_status rebk_get_partition(rebk_handle h, int64_t *row_off, int64_t *col_off, int64_t *tau_row,
                               int64_t *tau_col);

/*
 * Copies the FP64 block tables to host arrays: nr (s), nc (t) squared
 * Frobenius norms, cdf_r (s), cdf_c (t) inclusive prefix sums.  Any may be NULL.
 */
rebk_status rebk_get_tables(rebk_handle h, double *nr, double *nc, double *cdf_r, double *cdf_c);

/*
 * Copies the stored copy of A in the given precision to host memory as an
 * m x n row-major array of that type (8, 4 or 2 bytes per element; BF16 as
 * raw uint16 bits).  The copy is FP64 -> FP32 -> BF16, each round to nearest
 * even.
 */
rebk_status rebk_export_storage(rebk_handle h, int32_t storage, void *host_out);

/* ------------------------------------------------------------------------ */
/* Block-size autotuner                                                     */
/* ------------------------------------------------------------------------ */

/* One candidate of rebk_tune_tau. */
typedef struct {
    int64_t tau;           /* block size of rows and columns (clipped to m and n)      */
    double beta_max;       /* max(beta^I_max, beta^J_max) at this tau (Section 2.2)    */
    double alpha;          /* step size used: alpha_factor / beta_max                  */
    int64_t iterations;    /* mean iterations of the trials                            */
    double device_ms;      /* mean device time of a solve (rebk_stats.device_ms);
                              -1 if a trial missed the tolerance                        */
    int32_t status;        /* REBK_OK, or REBK_MAX_ITER / REBK_DIVERGED of the worst trial */
} rebk_tune_point;

/*
 * Measures the time to tolerance of Algorithm 1 for each candidate block size
 * taus[0..count) -- the same tau for the row and the column partition, as in
 * the experiments of Section 3 -- and returns the fastest in *best_tau.
 * For each candidate: a solver is created (A: m x n row-major, leading
 * dimension lda, on the device if A_on_device, else on the host and uploaded
 * once), alpha = alpha_factor / max(beta^I_max, beta^J_max) (alpha_factor <= 0
 * means 1.75, Section 3's empirical choice), one short untimed solve picks the
 * persistent kernel's launch shape, then `trials` solves with seeds seed,
 * seed+1, ... run to tol: plain FP64 (storage = REBK_FP64, rebk_solve_ex) or
 * mixed precision (REBK_FP32 / REBK_BF16, rebk_solve_refined); with x_ref
 * (device, n) the stop rule is the relative error, else the residual test of
 * rebk_solve.  b: device, m.  opt supplies stream, num_ctas, check_every and
 * extra storage (its tau fields are ignored).  points: host array of count
 * entries, filled in candidate order.
 * Returns REBK_MAX_ITER (best_tau = 0) when no candidate reached tol.
 * Errors: EINVAL (NULL pointers, count < 1, a tau < 1, unknown storage,
 * tol <= 0, max_iter < 1, trials < 1), EUNSUPPORTED (tau > 512), ENOMEM,
 * ECUDA.
 */
rebk_status rebk_tune_tau(const double *A, int64_t m, int64_t n, int64_t lda, int A_on_device,
                          const double *b, const double *x_ref, const int64_t *taus, int32_t count,
                          double alpha_factor, int32_t storage, double tol, int64_t max_iter,
                          uint64_t seed, int32_t trials, const rebk_options *opt,
                          rebk_tune_point *points, int64_t *best_tau);

/* ------------------------------------------------------------------------ */
/* Batches of independent systems                                           */
/* ------------------------------------------------------------------------ */

typedef struct rebk_batch_s *rebk_batch;

typedef struct {
    int32_t tau;          /* block size for rows and columns of every system (Section 3
                             partitions), 1..256; 0 = autotune over {16, 32, 64, 128, 256}
                             and, for 16 and 32, the column step's tile shape, on a
                             sample of the systems at the first solve                   */
    int32_t nrhs;         /* right-hand sides per system, 1..8 (all share one block
                             sequence per system)                                       */
    int32_t max_outer;    /* refinement passes at most; 0 = 6                           */
    int32_t check_every;  /* inner iterations between error tests; 0 = 10               */
    double inner_reduction; /* a pass ends once every RHS error is below this fraction
                               of its value at the pass start; 0 = 1e-4                */
    void *stream;         /* cudaStream_t for all work; NULL = legacy default stream    */
    int32_t col_path;     /* column-step tile shape for blocks of 16 or 32 columns: 0 =
                             16-byte vectors over tau/4 lanes of a row, 1 = one lane per
                             column; with tau = 0 the autotuner picks it               */
    int32_t cluster;      /* CTAs per thread-block cluster for the systems predicted to
                             run longest: each such system runs on a whole cluster (its
                             rows and columns split over the CTAs, the two block
                             products added up through distributed shared memory), the
                             others on one CTA each; 1 = every system on one CTA,
                             2 / 4 / 8; 0 = library choice: clusters of 2, and the
                             few longest systems (predicted at >= 2x the mean load
                             per SM, at most 8) on clusters of 4 in a launch of their
                             own beside the main one                                  */
    double joint_frac;    /* a system runs on a cluster when its predicted time (the
                             previous solve's iterations times a per-iteration cost
                             model) is at least joint_frac x the mean load per CTA;
                             0 = 0.25, and no clusters when every system qualifies     */
} rebk_batch_options;

typedef struct {
    int32_t converged;     /* systems whose every RHS reached the tolerance            */
    int32_t outer;         /* refinement passes run                                   */
    int64_t iterations;    /* inner iterations summed over systems                    */
    int64_t max_iterations;/* largest per-system inner iteration count                */
    double device_ms;      /* device time of the solve (CUDA events)                  */
    double inner_ms;       /* summed event time of the persistent batch launches      */
    double sweep_ms;       /* summed event time of the FP64 sweeps                    */
    int64_t launches;      /* kernels launched by the solve (graph nodes counted)     */
    int32_t tau;           /* block size in use                                       */
    int32_t graph;         /* 1 if the passes ran as one CUDA graph                   */
    int32_t col_path;      /* column-step tile shape for blocks of 16 / 32 columns: 0 =
                              16-byte vectors over tau/4 lanes of a row, 1 = one lane
                              per column (picked with tau by the autotuner)           */
    int32_t cluster;       /* CTAs per cluster of the main launch (1 = no clusters)   */
    int32_t joint;         /* systems of the main launch run on a whole cluster       */
    int32_t top_cluster;   /* CTAs per cluster of the launch of the longest systems
                              beside the main one (library choice; 0 = none)          */
    int32_t top_joint;     /* systems in that launch                                  */
} rebk_batch_stats;

/*
 * Creates a batch of `count` independent systems A_i x = b_i (Section 1 for
 * each: any shape, rank or consistency).  m[i], n[i] (host arrays) are the
 * shapes; A[i] (host array of pointers) points to row-major FP64 matrices with
 * leading dimension n[i], in host memory (A_on_device == 0) or device memory.
 * The library copies every matrix (FP64 for the refinement sweeps, FP32 for
 * the inner iterations) and builds each system's block tables; systems given
 * the same pointer with the same shape share one stored copy (a stream of
 * right-hand-side groups for one matrix: each system then holds up to eight
 * right-hand sides and its own block sequence).  alpha (host
 * array, may be NULL) gives each system's step size; NULL or a value <= 0 picks
 * 1.75 / beta_max of that system (Section 3's empirical choice).
 * Errors: EINVAL (count < 1, shapes, NULL pointers, options), ENOMEM, ECUDA.
 */
rebk_status rebk_batch_create(rebk_batch *out, int32_t count, const int64_t *m, const int64_t *n,
                              const double *const *A, int A_on_device, const double *alpha,
                              const rebk_batch_options *opt);

void rebk_batch_destroy(rebk_batch h);

/*
 * Solves every system of the batch for its nrhs right-hand sides by mixed
 * precision REBK (the correction form of rebk_solve_refined: FP32 inner
 * iterations, FP64 refinement of (x, z)), one persistent launch per
 * refinement pass in which each CTA takes systems from a queue.
 * B: device, the systems' right-hand sides concatenated, system i occupying
 *    m[i] rows of nrhs doubles (row-major m[i] x nrhs).
 * X: device, output, concatenated n[i] x nrhs blocks.
 * X_ref: device, n[i] x nrhs blocks of the known solutions A_i^+ b_i (the
 *    paper's stop rule, Section 3); a system stops when every RHS has
 *    ||x - x_ref|| <= tol ||x_ref||.  NULL: fixed passes (max_outer) of
 *    inner_iters iterations each, no stopping test.
 * max_iter bounds each system's inner iterations (systems that need more,
 * e.g. nearly square Gaussian ones, end unconverged).  Random draws: Philox
 * key (seed, system index), the same counter layout as rebk_solve.
 * status_out (device or NULL): int32 per system, REBK_OK or REBK_MAX_ITER.
 */
rebk_status rebk_batch_solve(rebk_batch h, const double *B, double *X, const double *X_ref, double tol,
                             int64_t max_iter, int64_t inner_iters, uint64_t seed, int32_t *status_out,
                             rebk_batch_stats *stats);

/*
 * rebk_batch_solve from given starting points: X0 (device, n[i] x nrhs
 * blocks like X, or NULL for x^0 = 0) and Z0 (device, m[i] x nrhs blocks like
 * B, or NULL for z^0 = b).  Theorem main's hypotheses are x^0 in range(A_i^T)
 * and z^0 in b + range(A_i) for every right-hand side (the learned warm start
 * x^0 = A^T y, z^0 = b - A x^0 meets both); the limit is then A_i^+ b.
 */
rebk_status rebk_batch_solve_ex(rebk_batch h, const double *B, double *X, const double *X_ref,
                                const double *X0, const double *Z0, double tol, int64_t max_iter,
                                int64_t inner_iters, uint64_t seed, int32_t *status_out,
                                rebk_batch_stats *stats);

/*
 * Records, during the following solves of the batch, what each system's
 * Algorithm 1 iterations did (for parity checks against a reference):
 * idx_out (device, count x idx_cap x 2 int32, or NULL = stop recording): entry
 * (i, k-1) holds (j_k, i_k), the column and row blocks system i drew at its
 * iteration k (Philox key (seed, i), the counter layout of rebk_solve), for
 * the iterations k <= idx_cap that the solve ran (entries past a system's last
 * iteration are left as they were); Z_out (device, laid out like B, or NULL):
 * the final z of every right-hand side.  The tuning solves of an autotuned
 * first solve (tau = 0) record too; set the block size to record one solve.
 * The buffers must stay valid until recording is switched off.
 * Errors: EINVAL (NULL handle, idx_out with idx_cap < 1).
 */
rebk_status rebk_batch_record(rebk_batch h, int32_t *idx_out, int64_t idx_cap, double *Z_out);

/* Block size in use and the number of systems (host outputs; either may be NULL). */
rebk_status rebk_batch_info(rebk_batch h, int32_t *tau, int32_t *count);

/* ------------------------------------------------------------------------ */
/* Learned warm start                                                        */
/* ------------------------------------------------------------------------ */

typedef struct rebk_mlp_s *rebk_mlp;

/*
 * Creates the warm-start network y = W3 relu(W2 relu(W1 b)) for right-hand
 * sides b of length m (W1: hidden x m, W2: hidden x hidden, W3: m x hidden,
 * row-major), tied to the m x n matrix A (FP64 row-major, leading dimension
 * n, host or device memory; the library keeps a BF16 copy) through its loss
 * mean ||A^T y - x_ls||^2.  The solve then starts from x^0 = A^T y (in
 * range(A^T)) and z^0 = b - A x^0 (in b + range(A)): the hypotheses of
 * Theorem main hold, so the limit is still A^+ b.  The paper has no learned
 * start; this is our extension.
 * init_weights: host array of three FP32 arrays, or NULL for He-initialised
 * weights drawn from `seed`.  batch_capacity: largest batch of any call.
 * Arithmetic: BF16 operands with FP32 accumulation (tensor cores), FP32
 * master weights, Adam.  stream: cudaStream_t (NULL = legacy default).
 */
rebk_status rebk_mlp_create(rebk_mlp *out, const double *A, int64_t m, int64_t n, int A_on_device,
                            int64_t hidden, int64_t batch_capacity, const float *const *init_weights,
                            uint64_t seed, void *stream);
void rebk_mlp_destroy(rebk_mlp h);

/* Training losses of the network (rebk_mlp_set_loss). */
enum { REBK_MLP_LOSS_X = 0, REBK_MLP_LOSS_Y_REL = 1 };

/*
 * Selects the loss of rebk_mlp_gradients / rebk_mlp_train_step and the output
 * scale s of the network, y = s W3 relu(W2 relu(W1 b)):
 *   REBK_MLP_LOSS_X (default, s = 1): mean ||A^T y - x_ls||^2, targets x_ls
 *     (batch x n);
 *   REBK_MLP_LOSS_Y_REL: mean ||y - y*||^2 / ||y*||^2, targets y* = (A^T)^+ x_ls
 *     (batch x m; the minimum-norm solution of A^T y = x_ls, a REBK solve with
 *     the matrix A^T).  It weighs the error of x^0 = A^T y along singular value
 *     sigma by 1 / sigma^2: the directions Theorem main's rate makes slowest.
 * s (> 0) lets the output reach ||y*|| without huge last-layer weights.
 * Errors: EINVAL (NULL network, unknown loss, s not positive and finite).
 */
rebk_status rebk_mlp_set_loss(rebk_mlp h, int32_t loss, double out_scale);

/* Y (device, batch x m) = network applied to the rows of Bm (device, batch x m). */
rebk_status rebk_mlp_forward(rebk_mlp h, const double *Bm, int64_t batch, double *Y);

/*
 * Gradients of the selected loss (rebk_mlp_set_loss; default (1/batch)
 * sum_b ||A^T y_b - x_ls,b||^2) for the rows of Bm (device, batch x m) and the
 * targets Xls (device: x_ls, batch x n, for REBK_MLP_LOSS_X; y*, batch x m, for
 * REBK_MLP_LOSS_Y_REL; e.g. produced by the solver).  loss (host) may be NULL;
 * grads_host (three host FP32 arrays, any NULL) receives dL/dW_l.
 */
rebk_status rebk_mlp_gradients(rebk_mlp h, const double *Bm, const double *Xls, int64_t batch, double *loss,
                               float *const *grads_host);

/* One Adam step (lr; beta1 0.9, beta2 0.999, eps 1e-8) on the same loss. */
rebk_status rebk_mlp_train_step(rebk_mlp h, const double *Bm, const double *Xls, int64_t batch, double lr,
                                double *loss);

/* Copies the FP32 master weights to three host arrays (any NULL). */
rebk_status rebk_mlp_get_weights(rebk_mlp h, float *const *weights_host);

/* m (input / output length) and n (columns of A) of the network (host outputs). */
rebk_status rebk_mlp_shape(rebk_mlp h, int64_t *m, int64_t *n);

/*
 * The BF16 GEMM the warm-start network runs on, for direct use:
 * C (M x N, FP32, row-major, leading dimension ldc) = alpha * A B^T with A
 * (M x K) and B (N x K) BF16 (raw bits), row-major with leading dimensions
 * lda, ldb >= K, all device pointers.  FP32 accumulation.  When K, lda and ldb
 * are multiples of 8 and A, B are 16-byte aligned it runs on the fifth-
 * generation tensor cores (tcgen05 with TMA-staged tiles, accumulator in
 * tensor memory; *path = 1), else on a small mma.sync kernel (*path = 0; path
 * may be NULL).  stream: cudaStream_t (NULL = legacy default); the call
 * synchronises it.  The paper has no counterpart.
 * Errors: EINVAL (NULL pointers, shapes), EUNSUPPORTED (a dimension above
 * 2^31), ENOMEM, ECUDA (including a bounded wait inside the kernel that gave up).
 */
rebk_status rebk_gemm_bf16(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B, int64_t ldb,
                           float alpha, float *C, int64_t ldc, void *stream, int32_t *path);

/*
 * Warm start for rebk_solve_ex / rebk_solve_refined: y = net(b),
 * x0 = A^T y and z0 = b - A x0 computed with the solver's FP64 copy of A.
 * b: device, m; x0: device, n; z0: device, m (outputs).  Pass them as
 * rebk_solve_ext.x0 / .z0.
 */
rebk_status rebk_warm_start(rebk_handle h, rebk_mlp net, const double *b, double *x0, double *z0);

/*
 * rebk_warm_start for `count` right-hand sides at once (the network runs on
 * batches of up to its capacity).  Grouped layout: right-hand side j is column
 * j % group of block j / group, each block row-major (length x group) -- the
 * layout rebk_batch_solve_ex uses for systems sharing A with group = nrhs;
 * group = 1 is one right-hand side per row.  B: device, count / group blocks of
 * m x group; X0, Z0: device outputs, blocks of n x group and m x group.
 * Errors: EINVAL (NULL pointers, count not a positive multiple of group, shape
 * mismatch), ENOMEM (scratch of capacity x (2 m + n) doubles), ECUDA.
 */
rebk_status rebk_warm_start_batch(rebk_handle h, rebk_mlp net, const double *B, int64_t count, int32_t group,
                                  double *X0, double *Z0);

/*
 * Plain FP64 REBK for a fixed number of iterations without allocating any
 * memory.  The paper has no counterpart to this call.  It exists for callers
 * that must not call cudaMalloc: hosts that route every device allocation
 * through their own allocator or memory budget and forbid any other, and
 * real-time serving loops that must not take the driver's allocation locks or
 * risk an out-of-memory failure mid-request.
 *
 * A (device, m x n row-major, leading dimension lda), b (device, m) are
 * inputs; x (device, n) and z (device, m) are outputs: x^iters and z^iters of
 * Algorithm 1 from z^0 = b, x^0 = 0 with Philox key (seed, 0) -- the same
 * iterates rebk_solve_ex gives with stream_id 0 and k0 0, up to the
 * summation order of the device's reductions.  alpha > 0 is required (no
 * beta_max estimate here).  stream is a cudaStream_t (NULL = legacy default).
 * The call reads a few status words back to the host and synchronises the
 * stream before it returns.
 *
 * Working memory is one 32 MiB device array inside the library (every GPU that
 * loads the library holds it until the process exits).  It must hold a
 * zero-padded copy of A plus the tables: m * ceil(n/64)*64 * 8 bytes plus
 * about 520 n + 48 (m/tau_row + n/tau_col) bytes; larger problems are
 * rejected with REBK_EUNSUPPORTED before any GPU work.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) while
 * that device is current.
 * All calls share the array and each call overwrites and re-zeroes what it
 * needs; calls whose GPU work overlaps (other streams, other host threads on
 * the same device) race on it: serialise them.  A launch that runs fewer
 * iterations than asked returns REBK_ECUDA.
 */
rebk_status rebk_solve_noalloc(const double *A, int64_t m, int64_t n, int64_t lda, int64_t tau_row,
                               int64_t tau_col, double alpha, const double *b, double *x, double *z,
                               int64_t iters, uint64_t seed, void *stream);

/* ------------------------------------------------------------------------ */
/* Sparse matrices                                                           */
/* ------------------------------------------------------------------------ */

typedef struct rebk_sparse_s *rebk_sparse;

typedef struct {
    int32_t num_ctas;      /* persistent grid size; 0 = one CTA per SM                 */
    int32_t check_every;   /* stopping-test period in iterations; 0 = 10               */
    int32_t power_iters;   /* power iterations per block for beta_max; 0 = 100         */
    void *stream;          /* cudaStream_t for all work; NULL = legacy default stream  */
} rebk_sparse_options;

/*
 * Creates a solver for a sparse m x n matrix A in CSR form (host arrays:
 * row_ptr[m + 1] int64 with row_ptr[0] = 0, col_idx[nnz] int32 strictly
 * increasing within each row, val[nnz] FP64).  Algorithm 1 of Du, Si, Sun
 * (arXiv:2001.04179) with row blocks of tau_row consecutive rows and column
 * blocks of tau_col consecutive columns (the Section 3 partition), sampled by
 * their squared Frobenius norms (sums of squared values, FP64) through the same
 * Philox counter layout and tables as rebk_solve: on the same matrix stored
 * densely the two draw the same blocks.  The library keeps CSR (row blocks) and
 * a CSC copy built at creation (column blocks) on the device.  alpha <= 0
 * picks 1.75 / beta_max (Section 3's empirical step), beta_max = the largest
 * ||block||_2^2 / ||block||_F^2 over all blocks, ||block||_2 from power
 * iterations (host, FP64).
 * Errors: EINVAL (shapes, NULL pointers, indices out of range or unsorted),
 * ENOMEM, ECUDA.
 */
rebk_status rebk_sparse_create(rebk_sparse *out, int64_t m, int64_t n, const int64_t *row_ptr,
                               const int32_t *col_idx, const double *val, int64_t tau_row, int64_t tau_col,
                               double alpha, const rebk_sparse_options *opt);
void rebk_sparse_destroy(rebk_sparse h);

/*
 * Plain FP64 Algorithm 1 on the sparse matrix, as rebk_solve_ex: b (device, m),
 * x (device, n, output), ext optional (x_ref stop rule checked every
 * check_every iterations, x0, z0, z_out, idx_out, k0, stream_id).  Without
 * x_ref the solve runs max_iter iterations.  One persistent launch runs many
 * iterations, two device-wide barriers each: the row gather of iteration k and
 * the column gather of iteration k+1 in one phase, the x and z scatters (FP64
 * atomic adds) in the next.  Results match the dense solve of the same matrix
 * up to summation order.
 */
rebk_status rebk_sparse_solve(rebk_sparse h, const double *b, double *x, double tol, int64_t max_iter,
                              uint64_t seed, const rebk_solve_ext *ext, rebk_stats *stats);

/*
 * Mixed precision on the sparse matrix, as rebk_solve_refined: the inner
 * sweeps run the correction form of Algorithm 1 with FP32 copies of the values
 * (made at creation, round to nearest) and FP32 arithmetic; the residuals
 * f = b - z - A x, g = A^T z and the updates z <- z - A s, x <- x + A^T v use
 * the FP64 values (CSR for A p, CSC for A^T q).  ropt->storage must be
 * REBK_FP32 (REBK_BF16: EUNSUPPORTED).  Stop: relative error <= tol with
 * ext->x_ref (a pass ends at inner_reduction (default 1e-4) of its starting
 * error or when the error stops falling), else the residual test of
 * rebk_solve after each pass.  max_iter bounds the total inner iterations.
 */
rebk_status rebk_sparse_solve_refined(rebk_sparse h, const double *b, double *x, double tol, int64_t max_iter,
                                      uint64_t seed, const rebk_refine_opts *ropt, const rebk_solve_ext *ext,
                                      rebk_stats *stats);

/* alpha in use, the beta_max estimate and the block counts (host outputs, any NULL). */
rebk_status rebk_sparse_info(rebk_sparse h, double *alpha, double *beta_max, int32_t *row_blocks,
                             int32_t *col_blocks);

/*
 * Self-test of the bounded device-wide waits.  One CTA of a launch waits, with
 * the device-wide barrier and the split-phase wait the sparse kernel uses, for
 * arrivals that never come; each wait gives up after timeout_ns (in [1e3, 1e9])
 * and records REBK_BARRIER_TIMEOUT, and the kernel returns -- nothing faults or
 * traps and the context stays usable.  codes (host, 2): the status of each wait
 * (REBK_BARRIER_TIMEOUT = they gave up as designed); *elapsed_ms (host, may be
 * NULL): device time spent in them.  Returns REBK_BARRIER_TIMEOUT when the waits
 * ran out as designed, REBK_OK if they were somehow satisfied; EINVAL, ENOMEM,
 * ECUDA otherwise.  Synchronises the device.
 */
rebk_status rebk_selftest_waits(int64_t timeout_ns, int32_t *codes, double *elapsed_ms);

/* Device rates measured by rebk_device_peaks. */
typedef struct {
    double fp64_tflops;  /* FP64 FMA rate (2 FLOPs per FMA), best of 3 launches      */
    double fp64_ms;      /* duration of that launch                                   */
    double sm_mhz;       /* SM clock during it (clock64 cycles / global-timer time)   */
    double l2_gbs;       /* L2 read bandwidth (16-byte loads that bypass L1)          */
    double l2_ms;        /* duration of the best L2 launch                            */
    double l2_bytes;     /* size of the buffer read (it fits in L2), read 8 times     */
} rebk_peaks;

/*
 * Measures the two rates the REBK paths are bounded by besides HBM bandwidth:
 * the FP64 FMA rate (the plain FP64 path does one FMA per block element it
 * loads) and the L2 read bandwidth (the sparse path's working set stays in
 * L2).  The paper has no counterpart; the numbers serve as roofline peaks.
 * Kernels run on stream (cudaStream_t, NULL = legacy default) and are timed
 * with CUDA events; the call allocates 48 MiB and synchronises.
 * Errors: EINVAL (out NULL), ENOMEM, ECUDA.
 */
rebk_status rebk_device_peaks(rebk_peaks *out, void *stream);

/* Message for the last failed call on this thread ("" if none). */
const char *rebk_last_error(void);

/* Library version string. */
const char *rebk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* REBK_H */
