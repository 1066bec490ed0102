/*
 * rebk_oracle.c -- plain, slow FP64 CPU reference of the randomized extended
 * block Kaczmarz method (REBK).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the oracle the CUDA solver is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  The solver library never includes, links or calls
 * anything in this directory, and this file shares no code with it.
 *
 * Source: K. Du, W.-T. Si, X.-H. Sun, "Randomized extended block Kaczmarz for
 * solving least squares", arXiv:2001.04179.
 *   - Algorithm 1 (Section 2): the REBK iteration.
 *   - Section 3: contiguous partitions of size tau (the last block may be
 *     shorter), z^0 = b, x^0 = 0.
 *   - Block sampling with probability ||A_{:,J_j}||_F^2 / ||A||_F^2 (column
 *     step) and ||A_{I_i,:}||_F^2 / ||A||_F^2 (row step), Algorithm 1.
 *
 * The paper does not name a random generator.  This oracle uses
 * Philox4x64-10 (J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written from that paper's definition:
 * key (seed, stream), counter (d, 0, 0, 0) where d = 2(k-1) is the column
 * draw and d = 2(k-1)+1 the row draw of iteration k (k = 1, 2, ...).  Word 0
 * of the output block gives u = (word0 >> 11) * 2^-53 in [0, 1); the picked
 * block is the smallest index whose cumulative norm exceeds u * ||A||_F^2.
 *
 * Built with -ffp-contract=off: every product and every sum is rounded on its
 * own, in natural index order, so the result is a fixed reference.  The
 * OpenMP pragmas below only split loops whose iterations write separate
 * outputs (one block column, one row, one column each), so a build with
 * -fopenmp computes every value in the same order as a serial one; they are
 * ignored without -fopenmp (the parity build).
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon et al., SC'11, Section 4.2 and Table 2 constants)    */
/* ------------------------------------------------------------------------ */

static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL; /* multiplier, word 0 */
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL; /* multiplier, word 2 */
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* key bump (golden ratio) */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* key bump (sqrt(3) - 1) */

static void mul_hi_lo(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* One Philox4x64 bijection with 10 rounds.  Round r uses key k_r, where
 * k_0 = key and k_{r+1} = k_r + (W0, W1).  A round maps (x0, x1, x2, x3) to
 * (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)). */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mul_hi_lo(PHILOX_M0, x0, &hi0, &lo0);
        mul_hi_lo(PHILOX_M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform double in [0, 1) for draw number d of stream (seed, stream). */
double orc_uniform(uint64_t seed, uint64_t stream, uint64_t d)
{
    uint64_t ctr[4] = {d, 0, 0, 0};
    uint64_t key[2] = {seed, stream};
    uint64_t out[4];
    orc_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * 0x1.0p-53;
}

/* Block pick for Algorithm 1: the smallest index b with cdf[b] > u * cdf[nb-1].
 * Blocks of zero norm have cdf[b] == cdf[b-1] and are never picked.  If the
 * product rounds up to the total, the last block of nonzero norm is taken. */
int64_t orc_pick(const double *cdf, int64_t nb, double u)
{
    double target = u * cdf[nb - 1];
    for (int64_t b = 0; b < nb; ++b)
        if (cdf[b] > target)
            return b;
    for (int64_t b = nb - 1; b > 0; --b)
        if (cdf[b] > cdf[b - 1])
            return b;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Block norm tables (Algorithm 1 sampling weights)                          */
/* ------------------------------------------------------------------------ */

/* nr[i] = ||A_{I_i,:}||_F^2 and nc[j] = ||A_{:,J_j}||_F^2 for the partitions
 * given by offsets (row_off[0] = 0 < ... < row_off[s] = m, likewise col_off).
 * Both are sums of squares taken in row-major order of A. */
void orc_block_norms(int64_t m, int64_t n, const double *A, int64_t lda,
                     int64_t s, const int64_t *row_off,
                     int64_t t, const int64_t *col_off,
                     double *nr, double *nc)
{
    for (int64_t i = 0; i < s; ++i) nr[i] = 0.0;
    for (int64_t j = 0; j < t; ++j) nc[j] = 0.0;
    int64_t bi = 0;
    for (int64_t r = 0; r < m; ++r) {
        while (r >= row_off[bi + 1]) ++bi;
        int64_t bj = 0;
        for (int64_t c = 0; c < n; ++c) {
            while (c >= col_off[bj + 1]) ++bj;
            double a = A[r * lda + c];
            double a2 = a * a;
            nr[bi] += a2;
            nc[bj] += a2;
        }
    }
    (void)n;
}

/* Inclusive prefix sums, left to right. */
void orc_cdf(const double *w, int64_t nb, double *cdf)
{
    double acc = 0.0;
    for (int64_t b = 0; b < nb; ++b) {
        acc += w[b];
        cdf[b] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1                                                              */
/* ------------------------------------------------------------------------ */

static double rel_err2(int64_t n, const double *x, const double *xref, double *ref2)
{
    double e2 = 0.0, r2 = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double d = x[j] - xref[j];
        e2 += d * d;
        r2 += xref[j] * xref[j];
    }
    *ref2 = r2;
    return e2;
}

/*
 * Runs iterations k = k0+1, ..., k0+max_iter of Algorithm 1 from the state
 * (z, x) it is given (in place):
 *
 *   pick j with probability ||A_{:,J_j}||_F^2 / ||A||_F^2
 *   z <- z - alpha / ||A_{:,J_j}||_F^2 * A_{:,J_j} (A_{:,J_j})^T z
 *   pick i with probability ||A_{I_i,:}||_F^2 / ||A||_F^2
 *   x <- x - alpha / ||A_{I_i,:}||_F^2 * (A_{I_i,:})^T (A_{I_i,:} x - b_{I_i} + z_{I_i})
 *
 * nr/nc are the block norms, cdf_r/cdf_c their prefix sums.  If x_ref is not
 * NULL and check_every > 0, after every check_every-th iteration the run stops
 * once ||x - x_ref||_2 <= tol * ||x_ref||_2 (squared comparison).  idx_out,
 * if not NULL, receives (j_k, i_k) for each iteration run.  Returns the number
 * of iterations run; work[] needs max(tau) doubles (any block size).
 */
int64_t orc_rebk(int64_t m, int64_t n, const double *A, int64_t lda,
                 int64_t s, const int64_t *row_off, int64_t t, const int64_t *col_off,
                 const double *nr, const double *nc,
                 const double *cdf_r, const double *cdf_c,
                 double alpha, uint64_t seed, uint64_t stream, int64_t k0,
                 const double *b, double *z, double *x,
                 int64_t max_iter, int64_t check_every,
                 const double *x_ref, double tol,
                 int32_t *idx_out, double *work)
{
    (void)m;
    for (int64_t it = 1; it <= max_iter; ++it) {
        uint64_t k = (uint64_t)(k0 + it);

        /* column step on z */
        int64_t j = orc_pick(cdf_c, t, orc_uniform(seed, stream, 2 * (k - 1)));
        int64_t c0 = col_off[j], c1 = col_off[j + 1];
        double cJ = alpha / nc[j];
        double *w = work;
#pragma omp parallel for schedule(static)
        for (int64_t l = c0; l < c1; ++l) {
            double acc = 0.0;
            for (int64_t r = 0; r < m; ++r)
                acc += A[r * lda + l] * z[r];
            w[l - c0] = acc;
        }
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < m; ++r) {
            double acc = 0.0;
            for (int64_t l = c0; l < c1; ++l)
                acc += A[r * lda + l] * w[l - c0];
            z[r] -= cJ * acc;
        }

        /* row step on x, with the updated z */
        int64_t i = orc_pick(cdf_r, s, orc_uniform(seed, stream, 2 * (k - 1) + 1));
        int64_t r0 = row_off[i], r1 = row_off[i + 1];
        double cI = alpha / nr[i];
        double *res = work;
#pragma omp parallel for schedule(static)
        for (int64_t l = r0; l < r1; ++l) {
            double acc = 0.0;
            for (int64_t c = 0; c < n; ++c)
                acc += A[l * lda + c] * x[c];
            res[l - r0] = acc - b[l] + z[l];
        }
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < n; ++c) {
            double acc = 0.0;
            for (int64_t l = r0; l < r1; ++l)
                acc += A[l * lda + c] * res[l - r0];
            x[c] -= cI * acc;
        }

        if (idx_out) {
            idx_out[2 * (it - 1)] = (int32_t)j;
            idx_out[2 * (it - 1) + 1] = (int32_t)i;
        }
        if (x_ref && check_every > 0 && it % check_every == 0) {
            double ref2;
            double e2 = rel_err2(n, x, x_ref, &ref2);
            if (e2 <= tol * tol * ref2)
                return it;
        }
    }
    return max_iter;
}

/*
 * Algorithm 1 written on corrections, for iterative refinement.
 *
 * Running Algorithm 1 from the state (x + dx, z + dz) with the same blocks is,
 * in exact arithmetic, the same as updating the corrections
 *
 *   dz <- dz - cJ * A_J (A_J^T dz + g_J),            g = A^T z
 *   dx <- dx - cI * A_I^T (A_I dx - f_I + dz_I),     f = b - z - A x
 *
 * with (x, z) held fixed.  The dual sums s (length n) and v (length m) record
 * the same steps, so that dz = -A s and dx = A^T v:
 *
 *   s_J += cJ * (A_J^T dz + g_J),      v_I -= cI * (A_I dx - f_I + dz_I).
 *
 * Alo holds the matrix the corrections are computed with (the reduced-
 * precision copy, as FP64 values); cJ and cI use the block norms nr/nc given.
 * dz, dx, s, v are updated in place.  If x_ref is not NULL and check_every > 0
 * the run stops once ||xbase + dx - x_ref||_2 <= err_abs after a check.
 * Returns the number of iterations run.
 */
int64_t orc_rebk_correction(int64_t m, int64_t n, const double *Alo, int64_t lda,
                            int64_t s_blocks, const int64_t *row_off,
                            int64_t t_blocks, const int64_t *col_off,
                            const double *nr, const double *nc,
                            const double *cdf_r, const double *cdf_c,
                            double alpha, uint64_t seed, uint64_t stream, int64_t k0,
                            const double *f, const double *g,
                            double *dz, double *dx, double *s, double *v,
                            int64_t max_iter, int64_t check_every,
                            const double *xbase, const double *x_ref, double err_abs,
                            int32_t *idx_out, double *work)
{
    for (int64_t it = 1; it <= max_iter; ++it) {
        uint64_t k = (uint64_t)(k0 + it);

        int64_t j = orc_pick(cdf_c, t_blocks, orc_uniform(seed, stream, 2 * (k - 1)));
        int64_t c0 = col_off[j], c1 = col_off[j + 1];
        double cJ = alpha / nc[j];
        double *w = work;
        for (int64_t l = c0; l < c1; ++l) {
            double acc = 0.0;
            for (int64_t r = 0; r < m; ++r)
                acc += Alo[r * lda + l] * dz[r];
            w[l - c0] = acc + g[l];
        }
        for (int64_t r = 0; r < m; ++r) {
            double acc = 0.0;
            for (int64_t l = c0; l < c1; ++l)
                acc += Alo[r * lda + l] * w[l - c0];
            dz[r] -= cJ * acc;
        }
        for (int64_t l = c0; l < c1; ++l)
            s[l] += cJ * w[l - c0];

        int64_t i = orc_pick(cdf_r, s_blocks, orc_uniform(seed, stream, 2 * (k - 1) + 1));
        int64_t r0 = row_off[i], r1 = row_off[i + 1];
        double cI = alpha / nr[i];
        double *res = work;
        for (int64_t l = r0; l < r1; ++l) {
            double acc = 0.0;
            for (int64_t c = 0; c < n; ++c)
                acc += Alo[l * lda + c] * dx[c];
            res[l - r0] = acc - f[l] + dz[l];
        }
        for (int64_t c = 0; c < n; ++c) {
            double acc = 0.0;
            for (int64_t l = r0; l < r1; ++l)
                acc += Alo[l * lda + c] * res[l - r0];
            dx[c] -= cI * acc;
        }
        for (int64_t l = r0; l < r1; ++l)
            v[l] -= cI * res[l - r0];

        if (idx_out) {
            idx_out[2 * (it - 1)] = (int32_t)j;
            idx_out[2 * (it - 1) + 1] = (int32_t)i;
        }
        if (x_ref && check_every > 0 && it % check_every == 0) {
            double e2 = 0.0;
            for (int64_t c = 0; c < n; ++c) {
                double d = (xbase ? xbase[c] : 0.0) + dx[c] - x_ref[c];
                e2 += d * d;
            }
            if (e2 <= err_abs * err_abs)
                return it;
        }
    }
    return max_iter;
}

/* ------------------------------------------------------------------------ */
/* Sampling without partitions (a reading of Section 4's variants)          */
/* ------------------------------------------------------------------------ */

/* Uniform double in [0, 1) for slot q of draw number d: Philox counter
 * (d, q, 0, 0), key (seed, stream), word 0.  Slot 0 is orc_uniform's draw. */
double orc_uniform_slot(uint64_t seed, uint64_t stream, uint64_t d, uint64_t q)
{
    uint64_t ctr[4] = {d, q, 0, 0};
    uint64_t key[2] = {seed, stream};
    uint64_t out[4];
    orc_philox4x64_10(ctr, key, out);
    return (double)(out[0] >> 11) * 0x1.0p-53;
}

/*
 * Algorithm 1 with index sets drawn without a partition.  Section 4 names
 * variants of REBK whose random samplings do not depend on partitions; the
 * reading taken here: iteration k draws tau_c column indices j_1..j_{tau_c}
 * independently, each with probability ||A_{:,j}||^2 / ||A||_F^2 (slot q of
 * column draw 2(k-1)), and tau_r row indices i_1..i_{tau_r} independently with
 * probability ||A_{i,:}||^2 / ||A||_F^2 (slot q of row draw 2(k-1)+1).  A_J is
 * the m x tau_c matrix of the drawn columns in draw order (a column drawn
 * twice appears twice) and A_I the tau_r x n matrix of the drawn rows; the
 * step is Algorithm 1's with these matrices:
 *
 *   z <- z - alpha / ||A_J||_F^2 * A_J A_J^T z
 *   x <- x - alpha / ||A_I||_F^2 * A_I^T (A_I x - b_I + z_I)
 *
 * with ||A_J||_F^2 = sum_q ||A_{:,j_q}||^2 (in draw order), likewise for I.
 * (This is RABK's step with weights ||a_i||^2 / ||A_I||_F^2 over the drawn
 * set.)  With tau_r = tau_c = 1 it is the randomized extended Kaczmarz
 * method.  cn / rn: squared column / row norms; cdf_c / cdf_r: their inclusive
 * prefix sums.  idx_out (optional): tau_c + tau_r entries per iteration, the
 * column draws then the row draws.  work: tau_c + tau_r doubles.  Stopping as
 * orc_rebk.  Returns the number of iterations run.
 */
int64_t orc_rebk_free(int64_t m, int64_t n, const double *A, int64_t lda,
                      const double *rn, const double *cn,
                      const double *cdf_r, const double *cdf_c,
                      int64_t tau_r, int64_t tau_c,
                      double alpha, uint64_t seed, uint64_t stream, int64_t k0,
                      const double *b, double *z, double *x,
                      int64_t max_iter, int64_t check_every,
                      const double *x_ref, double tol,
                      int32_t *idx_out, int64_t *jset, int64_t *iset, double *work)
{
    for (int64_t it = 1; it <= max_iter; ++it) {
        uint64_t k = (uint64_t)(k0 + it);

        /* column step on z */
        double fJ = 0.0;
        for (int64_t q = 0; q < tau_c; ++q) {
            jset[q] = orc_pick(cdf_c, n, orc_uniform_slot(seed, stream, 2 * (k - 1), (uint64_t)q));
            fJ += cn[jset[q]];
        }
        double cJ = alpha / fJ;
        double *w = work;
        for (int64_t q = 0; q < tau_c; ++q) {
            double acc = 0.0;
            for (int64_t r = 0; r < m; ++r)
                acc += A[r * lda + jset[q]] * z[r];
            w[q] = acc;
        }
        for (int64_t r = 0; r < m; ++r) {
            double acc = 0.0;
            for (int64_t q = 0; q < tau_c; ++q)
                acc += A[r * lda + jset[q]] * w[q];
            z[r] -= cJ * acc;
        }

        /* row step on x, with the updated z */
        double fI = 0.0;
        for (int64_t q = 0; q < tau_r; ++q) {
            iset[q] = orc_pick(cdf_r, m, orc_uniform_slot(seed, stream, 2 * (k - 1) + 1, (uint64_t)q));
            fI += rn[iset[q]];
        }
        double cI = alpha / fI;
        double *res = work + tau_c;
        for (int64_t q = 0; q < tau_r; ++q) {
            int64_t l = iset[q];
            double acc = 0.0;
            for (int64_t c = 0; c < n; ++c)
                acc += A[l * lda + c] * x[c];
            res[q] = acc - b[l] + z[l];
        }
        for (int64_t c = 0; c < n; ++c) {
            double acc = 0.0;
            for (int64_t q = 0; q < tau_r; ++q)
                acc += A[iset[q] * lda + c] * res[q];
            x[c] -= cI * acc;
        }

        if (idx_out) {
            int32_t *row = idx_out + (it - 1) * (tau_c + tau_r);
            for (int64_t q = 0; q < tau_c; ++q) row[q] = (int32_t)jset[q];
            for (int64_t q = 0; q < tau_r; ++q) row[tau_c + q] = (int32_t)iset[q];
        }
        if (x_ref && check_every > 0 && it % check_every == 0) {
            double ref2;
            double e2 = rel_err2(n, x, x_ref, &ref2);
            if (e2 <= tol * tol * ref2)
                return it;
        }
    }
    return max_iter;
}
