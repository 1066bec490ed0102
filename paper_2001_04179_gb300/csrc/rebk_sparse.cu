// rebk_sparse.cu -- Algorithm 1 of Du, Si, Sun (arXiv:2001.04179) on a sparse
// matrix: CSR for the row blocks, a CSC copy for the column blocks.
//
// One persistent cooperative launch runs many iterations, one device-wide
// barrier each.  x and z have two copies each: at iteration k one copy of x holds
// x^{k-1} and the other x^{k-2}, one copy of z holds z^k and the other z^{k-1}.
// With the block indices sampled before the launch (as in the dense path),
// iteration k is one phase:
//   gathers from the current copies: r^k = A_{I_k,:} x^{k-1} - b_{I_k} + z^k_{I_k}
//     over CSR, the column gather of the next iteration w = A_{:,J_{k+1}}^T z^k
//     over CSC, and every check_every iterations each CTA's share of
//     ||x^{k-1} - x_ref||^2;
//   scatters into the other copies, by FP64 atomic adds: -c_I A_{I_k,:}^T r^k and
//     again the previous iteration's -c_I' A_{I_{k-1},:}^T r^{k-1} into x (which
//     turns x^{k-2} into x^k), -c_J A_{:,J_{k+1}} w^{k+1} and again -c_J'
//     A_{:,J_k} w^k into z (z^{k-1} into z^{k+1});                      barrier
// so no copy is read and written in the same phase.  Each update is added twice,
// once into each copy, in exchange for the second barrier per iteration.  (z^1
// comes from a prologue gather / scatter.)  Each CTA owns a contiguous share of
// the sampled block's columns (rows), whose entries are one CSC (CSR) range: its
// threads gather it in one round, warps adding each line's products by shuffles
// before one shared atomic per line; it keeps its lines' r and w, and their entry
// ranges, for the replay of the next iteration.  On a converged stop at iteration
// k, x = x^{k-1} and z = z^k; the final iterates are copied into x and z (the
// first copies) before the kernel ends.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "rebk.h"
#include "rebk_device.cuh"
#include "rebk_internal.h"

namespace rebk {
namespace {

constexpr int kST = 512;                     // threads per CTA
constexpr int kSW = kST / 32;
constexpr int kOwnMax = 512;                 // columns / rows of a block one CTA may own
constexpr int64_t kSparseChunk = 1 << 20;    // iterations sampled per launch
constexpr int64_t kSparseLaunchMax = 4000000;  // barrier counter headroom (one barrier per iteration)

struct SparseArgs {
    int64_t m, n;
    int tau_r, tau_c;
    const int64_t *rp;   // CSR row pointers (m + 1)
    const int32_t *ci;   // CSR column indices
    const void *rv;      // CSR values (T)
    const int64_t *cp;   // CSC column pointers (n + 1)
    const int32_t *ri;   // CSC row indices
    const void *cv;      // CSC values (T)
    const void *coef_r, *coef_c;  // T: alpha / ||block||_F^2 (0 for zero blocks)
    const int32_t *idx;  // 2 * iters: (j_k, i_k)
    int64_t iters;
    void *z, *x;         // T: z and x (plain), the corrections dz and dx (CORR)
    void *z2, *x2;       // T: second copies, equal to z and x at launch
    const double *b;     // b (plain), f = b - z - A x (CORR)
    const double *g;     // CORR: A^T z
    void *sdual, *vdual; // CORR (T): duals s (n) and v (m), dz = -A s, dx = A^T v
    const double *x_ref;  // NULL = no test
    const double *x_base; // CORR: the test uses x_base + dx
    double tol2_abs;
    int64_t check_every, check_offset;
    double *acc;          // [3] rotating error accumulators, zeroed before launch
    int *bad;             // non-finite reduction seen, zeroed before launch
    unsigned int *bar;
    int *status;
    int64_t *iters_done;
    unsigned long long timeout_ns;
};

__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    __syncthreads();  // red free (its last readers are past this point)
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kSW; ++w) t += red[w];
    return t;
}

// Line of entry e among the CTA's nq lines: bnd[q] <= e < bnd[q + 1].
__device__ __forceinline__ int line_of(const int64_t *bnd, int nq, int64_t e) {
    int lo = 0, hi = nq;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bnd[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

// part[q] = sum over the entries e of line q of val[e] * vec[idx[e]], for the CTA's
// contiguous lines (entries bnd[0] .. bnd[nq]).  Each round, warp w takes 32
// consecutive entries (sorted by line, so they span one line or a few); the warp
// adds each line's products with a shuffle sum and one lane adds that to part[].
template <typename T>
__device__ __forceinline__ void gather_lines(const int64_t *bnd, int nq, const int32_t *__restrict__ idx,
                                             const T *__restrict__ val, const T *vec, T *part) {
    for (int q = threadIdx.x; q < nq; q += kST) part[q] = T(0);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t base = bnd[0]; base < bnd[nq]; base += kST) {  // uniform over the CTA
        const int64_t e = base + threadIdx.x;
        const bool in = e < bnd[nq];
        int q = 0x7fffffff;
        T prod = T(0);
        if (in) {
            q = line_of(bnd, nq, e);
            prod = val[e] * vec[idx[e]];
        }
        const int qlo = __reduce_min_sync(0xffffffffu, q);
        const int qhi = __reduce_max_sync(0xffffffffu, in ? q : -1);
        for (int qq = qlo; qq <= qhi; ++qq) {  // warp-uniform bounds
            const T t = warp_sum(in && q == qq ? prod : T(0));
            if (lane == 0) atomicAdd(part + qq, t);
        }
    }
    __syncthreads();
}

// One entry of an iteration's joint list, kept in registers from the gather
// phase for the scatter phase: its line (rows first, then columns; -1 = none),
// its index into the other dimension and its value.
template <typename T> struct Entry {
    int q;
    int32_t idx;
    T val;
};

// Both gathers of an iteration in one pass: the CTA's rows (CSR entries br[0] ..
// br[nqr], against x) and columns (CSC entries bc[0] .. bc[nqc], against z) as one
// list of nqr + nqc lines; part[q] gets line q's sum (rows first).  Each thread
// takes two entries per round so that both loads and both gathers are in flight;
// the entries of the first round are returned in f0, f1 (entries tid and
// kST + tid of the list) for the scatters.
template <typename T>
__device__ __forceinline__ void gather_rows_cols(const int64_t *br, int nqr, const int32_t *__restrict__ ci,
                                                 const T *__restrict__ rv, const T *x, const int64_t *bc,
                                                 int nqc, const int32_t *__restrict__ ri,
                                                 const T *__restrict__ cv, const T *z, T *part, Entry<T> &f0,
                                                 Entry<T> &f1) {
    const int nl = nqr + nqc;
    for (int q = threadIdx.x; q < nl; q += kST) part[q] = T(0);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nr = nqr > 0 ? br[nqr] - br[0] : 0, nc = nqc > 0 ? bc[nqc] - bc[0] : 0, tot = nr + nc;
    auto entry = [&](int64_t g, Entry<T> &f, T *prod) {  // entry g of the joint list
        if (g >= tot) {
            f.q = -1;
            f.idx = 0;
            f.val = T(0);
            *prod = T(0);
        } else if (g < nr) {
            const int64_t e = br[0] + g;
            f.q = line_of(br, nqr, e);
            f.idx = ci[e];
            f.val = rv[e];
            *prod = f.val * x[f.idx];
        } else {
            const int64_t e = bc[0] + (g - nr);
            f.q = nqr + line_of(bc, nqc, e);
            f.idx = ri[e];
            f.val = cv[e];
            *prod = f.val * z[f.idx];
        }
    };
    auto add_lines = [&](int q, T prod) {  // per warp: one shuffle sum and one atomic per line
        const int qlo = __reduce_min_sync(0xffffffffu, q >= 0 ? q : 0x7fffffff);
        const int qhi = __reduce_max_sync(0xffffffffu, q);
        for (int qq = qlo; qq <= qhi; ++qq) {
            const T t = warp_sum(q == qq ? prod : T(0));
            if (lane == 0) atomicAdd(part + qq, t);
        }
    };
    for (int64_t base = 0; base < tot; base += 2 * kST) {  // uniform over the CTA
        Entry<T> e0, e1;
        T p0, p1;
        entry(base + threadIdx.x, e0, &p0);
        entry(base + kST + threadIdx.x, e1, &p1);
        add_lines(e0.q, p0);
        add_lines(e1.q, p1);
        if (base == 0) {
            f0 = e0;
            f1 = e1;
        }
    }
    if (tot == 0) f0.q = f1.q = -1;
    __syncthreads();
}

// T = double, CORR = false: Algorithm 1 in FP64 on (z, x).
// T = float, CORR = true: the same iteration on the corrections (dz, dx) with the
// FP32 copies of the values and FP32 arithmetic, the residuals f = b - z - A x and
// g = A^T z held fixed in FP64 (see rebk_solve_refined):
//   w = A_J^T dz + g_J,  dz <- dz - c_J A_J w,  s_J += c_J w
//   r = A_I dx - f_I + dz_I,  dx <- dx - c_I A_I^T r,  v_I -= c_I r.
// The duals are updated in the scatter phase, so a stop after the gathers of
// iteration k leaves (dx, dz, s, v) consistent: dz = -A s and dx = A^T v.
template <typename T, bool CORR>
__global__ void __launch_bounds__(kST, 1) rebk_sparse_kernel(const __grid_constant__ SparseArgs a) {
    __shared__ double red[kSW];
    // two slots each, by iteration parity: w of the CTA's columns of J_u (slot u & 1),
    // r of its rows of I_u (slot u & 1), and those lines' entry boundaries
    __shared__ T wq[2][kOwnMax];
    __shared__ T rq[2][kOwnMax];
    __shared__ int64_t bc[2][kOwnMax + 1];
    __shared__ int64_t br[2][kOwnMax + 1];
    __shared__ T part[2 * kOwnMax];         // the joint gather's line sums
    __shared__ int s_flag;
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
    const T *rv = static_cast<const T *>(a.rv), *cv = static_cast<const T *>(a.cv);
    const T *coef_r = static_cast<const T *>(a.coef_r), *coef_c = static_cast<const T *>(a.coef_c);
    T *const x0 = static_cast<T *>(a.x), *const x1 = static_cast<T *>(a.x2);
    T *const z0 = static_cast<T *>(a.z), *const z1 = static_cast<T *>(a.z2);
    auto xb = [&](int64_t u) { return (u & 1) ? x1 : x0; };
    auto zb = [&](int64_t u) { return (u & 1) ? z1 : z0; };
    T *sdual = static_cast<T *>(a.sdual), *vdual = static_cast<T *>(a.vdual);
    const int64_t K = a.iters;
    const bool check = a.x_ref != nullptr && a.check_every > 0;
    const int64_t xs0 = a.n * cta / G, xs1 = a.n * (cta + 1) / G;  // this CTA's share of x
    const int64_t zs0 = a.m * cta / G, zs1 = a.m * (cta + 1) / G;  // and of z
    unsigned int phase = 0;
    auto barrier = [&]() -> bool {
        ++phase;
        return grid_barrier(a.bar, (unsigned)G * phase, a.status, a.timeout_ns, &s_flag);
    };
    // -c A^T r (rows, into x) or -c A w (columns, into z) for a CTA's lines, all entries
    // reloaded from the matrix
    auto scatter_rows = [&](T *dst, const int64_t *b, int nq, const T *rr, T c) {
        for (int64_t e = (nq > 0 ? b[0] : 0) + tid; nq > 0 && e < b[nq]; e += kST)
            atomicAdd(dst + a.ci[e], -c * rv[e] * rr[line_of(b, nq, e)]);
    };
    auto scatter_cols = [&](T *dst, const int64_t *b, int nq, const T *ww, T c) {
        for (int64_t e = (nq > 0 ? b[0] : 0) + tid; nq > 0 && e < b[nq]; e += kST)
            atomicAdd(dst + a.ri[e], -c * cv[e] * ww[line_of(b, nq, e)]);
    };
    int64_t done = K;
    int stop = 0;
    bool z_from_first = false;  // the prologue stopped: z^0 is in the first copy
    // the previous iteration's lines, for the replays: rows of I_{k-1}, columns of J_k
    int64_t lp0 = 0, cp0 = 0;
    int nqrp = 0, nqcp = 0;
    T cIp = T(0), cJp = T(0);
    // prologue: w^1 from z^0 (first copy), -c A w^1 into the second copy (z^1)
    if (K >= 1) {
        const int j = __ldg(a.idx);
        const int64_t ja = (int64_t)j * a.tau_c, jb = ja + a.tau_c < a.n ? ja + a.tau_c : a.n;
        cp0 = ja + (jb - ja) * cta / G;
        nqcp = (int)(ja + (jb - ja) * (cta + 1) / G - cp0);
        cJp = coef_c[j];
        for (int q = tid; q <= nqcp; q += kST) bc[1][q] = a.cp[cp0 + q];
        __syncthreads();
        if (nqcp > 0) gather_lines(bc[1], nqcp, a.ri, cv, z0, wq[1]);
        if (CORR)
            for (int q = tid; q < nqcp; q += kST) wq[1][q] += (T)a.g[cp0 + q];
        if (tid < nqcp && !isfinite(wq[1][tid])) atomicExch(a.bad, 1);
        __syncthreads();
        scatter_cols(z1, bc[1], nqcp, wq[1], cJp);
        if (!barrier()) return;
        if (*reinterpret_cast<volatile int *>(a.bad) != 0) {
            stop = 5;
            done = 0;
            z_from_first = true;
        }
    }
    // Block boundaries and b of the rows for the next iteration, loaded during the
    // previous phase (they do not change) so that a phase starts with its line
    // ranges in place.
    int64_t nb_r[2] = {0, 0}, nb_c[2] = {0, 0};
    double nb_b = 0.0;
    bool have_next = false;
    auto shares = [&](int64_t kk, int64_t *l0, int *nqr, int64_t *c0, int *nq_c) {
        const int i = __ldg(a.idx + 2 * (kk - 1) + 1);
        const int64_t ia = (int64_t)i * a.tau_r, ib = ia + a.tau_r < a.m ? ia + a.tau_r : a.m;
        *l0 = ia + (ib - ia) * cta / G;
        *nqr = (int)(ia + (ib - ia) * (cta + 1) / G - *l0);
        *c0 = 0;
        *nq_c = 0;
        if (kk < K) {  // the column share of J_{kk+1} (none after the last iteration)
            const int j = __ldg(a.idx + 2 * kk);
            const int64_t ja = (int64_t)j * a.tau_c, jb = ja + a.tau_c < a.n ? ja + a.tau_c : a.n;
            *c0 = ja + (jb - ja) * cta / G;
            *nq_c = (int)(ja + (jb - ja) * (cta + 1) / G - *c0);
        }
    };
    int64_t l0 = 0;
    int nqr = 0;
    T cI = T(0);
    for (int64_t k = 1; stop == 0 && k <= K; ++k) {
        const int sk = (int)(k & 1), sn = (int)((k + 1) & 1);  // slots of I_k / J_k and of J_{k+1}
        int64_t c0;
        int nqc;
        shares(k, &l0, &nqr, &c0, &nqc);
        cI = coef_r[__ldg(a.idx + 2 * (k - 1) + 1)];
        const T cJ = nqc > 0 ? coef_c[__ldg(a.idx + 2 * k)] : T(0);
        if (have_next) {  // nqr, nqc <= kOwnMax = kST: entries tid and kST + tid
            if (tid <= nqr) br[sk][tid] = nb_r[0];
            if (kST + tid <= nqr) br[sk][kST + tid] = nb_r[1];
            if (tid <= nqc) bc[sn][tid] = nb_c[0];
            if (kST + tid <= nqc) bc[sn][kST + tid] = nb_c[1];
        } else {
            for (int q = tid; q <= nqr; q += kST) br[sk][q] = a.rp[l0 + q];
            for (int q = tid; q <= nqc; q += kST) bc[sn][q] = a.cp[c0 + q];
            nb_b = tid < nqr ? a.b[l0 + tid] : 0.0;
        }
        __syncthreads();
        // ---- gathers from x^{k-1} and z^k: r^k, w^{k+1}, test of x^{k-1} ----
        const T *xc = xb(k - 1), *zc = zb(k);
        Entry<T> f0, f1;
        gather_rows_cols(br[sk], nqr, a.ci, rv, xc, bc[sn], nqc, a.ri, cv, zc, part, f0, f1);
        if (tid < nqr) {
            const T rl = part[tid] - (T)nb_b + zc[l0 + tid];
            rq[sk][tid] = rl;
            if (!isfinite(rl)) atomicExch(a.bad, 1);
        }
        for (int q = tid; q < nqc; q += kST) {
            wq[sn][q] = CORR ? part[nqr + q] + (T)a.g[c0 + q] : part[nqr + q];
            if (!isfinite(wq[sn][q])) atomicExch(a.bad, 1);
        }
        const bool due = check && k >= 2 && (a.check_offset + k - 1) % a.check_every == 0;
        if (due) {
            double e2 = 0.0;
            for (int64_t c = xs0 + tid; c < xs1; c += kST) {
                const double xv = CORR ? a.x_base[c] + (double)xc[c] : (double)xc[c];
                const double d = xv - a.x_ref[c];
                e2 = fma(d, d, e2);
            }
            e2 = block_sum(e2, red);
            if (tid == 0) atomicAdd(a.acc + k % 3, e2);
        }
        if (cta == 0 && tid == 0) a.acc[(k + 1) % 3] = 0.0;  // the slot two tests ahead
        __syncthreads();  // rq, wq complete
        // ---- scatters into the other copies: x^{k-2} -> x^k, z^{k-1} -> z^{k+1} ----
        T *xo = xb(k), *zo = zb(k + 1);
        // the first round's entries of this iteration from registers, the rest reloaded
        auto scatter = [&](const Entry<T> &f) {
            if (f.q < 0) return;
            if (f.q < nqr) atomicAdd(xo + f.idx, -cI * f.val * rq[sk][f.q]);
            else atomicAdd(zo + f.idx, -cJ * f.val * wq[sn][f.q - nqr]);
        };
        scatter(f0);
        scatter(f1);
        {
            const int64_t nr = nqr > 0 ? br[sk][nqr] - br[sk][0] : 0, nc = nqc > 0 ? bc[sn][nqc] - bc[sn][0] : 0;
            for (int64_t g = 2 * kST + tid; g < nr + nc; g += kST) {
                if (g < nr) {
                    const int64_t e = br[sk][0] + g;
                    atomicAdd(xo + a.ci[e], -cI * rv[e] * rq[sk][line_of(br[sk], nqr, e)]);
                } else {
                    const int64_t e = bc[sn][0] + (g - nr);
                    atomicAdd(zo + a.ri[e], -cJ * cv[e] * wq[sn][line_of(bc[sn], nqc, e)]);
                }
            }
        }
        // the previous iteration's updates again: r^{k-1} into x, w^k into z
        if (k >= 2) scatter_rows(xo, br[sn], nqrp, rq[sn], cIp);
        scatter_cols(zo, bc[sk], nqcp, wq[sk], cJp);
        if (CORR) {  // duals one iteration behind, so that a stop leaves them consistent
            if (k >= 2 && tid < nqrp) vdual[lp0 + tid] -= cIp * rq[sn][tid];
            for (int q = tid; q < nqcp; q += kST) sdual[cp0 + q] += cJp * wq[sk][q];
        }
        // boundaries and b of iteration k + 1 (read-only arrays)
        have_next = k < K;
        if (have_next) {
            int64_t l0n, c0n;
            int nqrn, nqcn;
            shares(k + 1, &l0n, &nqrn, &c0n, &nqcn);
            nb_r[0] = tid <= nqrn ? a.rp[l0n + tid] : 0;
            nb_r[1] = kST + tid <= nqrn ? a.rp[l0n + kST + tid] : 0;
            nb_c[0] = tid <= nqcn ? a.cp[c0n + tid] : 0;
            nb_c[1] = kST + tid <= nqcn ? a.cp[c0n + kST + tid] : 0;
            nb_b = tid < nqrn ? a.b[l0n + tid] : 0.0;
        }
        lp0 = l0;
        nqrp = nqr;
        cIp = cI;
        cp0 = c0;
        nqcp = nqc;
        cJp = cJ;
        if (!barrier()) return;
        if (*reinterpret_cast<volatile int *>(a.bad) != 0) {
            stop = 5;
            done = k - 1;
            break;
        }
        if (due && __ldcg(a.acc + k % 3) <= a.tol2_abs) {  // every CTA reads the same sum
            stop = 1;
            done = k - 1;
            break;
        }
    }
    if (CORR && stop == 0 && K >= 1) {  // the last iteration's r into v
        const int sl = (int)(K & 1);
        if (tid < nqr) vdual[l0 + tid] -= cI * rq[sl][tid];
    }
    // x^done and z^(done+1) (z^K after K iterations, z^0 after a prologue stop) into the
    // first copies; every CTA has passed the last barrier, so no phase is running
    if (K >= 1) {
        const T *xf = xb(done);
        const T *zf = z_from_first ? z0 : (stop == 0 ? zb(K) : zb(done + 1));
        if (xf != x0)
            for (int64_t c = xs0 + tid; c < xs1; c += kST) x0[c] = xf[c];
        if (zf != z0)
            for (int64_t r = zs0 + tid; r < zs1; r += kST) z0[r] = zf[r];
    }
    if (cta == 0 && tid == 0) {
        *a.iters_done = done;
        if (stop == 5) atomicExch(a.status, 5);
    }
}

// y[l] = sum over line l's entries of val[e] * p[idx[e]] (one warp per line; FP64
// products of the FP64 values with an FP64 or FP32 vector): A p over CSR, A^T q over CSC.
template <typename TP>
__global__ void sparse_lines_kernel(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                    const double *__restrict__ val, const TP *__restrict__ p, int64_t lines,
                                    double *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t l = blockIdx.x * wpb + (threadIdx.x >> 5); l < lines; l += (int64_t)gridDim.x * wpb) {
        double s = 0.0;
        for (int64_t e = ptr[l] + lane; e < ptr[l + 1]; e += 32) s = fma(val[e], (double)p[idx[e]], s);
        s = warp_sum(s);
        if (lane == 0) y[l] = s;
    }
}

template <typename TP>
cudaError_t sparse_lines(const int64_t *ptr, const int32_t *idx, const double *val, const TP *p, int64_t lines,
                         double *y, cudaStream_t st) {
    int64_t blocks = (lines + 7) / 8;
    if (blocks > 4096) blocks = 4096;
    sparse_lines_kernel<TP><<<(unsigned)blocks, 256, 0, st>>>(ptr, idx, val, p, lines, y);
    return cudaGetLastError();
}

// Host-side power iterations (FP64) for the spectral norms of the blocks.
double block_spectral_sq(const std::vector<int64_t> &ptr, const std::vector<int32_t> &idx,
                         const std::vector<double> &val, int64_t l0, int64_t l1, int64_t other, int iters) {
    // ||B||_2^2 for B = the lines l0..l1-1 of the compressed matrix (rows of CSR or
    // columns of CSC) by power iterations on B^T B; entries index the other dimension.
    std::vector<int32_t> cols;
    for (int64_t l = l0; l < l1; ++l)
        for (int64_t e = ptr[l]; e < ptr[l + 1]; ++e) cols.push_back(idx[e]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    if (cols.empty()) return 0.0;
    std::vector<int32_t> pos;  // entry -> position in cols
    pos.reserve(ptr[l1] - ptr[l0]);
    for (int64_t e = ptr[l0]; e < ptr[l1]; ++e)
        pos.push_back((int32_t)(std::lower_bound(cols.begin(), cols.end(), idx[e]) - cols.begin()));
    (void)other;
    const int64_t nc = (int64_t)cols.size(), nl = l1 - l0;
    std::vector<double> v(nc), u(nl), w(nc);
    for (int64_t c = 0; c < nc; ++c) v[c] = 1.0 + 0.5 * std::sin(0.37 * (double)(c + 1));  // fixed start
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
        double nv = 0.0;
        for (double t : v) nv += t * t;
        nv = std::sqrt(nv);
        if (nv == 0.0) return 0.0;
        for (double &t : v) t /= nv;
        for (int64_t l = 0; l < nl; ++l) {
            double s = 0.0;
            for (int64_t e = ptr[l0 + l]; e < ptr[l0 + l + 1]; ++e) s += val[e] * v[pos[e - ptr[l0]]];
            u[l] = s;
        }
        std::fill(w.begin(), w.end(), 0.0);
        for (int64_t l = 0; l < nl; ++l)
            for (int64_t e = ptr[l0 + l]; e < ptr[l0 + l + 1]; ++e) w[pos[e - ptr[l0]]] += val[e] * u[l];
        double rq = 0.0;
        for (int64_t c = 0; c < nc; ++c) rq += v[c] * w[c];
        lam = rq;
        v.swap(w);
    }
    return lam;
}

}  // namespace
}  // namespace rebk

using namespace rebk;

struct rebk_sparse_s {
    int64_t m = 0, n = 0, nnz = 0;
    int tau_r = 1, tau_c = 1, s = 0, t = 0, fb_r = 0, fb_c = 0;
    double alpha = 0.0, beta = 0.0, fro2 = 0.0;
    int G = 0, check_every = 10;
    cudaStream_t stream = nullptr;
    int64_t *rp = nullptr, *cp = nullptr;
    int32_t *ci = nullptr, *ri = nullptr, *idx = nullptr;
    double *rv = nullptr, *cv = nullptr, *cdf_r = nullptr, *cdf_c = nullptr, *coef_r = nullptr, *coef_c = nullptr;
    double *zbuf = nullptr, *acc = nullptr, *small = nullptr;
    float *rv32 = nullptr, *cv32 = nullptr, *coef_r32 = nullptr, *coef_c32 = nullptr;  // mixed precision
    double *f = nullptr, *g = nullptr, *ym = nullptr, *yn = nullptr;                 // FP64 residuals
    float *dz = nullptr, *dx = nullptr, *sd = nullptr, *vd = nullptr;                // corrections, duals
    void *copy2 = nullptr;  // the kernel's second copies of x and z (8 (m + n) + 256 bytes)
    int *bad = nullptr, *status = nullptr;
    unsigned int *bar = nullptr;
    int64_t *iters_done = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, k0 = nullptr, k1 = nullptr;
};

namespace {

rebk_status sfail(rebk_status s, const std::string &msg) {
    set_last_error(msg);
    return s;
}

#define SCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess) return sfail(e__ == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA, \
                                             std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

void free_sparse(rebk_sparse h) {
    if (!h) return;
    void *p[] = {h->rp, h->cp, h->ci, h->ri, h->idx, h->rv, h->cv, h->cdf_r, h->cdf_c, h->coef_r, h->coef_c,
                 h->zbuf, h->acc, h->small, h->bad, h->status, h->bar, h->iters_done, h->rv32, h->cv32,
                 h->coef_r32, h->coef_c32, h->f, h->g, h->ym, h->yn, h->dz, h->dx, h->sd, h->vd, h->copy2};
    for (void *q : p)
        if (q) cudaFree(q);
    cudaEvent_t e[] = {h->ev0, h->ev1, h->k0, h->k1};
    for (cudaEvent_t q : e)
        if (q) cudaEventDestroy(q);
    delete h;
}

// squared Frobenius norms of consecutive groups of tau lines, their prefix sums,
// the last group of nonzero norm
void group_tables(const std::vector<int64_t> &ptr, const std::vector<double> &val, int64_t lines, int tau,
                  std::vector<double> &norms, std::vector<double> &cdf, int *fallback) {
    const int64_t g = (lines + tau - 1) / tau;
    norms.assign(g, 0.0);
    cdf.assign(g, 0.0);
    for (int64_t b = 0; b < g; ++b) {
        double s = 0.0;
        const int64_t l1 = std::min(lines, (b + 1) * tau);
        for (int64_t l = b * tau; l < l1; ++l)
            for (int64_t e = ptr[l]; e < ptr[l + 1]; ++e) s += val[e] * val[e];
        norms[b] = s;
    }
    double run = 0.0;
    *fallback = 0;
    for (int64_t b = 0; b < g; ++b) {
        run += norms[b];
        cdf[b] = run;
        if (norms[b] > 0.0) *fallback = (int)b;
    }
}

}  // namespace

namespace {

// Fields of the kernel arguments that every launch of a handle shares.
SparseArgs sparse_args(rebk_sparse h, bool corr) {
    SparseArgs a;
    memset(&a, 0, sizeof(a));
    a.m = h->m;
    a.n = h->n;
    a.tau_r = h->tau_r;
    a.tau_c = h->tau_c;
    a.rp = h->rp;
    a.ci = h->ci;
    a.cp = h->cp;
    a.ri = h->ri;
    a.rv = corr ? (const void *)h->rv32 : (const void *)h->rv;
    a.cv = corr ? (const void *)h->cv32 : (const void *)h->cv;
    a.coef_r = corr ? (const void *)h->coef_r32 : (const void *)h->coef_r;
    a.coef_c = corr ? (const void *)h->coef_c32 : (const void *)h->coef_c;
    a.check_every = h->check_every;
    a.acc = h->acc;
    a.bad = h->bad;
    a.bar = h->bar;
    a.status = h->status;
    a.iters_done = h->iters_done;
    a.timeout_ns = kBarrierTimeoutNs;
    return a;
}

// Samples the blocks of iterations kfirst+1 .. kfirst+K into idx and runs them in one
// persistent launch; returns the device status (0, 5 diverged, 6 barrier timeout),
// the iterations done and the launch's CUDA-event time.
rebk_status sparse_launch(rebk_sparse h, bool corr, SparseArgs &a, uint64_t seed, uint64_t stream_id,
                          int64_t kfirst, int64_t K, int32_t *idx, int *dev_status, int64_t *done, float *ms) {
    const cudaStream_t st = h->stream;
    SCK(sample_blocks(seed, stream_id, kfirst, K, h->cdf_r, h->s, h->cdf_c, h->t, h->fb_r, h->fb_c, idx, st));
    SCK(cudaMemsetAsync(h->acc, 0, sizeof(double) * 4, st));
    SCK(cudaMemsetAsync(h->bad, 0, sizeof(int), st));
    SCK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    SCK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned int), st));
    a.idx = idx;
    a.iters = K;
    // second copies of x and z, equal to them at launch (the kernel writes the final
    // iterates back into x and z)
    const size_t es = corr ? sizeof(float) : sizeof(double);
    a.x2 = h->copy2;
    a.z2 = static_cast<char *>(h->copy2) + (((size_t)h->n * es + 255) & ~(size_t)255);
    SCK(cudaMemcpyAsync(a.x2, a.x, (size_t)h->n * es, cudaMemcpyDeviceToDevice, st));
    SCK(cudaMemcpyAsync(a.z2, a.z, (size_t)h->m * es, cudaMemcpyDeviceToDevice, st));
    void *params[] = {&a};
    void *fn = corr ? reinterpret_cast<void *>(&rebk_sparse_kernel<float, true>)
                    : reinterpret_cast<void *>(&rebk_sparse_kernel<double, false>);
    SCK(cudaEventRecord(h->k0, st));
    SCK(cudaLaunchCooperativeKernel(fn, dim3(h->G), dim3(kST), params, 0, st));
    SCK(cudaEventRecord(h->k1, st));
    *dev_status = 0;
    *done = 0;
    SCK(cudaMemcpyAsync(dev_status, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(done, h->iters_done, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    *ms = 0.f;
    cudaEventElapsedTime(ms, h->k0, h->k1);
    return REBK_OK;
}

rebk_status fetch(rebk_sparse h, double *v, int count) {
    SCK(cudaMemcpyAsync(v, h->small, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
    SCK(cudaStreamSynchronize(h->stream));
    return REBK_OK;
}

void sparse_stats(rebk_stats *stats, int64_t iters, int outer, rebk_status result, double rel, double rf,
                  double rg, double dms, double kms, int64_t launches, int64_t grid_launches) {
    if (!stats) return;
    memset(stats, 0, sizeof(*stats));
    stats->iterations = iters;
    stats->outer = outer;
    stats->status = result;
    stats->rel_err = rel;
    stats->resid_f = rf;
    stats->resid_g = rg;
    stats->device_ms = dms;
    stats->kernel_ms = kms;
    stats->launches = launches;
    stats->grid_launches = grid_launches;
}

}  // namespace

extern "C" {

rebk_status rebk_sparse_create(rebk_sparse *out, int64_t m, int64_t n, const int64_t *row_ptr,
                               const int32_t *col_idx, const double *val, int64_t tau_row, int64_t tau_col,
                               double alpha, const rebk_sparse_options *opt) {
    set_last_error("");
    if (!out) return sfail(REBK_EINVAL, "out is NULL");
    *out = nullptr;
    if (m < 1 || n < 1 || m > INT32_MAX || n > INT32_MAX) return sfail(REBK_EINVAL, "need 1 <= m, n < 2^31");
    if (!row_ptr || !col_idx || !val) return sfail(REBK_EINVAL, "NULL CSR array");
    if (tau_row < 1 || tau_col < 1) return sfail(REBK_EINVAL, "block sizes must be >= 1");
    if (!std::isfinite(alpha)) return sfail(REBK_EINVAL, "alpha is not finite");
    rebk_sparse_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.num_ctas < 0 || o.check_every < 0 || o.power_iters < 0) return sfail(REBK_EINVAL, "negative option");
    const int64_t nnz = row_ptr[m];
    if (row_ptr[0] != 0 || nnz < 0) return sfail(REBK_EINVAL, "row_ptr must start at 0");
    for (int64_t i = 0; i < m; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return sfail(REBK_EINVAL, "row_ptr must be nondecreasing");
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (col_idx[e] < 0 || col_idx[e] >= n) return sfail(REBK_EINVAL, "column index out of range");
            if (e > row_ptr[i] && col_idx[e] <= col_idx[e - 1])
                return sfail(REBK_EINVAL, "column indices must increase within a row");
            if (!std::isfinite(val[e])) return sfail(REBK_EINVAL, "non-finite value");
        }
    }
    rebk_sparse h = new rebk_sparse_s();
    h->m = m;
    h->n = n;
    h->nnz = nnz;
    h->tau_r = (int)std::min<int64_t>(tau_row, m);
    h->tau_c = (int)std::min<int64_t>(tau_col, n);
    h->s = (int)((m + h->tau_r - 1) / h->tau_r);
    h->t = (int)((n + h->tau_c - 1) / h->tau_c);
    h->check_every = o.check_every > 0 ? o.check_every : 10;
    h->stream = static_cast<cudaStream_t>(o.stream);
    auto fin = [&](rebk_status s) {
        if (s != REBK_OK) free_sparse(h);
        return s;
    };
    // host CSR and CSC (stable: entries of a column in increasing row order)
    std::vector<int64_t> rp(row_ptr, row_ptr + m + 1), cp(n + 1, 0);
    std::vector<int32_t> ci(col_idx, col_idx + nnz), ri(nnz);
    std::vector<double> rv(val, val + nnz), cv(nnz);
    for (int64_t e = 0; e < nnz; ++e) ++cp[ci[e] + 1];
    for (int64_t c = 0; c < n; ++c) cp[c + 1] += cp[c];
    {
        std::vector<int64_t> next(cp.begin(), cp.end() - 1);
        for (int64_t i = 0; i < m; ++i)
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                const int64_t d = next[ci[e]]++;
                ri[d] = (int32_t)i;
                cv[d] = rv[e];
            }
    }
    // tables (Algorithm 1 sampling), FP64
    std::vector<double> nr, nc, cdf_r, cdf_c;
    group_tables(rp, rv, m, h->tau_r, nr, cdf_r, &h->fb_r);
    group_tables(cp, cv, n, h->tau_c, nc, cdf_c, &h->fb_c);
    h->fro2 = h->s > 0 ? cdf_r[h->s - 1] : 0.0;
    // step: alpha, or 1.75 / beta_max with ||block||_2^2 from power iterations
    const int piters = o.power_iters > 0 ? o.power_iters : 100;
    double beta = 0.0;
    if (alpha <= 0.0) {  // blocks split over host threads; each ratio written once
        std::vector<double> ratio(h->s + h->t, 0.0);
        auto work = [&](int first, int stride) {
            for (int b = first; b < h->s + h->t; b += stride) {
                if (b < h->s) {
                    if (nr[b] > 0.0)
                        ratio[b] = block_spectral_sq(rp, ci, rv, (int64_t)b * h->tau_r,
                                                     std::min<int64_t>(m, (int64_t)(b + 1) * h->tau_r), n, piters) /
                                   nr[b];
                } else {
                    const int c = b - h->s;
                    if (nc[c] > 0.0)
                        ratio[b] = block_spectral_sq(cp, ri, cv, (int64_t)c * h->tau_c,
                                                     std::min<int64_t>(n, (int64_t)(c + 1) * h->tau_c), m, piters) /
                                   nc[c];
                }
            }
        };
        const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int q = 1; q < nt; ++q) pool.emplace_back(work, q, nt);
        work(0, nt);
        for (auto &th : pool) th.join();
        for (double r : ratio) beta = std::max(beta, r);
    }
    h->beta = beta;
    h->alpha = alpha > 0.0 ? alpha : (beta > 0.0 ? 1.75 / beta : 1.0);
    std::vector<double> kr(h->s), kc(h->t);
    for (int b = 0; b < h->s; ++b) kr[b] = nr[b] > 0.0 ? h->alpha / nr[b] : 0.0;
    for (int b = 0; b < h->t; ++b) kc[b] = nc[b] > 0.0 ? h->alpha / nc[b] : 0.0;
    // device copies
#define SCKH(call)                                                                                 \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess)                                                                    \
            return fin(sfail(e__ == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA,          \
                             std::string(#call) + ": " + cudaGetErrorString(e__)));                \
    } while (0)
    auto up = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(dst, bytes > 0 ? bytes : 8);
        if (e == cudaSuccess && bytes > 0) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
        return e;
    };
    SCKH(up((void **)&h->rp, rp.data(), sizeof(int64_t) * (m + 1)));
    SCKH(up((void **)&h->cp, cp.data(), sizeof(int64_t) * (n + 1)));
    SCKH(up((void **)&h->ci, ci.data(), sizeof(int32_t) * nnz));
    SCKH(up((void **)&h->ri, ri.data(), sizeof(int32_t) * nnz));
    SCKH(up((void **)&h->rv, rv.data(), sizeof(double) * nnz));
    SCKH(up((void **)&h->cv, cv.data(), sizeof(double) * nnz));
    SCKH(up((void **)&h->cdf_r, cdf_r.data(), sizeof(double) * h->s));
    SCKH(up((void **)&h->cdf_c, cdf_c.data(), sizeof(double) * h->t));
    SCKH(up((void **)&h->coef_r, kr.data(), sizeof(double) * h->s));
    SCKH(up((void **)&h->coef_c, kc.data(), sizeof(double) * h->t));
    {  // FP32 copies for the mixed-precision solve (round to nearest)
        std::vector<float> r32(rv.begin(), rv.end()), c32(cv.begin(), cv.end());
        std::vector<float> kr32(kr.begin(), kr.end()), kc32(kc.begin(), kc.end());
        SCKH(up((void **)&h->rv32, r32.data(), sizeof(float) * nnz));
        SCKH(up((void **)&h->cv32, c32.data(), sizeof(float) * nnz));
        SCKH(up((void **)&h->coef_r32, kr32.data(), sizeof(float) * h->s));
        SCKH(up((void **)&h->coef_c32, kc32.data(), sizeof(float) * h->t));
    }
    SCKH(cudaMalloc(&h->f, sizeof(double) * m));
    SCKH(cudaMalloc(&h->ym, sizeof(double) * m));
    SCKH(cudaMalloc(&h->g, sizeof(double) * n));
    SCKH(cudaMalloc(&h->yn, sizeof(double) * n));
    SCKH(cudaMalloc(&h->dz, sizeof(float) * m));
    SCKH(cudaMalloc(&h->vd, sizeof(float) * m));
    SCKH(cudaMalloc(&h->dx, sizeof(float) * n));
    SCKH(cudaMalloc(&h->sd, sizeof(float) * n));
    SCKH(cudaMalloc(&h->idx, sizeof(int32_t) * 2 * kSparseChunk));
    SCKH(cudaMalloc(&h->zbuf, sizeof(double) * m));
    SCKH(cudaMalloc(&h->copy2, sizeof(double) * (m + n) + 256));  // z's copy starts 256-aligned
    SCKH(cudaMalloc(&h->acc, sizeof(double) * 4));
    SCKH(cudaMalloc(&h->small, sizeof(double) * 4));
    SCKH(cudaMalloc(&h->bad, sizeof(int)));
    SCKH(cudaMalloc(&h->status, sizeof(int)));
    SCKH(cudaMalloc(&h->bar, sizeof(unsigned int)));
    SCKH(cudaMalloc(&h->iters_done, sizeof(int64_t)));
    SCKH(cudaEventCreate(&h->ev0));
    SCKH(cudaEventCreate(&h->ev1));
    SCKH(cudaEventCreate(&h->k0));
    SCKH(cudaEventCreate(&h->k1));
    // grid: one CTA per SM (cooperative), enough CTAs for every block's lines
    int dev = 0, sms = 1, per = 0, per32 = 0;
    SCKH(cudaGetDevice(&dev));
    SCKH(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SCKH(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rebk_sparse_kernel<double, false>, kST, 0));
    SCKH(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per32, rebk_sparse_kernel<float, true>, kST, 0));
    per = std::min(per, per32);
    const int gmax = sms * std::max(1, std::min(per, 1));
    int G = o.num_ctas > 0 ? std::min(o.num_ctas, gmax) : gmax;
    const int need = (int)((std::max(h->tau_r, h->tau_c) + kOwnMax - 1) / kOwnMax);
    if (G < need) G = std::min(gmax, need);
    if ((int64_t)G * kOwnMax < std::max(h->tau_r, h->tau_c))
        return fin(sfail(REBK_EUNSUPPORTED, "block size too large for the persistent grid"));
    h->G = G;
    *out = h;
    return REBK_OK;
}

void rebk_sparse_destroy(rebk_sparse h) { free_sparse(h); }

rebk_status rebk_sparse_info(rebk_sparse h, double *alpha, double *beta_max, int32_t *row_blocks,
                             int32_t *col_blocks) {
    if (!h) return sfail(REBK_EINVAL, "NULL handle");
    if (alpha) *alpha = h->alpha;
    if (beta_max) *beta_max = h->beta;
    if (row_blocks) *row_blocks = h->s;
    if (col_blocks) *col_blocks = h->t;
    return REBK_OK;
}

rebk_status rebk_sparse_solve(rebk_sparse h, const double *b, double *x, double tol, int64_t max_iter,
                              uint64_t seed, const rebk_solve_ext *ext, rebk_stats *stats) {
    set_last_error("");
    if (!h) return sfail(REBK_EINVAL, "NULL handle");
    if (!b || !x) return sfail(REBK_EINVAL, "b and x must be device pointers");
    if (max_iter < 0 || !std::isfinite(tol)) return sfail(REBK_EINVAL, "bad tol / max_iter");
    rebk_solve_ext e;
    memset(&e, 0, sizeof(e));
    if (ext) e = *ext;
    if (e.k0 < 0) return sfail(REBK_EINVAL, "k0 < 0");
    const cudaStream_t st = h->stream;
    double *z = e.z_out ? e.z_out : h->zbuf;
    SCK(cudaEventRecord(h->ev0, st));
    if (e.z0) SCK(cudaMemcpyAsync(z, e.z0, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    else SCK(cudaMemcpyAsync(z, b, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    if (e.x0) SCK(cudaMemcpyAsync(x, e.x0, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, st));
    else SCK(cudaMemsetAsync(x, 0, sizeof(double) * h->n, st));
    double refn = 0.0;
    if (e.x_ref) {
        SCK(sum_sq(e.x_ref, h->n, h->small, st));
        double v[2];
        rebk_status fs = fetch(h, v, 2);
        if (fs != REBK_OK) return fs;
        refn = std::sqrt(v[1]);
    }
    const double thr = tol * refn;
    int64_t extra = e.x_ref ? 2 : 0;  // sum_sq, err_norms
    int64_t total = 0, launches = 0, grid_launches = 0;
    double kernel_ms = 0.0;
    rebk_status result = REBK_MAX_ITER;
    bool converged = false;
    while (total < max_iter && h->fro2 > 0.0) {
        const int64_t K = std::min({max_iter - total, kSparseChunk, kSparseLaunchMax});
        int32_t *idx = e.idx_out ? e.idx_out + 2 * total : h->idx;
        SparseArgs a = sparse_args(h, false);
        a.z = z;
        a.x = x;
        a.b = b;
        a.x_ref = e.x_ref;
        a.tol2_abs = thr * thr;
        a.check_offset = total;
        int ds = 0;
        int64_t done = 0;
        float ms = 0.f;
        rebk_status ls = sparse_launch(h, false, a, seed, e.stream_id, e.k0 + total, K, idx, &ds, &done, &ms);
        if (ls != REBK_OK) return ls;
        launches += 2;  // sample_kernel, rebk_sparse_kernel
        ++grid_launches;
        kernel_ms += ms;
        if (ds != 6) total += done;
        if (ds == 6) {
            result = REBK_BARRIER_TIMEOUT;
            sfail(result, "device-wide barrier timed out");
            break;
        }
        if (ds == 5) {
            result = REBK_DIVERGED;
            sfail(result, "iteration diverged (Inf/NaN)");
            break;
        }
        if (done < K) {
            converged = true;
            result = REBK_OK;
            break;
        }
    }
    double rel = -1.0;
    if (e.x_ref && result != REBK_BARRIER_TIMEOUT) {
        SCK(err_norms(nullptr, x, e.x_ref, h->n, h->small, st));
        double v[2];
        rebk_status fs = fetch(h, v, 2);
        if (fs != REBK_OK) return fs;
        rel = refn > 0 ? std::sqrt(v[0]) / refn : std::sqrt(v[0]);
        if (!converged && result == REBK_MAX_ITER && rel <= tol) result = REBK_OK;
    } else if (!e.x_ref && result == REBK_MAX_ITER) {
        result = REBK_OK;  // fixed iteration count
    }
    if (h->fro2 == 0.0) result = REBK_OK;  // A = 0: x = 0 is A^+ b
    SCK(cudaEventRecord(h->ev1, st));
    SCK(cudaEventSynchronize(h->ev1));
    float dms = 0.f;
    cudaEventElapsedTime(&dms, h->ev0, h->ev1);
    sparse_stats(stats, total, 0, result, rel, -1, -1, dms, kernel_ms, launches + extra, grid_launches);
    return result;
}

rebk_status rebk_sparse_solve_refined(rebk_sparse h, const double *b, double *x, double tol, int64_t max_iter,
                                      uint64_t seed, const rebk_refine_opts *ropt, const rebk_solve_ext *ext,
                                      rebk_stats *stats) {
    set_last_error("");
    if (!h) return sfail(REBK_EINVAL, "NULL handle");
    if (!b || !x) return sfail(REBK_EINVAL, "b and x must be device pointers");
    if (max_iter < 0 || !std::isfinite(tol)) return sfail(REBK_EINVAL, "bad tol / max_iter");
    rebk_refine_opts ro;
    memset(&ro, 0, sizeof(ro));
    ro.storage = REBK_FP32;
    if (ropt) ro = *ropt;
    if (ro.storage == REBK_BF16) return sfail(REBK_EUNSUPPORTED, "sparse mixed precision stores FP32 values only");
    if (ro.storage != REBK_FP32) return sfail(REBK_EINVAL, "refinement storage must be REBK_FP32");
    if (ro.max_outer < 0 || ro.inner_iters < 0 || ro.inner_reduction < 0)
        return sfail(REBK_EINVAL, "negative refinement option");
    const int max_outer = ro.max_outer > 0 ? ro.max_outer : 30;
    const double red = ro.inner_reduction > 0 ? ro.inner_reduction : 1e-4;
    rebk_solve_ext e;
    memset(&e, 0, sizeof(e));
    if (ext) e = *ext;
    if (e.k0 < 0) return sfail(REBK_EINVAL, "k0 < 0");
    const cudaStream_t st = h->stream;
    double *z = e.z_out ? e.z_out : h->zbuf;
    int64_t launches = 0, grid_launches = 0;
    double kernel_ms = 0.0;
    SCK(cudaEventRecord(h->ev0, st));
    if (e.z0) SCK(cudaMemcpyAsync(z, e.z0, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    else SCK(cudaMemcpyAsync(z, b, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    if (e.x0) SCK(cudaMemcpyAsync(x, e.x0, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, st));
    else SCK(cudaMemsetAsync(x, 0, sizeof(double) * h->n, st));
    const bool use_ref = e.x_ref != nullptr;
    double refn = 0.0;
    if (use_ref) {
        SCK(sum_sq(e.x_ref, h->n, h->small, st));
        ++launches;
        double v[2];
        rebk_status fs = fetch(h, v, 2);
        if (fs != REBK_OK) return fs;
        refn = std::sqrt(v[1]);
    }
    int64_t inner_max = ro.inner_iters;
    if (inner_max <= 0) {
        if (use_ref) {
            inner_max = 1000000;
        } else {
            const double per_iter = (double)h->tau_r * h->n + (double)h->tau_c * h->m;
            inner_max = std::max<int64_t>(200, (int64_t)(40.0 * (double)h->m * h->n / per_iter));
        }
    }
    int64_t total = 0;
    int outer = 0;
    rebk_status result = REBK_MAX_ITER;
    double rel = -1, rf = -1, rg = -1, prev_res = -1;
    bool x_zero = e.x0 == nullptr;  // x^0 = 0: A x vanishes in the first residual
    for (outer = 0; h->fro2 > 0.0 && max_iter > 0 && outer < max_outer; ++outer) {
        double e0 = 0.0;
        if (use_ref) {  // the error test needs x only: before the residuals
            SCK(err_norms(nullptr, x, e.x_ref, h->n, h->small, st));
            ++launches;
            double v[2];
            rebk_status fs = fetch(h, v, 2);
            if (fs != REBK_OK) return fs;
            e0 = std::sqrt(v[0]);
            rel = refn > 0 ? e0 / refn : e0;
            if (rel <= tol) {
                result = REBK_OK;
                break;
            }
        }
        // f = b - z - A x (CSR), g = A^T z (CSC), FP64 values
        if (x_zero) SCK(cudaMemsetAsync(h->ym, 0, sizeof(double) * h->m, st));
        else SCK(sparse_lines<double>(h->rp, h->ci, h->rv, x, h->m, h->ym, st));
        SCK(sparse_lines<double>(h->cp, h->ri, h->cv, z, h->n, h->g, st));
        SCK(form_f(b, z, h->ym, h->f, h->m, st));
        launches += x_zero ? 2 : 3;
        x_zero = false;
        if (!use_ref) {
            SCK(sum_sq(h->f, h->m, h->small, st));
            SCK(sum_sq(h->g, h->n, h->small + 2, st));
            launches += 2;
            double v[4];
            rebk_status fs = fetch(h, v, 4);
            if (fs != REBK_OK) return fs;
            SCK(sum_sq(b, h->m, h->small, st));
            ++launches;
            double vb[2];
            fs = fetch(h, vb, 2);
            if (fs != REBK_OK) return fs;
            const double nb = std::sqrt(vb[1]);
            rf = nb > 0 ? std::sqrt(v[1]) / nb : 0.0;
            rg = nb > 0 ? std::sqrt(v[3]) / (std::sqrt(h->fro2) * nb) : 0.0;
            const double res = std::max(rf, rg);
            if (res <= tol) {
                result = REBK_OK;
                break;
            }
            if (prev_res > 0 && res > 0.1 * prev_res) inner_max = std::min<int64_t>(inner_max * 2, 1 << 24);
            prev_res = res;
        }
        if (total >= max_iter) break;
        // inner sweeps on corrections from zero
        SCK(fill_zero_f32(h->dz, h->m, st));
        SCK(fill_zero_f32(h->vd, h->m, st));
        SCK(fill_zero_f32(h->dx, h->n, st));
        SCK(fill_zero_f32(h->sd, h->n, st));
        launches += 4;
        const int64_t iters = std::min(inner_max, max_iter - total);
        int64_t ran = 0, grow = 4096;  // chunks of 4096, 4096, 8192, ... iterations with a reference
        int chunks = 0;
        // The pass ends at its error test, or once the error of x + dx stops falling
        // (the floor the FP32 values set), as in the dense mixed-precision solve.
        double e_prev = e0, rate_prev = -1.0;
        while (ran < iters) {
            int64_t chunk = std::min({iters - ran, kSparseChunk, kSparseLaunchMax});
            if (use_ref) {
                chunk = std::min(chunk, grow);
                if (++chunks >= 2) grow = std::min<int64_t>(grow * 2, kSparseChunk);
            }
            SparseArgs a = sparse_args(h, true);
            a.z = h->dz;
            a.x = h->dx;
            a.b = h->f;
            a.g = h->g;
            a.sdual = h->sd;
            a.vdual = h->vd;
            a.check_offset = ran;
            if (use_ref) {
                const double thr = std::max(tol * refn, red * e0);
                a.x_ref = e.x_ref;
                a.x_base = x;
                a.tol2_abs = thr * thr;
            }
            int32_t *idx = e.idx_out ? e.idx_out + 2 * (total + ran) : h->idx;
            int ds = 0;
            int64_t done = 0;
            float ms = 0.f;
            rebk_status ls = sparse_launch(h, true, a, seed, e.stream_id, e.k0 + total + ran, chunk, idx, &ds, &done,
                                           &ms);
            if (ls != REBK_OK) return ls;
            launches += 2;
            ++grid_launches;
            kernel_ms += ms;
            if (ds == 6) {
                sparse_stats(stats, total + ran, outer + 1, REBK_BARRIER_TIMEOUT, -1, -1, -1, 0, kernel_ms, launches,
                             grid_launches);
                return sfail(REBK_BARRIER_TIMEOUT, "device-wide barrier timed out");
            }
            ran += done;
            if (ds == 5) {
                sparse_stats(stats, total + ran, outer + 1, REBK_DIVERGED, -1, -1, -1, 0, kernel_ms, launches,
                             grid_launches);
                return sfail(REBK_DIVERGED, "inner iteration diverged (Inf/NaN)");
            }
            if (done < chunk) break;  // error test met
            if (use_ref && ran < iters) {
                SCK(err_norms_f32(x, h->dx, e.x_ref, h->n, h->small, st));
                ++launches;
                double v[2];
                rebk_status fs = fetch(h, v, 2);
                if (fs != REBK_OK) return fs;
                const double e_now = std::sqrt(v[0]);
                if (!(e_now < e_prev)) break;
                const double rate = std::log(e_prev / e_now) / (double)done;
                if (rate_prev > 0.0 && rate < 0.1 * rate_prev) break;
                rate_prev = rate;
                e_prev = e_now;
            }
        }
        total += ran;
        // z <- z - A s (CSR), x <- x + A^T v (CSC), FP64 values
        SCK(sparse_lines<float>(h->rp, h->ci, h->rv, h->sd, h->m, h->ym, st));
        SCK(sparse_lines<float>(h->cp, h->ri, h->cv, h->vd, h->n, h->yn, st));
        SCK(apply_update(x, h->yn, h->n, z, h->ym, h->m, st));
        launches += 3;
    }
    if (h->fro2 == 0.0 || max_iter == 0) {
        result = h->fro2 == 0.0 || !use_ref ? REBK_OK : REBK_MAX_ITER;
    }
    if (result != REBK_OK && h->fro2 > 0.0) {  // final test after the last pass
        if (use_ref) {
            SCK(err_norms(nullptr, x, e.x_ref, h->n, h->small, st));
            ++launches;
            double v[2];
            rebk_status fs = fetch(h, v, 2);
            if (fs != REBK_OK) return fs;
            rel = refn > 0 ? std::sqrt(v[0]) / refn : std::sqrt(v[0]);
            if (rel <= tol) result = REBK_OK;
        } else if (max_iter > 0) {
            SCK(sparse_lines<double>(h->rp, h->ci, h->rv, x, h->m, h->ym, st));
            SCK(sparse_lines<double>(h->cp, h->ri, h->cv, z, h->n, h->g, st));
            SCK(form_f(b, z, h->ym, h->f, h->m, st));
            SCK(sum_sq(h->f, h->m, h->small, st));
            SCK(sum_sq(h->g, h->n, h->small + 2, st));
            launches += 5;
            double v[4];
            rebk_status fs = fetch(h, v, 4);
            if (fs != REBK_OK) return fs;
            SCK(sum_sq(b, h->m, h->small, st));
            ++launches;
            double vb[2];
            fs = fetch(h, vb, 2);
            if (fs != REBK_OK) return fs;
            const double nb = std::sqrt(vb[1]);
            rf = nb > 0 ? std::sqrt(v[1]) / nb : 0.0;
            rg = nb > 0 ? std::sqrt(v[3]) / (std::sqrt(h->fro2) * nb) : 0.0;
            if (std::max(rf, rg) <= tol) result = REBK_OK;
        }
    }
    if (use_ref && rel < 0 && result != REBK_BARRIER_TIMEOUT) {
        SCK(err_norms(nullptr, x, e.x_ref, h->n, h->small, st));
        ++launches;
        double v[2];
        rebk_status fs = fetch(h, v, 2);
        if (fs != REBK_OK) return fs;
        rel = refn > 0 ? std::sqrt(v[0]) / refn : std::sqrt(v[0]);
    }
    SCK(cudaEventRecord(h->ev1, st));
    SCK(cudaEventSynchronize(h->ev1));
    float dms = 0.f;
    cudaEventElapsedTime(&dms, h->ev0, h->ev1);
    sparse_stats(stats, total, outer, result, rel, rf, rg, dms, kernel_ms, launches, grid_launches);
    return result;
}

}  // extern "C"
