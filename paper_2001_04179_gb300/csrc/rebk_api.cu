// rebk_api.cu -- C ABI of the REBK solver (see include/rebk.h).
//
// Host logic only: argument checks, device buffers of the handle, the outer
// loops (stopping tests, chunked launches, the FP64 refinement passes) and the
// choice of the persistent kernel's CTA count.  Every arithmetic step of the
// method runs in the kernels of rebk_grid.cu and rebk_setup.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "rebk.h"
#include "rebk_internal.h"

using namespace rebk;

namespace {

thread_local std::string g_last_error;

rebk_status fail(rebk_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

rebk_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess) return cuda_fail(e__, #call);                                      \
    } while (0)

// a call that launches one kernel of this library: counted in the solve stats
#define LK(h, call)                                                                                \
    do {                                                                                           \
        ++(h)->launches;                                                                           \
        CK(call);                                                                                  \
    } while (0)

int64_t round_up(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

struct Workspace {
    unsigned int bar;
    unsigned int bar_x;
    int status;
    int64_t iters_done;
    double small[8];
};

}  // namespace

struct rebk_handle_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t m = 0, n = 0, lda = 0;
    int tau_r = 0, tau_c = 0, s = 0, t = 0;
    double alpha = 0.0, fro2 = 0.0;
    int fb[2] = {0, 0};
    double *A64 = nullptr;
    float *A32 = nullptr;
    __nv_bfloat16 *A16 = nullptr;
    double *nr = nullptr, *nc = nullptr, *cdf_r = nullptr, *cdf_c = nullptr;
    int *d_fallback = nullptr;
    // partition: offsets on the device (NULL = contiguous blocks of tau_r / tau_c)
    int64_t *d_row_off = nullptr, *d_col_off = nullptr;
    std::vector<int64_t> row_off, col_off;  // host copies (always filled)
    int col_align = 0;
    void *acc = nullptr;  // 2 chains x 3 sets x acc_r replicas x acc_w, 8 bytes per entry
    int acc_w = 0, acc_r = kAccReplicas;
    double *coef_r64 = nullptr, *coef_c64 = nullptr;
    float *coef_r32 = nullptr, *coef_c32 = nullptr;
    GridArgs prep[3];       // prepared launch arguments per mode (for prepG CTAs)
    int prepG[3] = {0, 0, 0};
    Workspace *ws = nullptr;
    double *zbuf = nullptr, *f = nullptr, *g = nullptr, *ym = nullptr, *yn = nullptr;
    float *dz = nullptr, *dx = nullptr, *sd = nullptr, *vd = nullptr;
    int64_t check_every = 0;
    int num_ctas_opt = 0;
    int G[3] = {0, 0, 0};
    bool beta_done = false;
    double beta_r = 0.0, beta_c = 0.0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int32_t *idxbuf = nullptr;  // sampled block indices of one launch
    int64_t idx_cap = 0;        // capacity in iterations
    // per-solve counters (reset at the start of each solve)
    int64_t launches = 0, grid_launches = 0;
    double kernel_ms = 0.0;
    std::vector<cudaEvent_t> sweep_ev;  // start/stop pairs of the FP64 sweeps
    size_t sweep_used = 0;
    cudaEvent_t kev0 = nullptr, kev1 = nullptr;
    // partition-free sampling (rebk_solve_free): per-row / per-column tables,
    // built on first use; draws of one launch; accumulators
    double *fr_rn = nullptr, *fr_cn = nullptr, *fr_cdf_r = nullptr, *fr_cdf_c = nullptr;
    int fr_fb[2] = {0, 0};
    int32_t *fr_idx = nullptr;
    int64_t fr_idx_cap = 0;  // in int32 entries
    double *fr_acc = nullptr;
    int fr_acc_w = 0;
    double *fr_AT = nullptr;  // FP64 A^T (n rows of fr_ldt), built on the first partition-free solve
    int64_t fr_ldt = 0;
    // several right-hand sides at once (rebk_solve_multi): one device buffer
    void *mr_buf = nullptr;
    size_t mr_bytes = 0;
};

namespace {

void free_handle(rebk_handle h) {
    if (!h) return;
    void *ptrs[] = {h->A64, h->A32, h->A16, h->nr, h->nc, h->cdf_r, h->cdf_c, h->d_fallback, h->acc,
                    h->d_row_off, h->d_col_off, h->fr_rn, h->fr_cn, h->fr_cdf_r, h->fr_cdf_c,
                    h->fr_idx, h->fr_acc, h->fr_AT, h->mr_buf,
                    h->coef_r64, h->coef_c64, h->coef_r32, h->coef_c32,
                    h->ws, h->zbuf, h->f, h->g, h->ym, h->yn, h->dz, h->dx, h->sd, h->vd,
                    h->idxbuf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->kev0) cudaEventDestroy(h->kev0);
    if (h->kev1) cudaEventDestroy(h->kev1);
    for (cudaEvent_t e : h->sweep_ev) cudaEventDestroy(e);
    delete h;
}

int mode_index(Mode m) { return m == Mode::PlainF64 ? 0 : (m == Mode::CorrF32 ? 1 : 2); }

constexpr size_t kSmemLimit = 227 * 1024;

// Launch arguments that depend only on the handle, the mode and the CTA count
// G: matrix copy, tables, workspace, owned-slice capacities and, when the
// tiles fit twice in shared memory, the TMA box geometry and tensor maps.
GridArgs base_args(rebk_handle h, Mode mode, int G) {
    const int mi = mode == Mode::PlainF64 ? 0 : (mode == Mode::CorrF32 ? 1 : 2);
    if (h->prepG[mi] == G) return h->prep[mi];
    GridArgs a;
    memset(&a, 0, sizeof(a));
    a.A = mode == Mode::PlainF64 ? (const void *)h->A64
                                 : (mode == Mode::CorrF32 ? (const void *)h->A32 : (const void *)h->A16);
    a.lda = h->lda;
    a.m = h->m;
    a.n = h->n;
    a.tau_r = h->tau_r;
    a.tau_c = h->tau_c;
    a.s = h->s;
    a.t = h->t;
    a.row_off = h->d_row_off;
    a.col_off = h->d_col_off;
    a.col_align = h->col_align;
    a.cdf_r = h->cdf_r;
    a.cdf_c = h->cdf_c;
    a.nr = h->nr;
    a.nc = h->nc;
    a.coef_r = mode == Mode::PlainF64 ? (const void *)h->coef_r64 : (const void *)h->coef_r32;
    a.coef_c = mode == Mode::PlainF64 ? (const void *)h->coef_c64 : (const void *)h->coef_c32;
    a.fb_r = h->fb[0];
    a.fb_c = h->fb[1];
    a.alpha = h->alpha;
    a.acc = h->acc;
    a.acc_w = h->acc_w;
    a.acc_r = acc_replicas(mode);
    a.nrow_cap = (int)((h->m + G - 1) / G) + 1;
    const int64_t nu = (h->n + 7) / 8;
    a.ncol_cap = (int)(8 * ((nu + G - 1) / G)) + 8;
    a.bar = &h->ws->bar;
    a.bar_x = &h->ws->bar_x;
    a.status = &h->ws->status;
    a.iters_done = &h->ws->iters_done;
    a.timeout_ns = kBarrierTimeoutNs;
    a.use_tma = 0;
    if (mode != Mode::PlainF64 && a.A != nullptr && tma_geometry(mode, a)) {
        a.use_tma = 1;
        if (grid_smem_bytes(mode, a) > kSmemLimit || tma_encode(mode, a) != cudaSuccess) a.use_tma = 0;
    }
    h->prep[mi] = a;
    h->prepG[mi] = G;
    return a;
}

constexpr int64_t kIdxChunkMax = 1 << 20;  // iterations sampled per launch (internal buffer)

// Samples the block indices of iterations k0+1 .. k0+K into `user` (if not
// NULL) or the handle's buffer; sets a.idx.
rebk_status sample_into(rebk_handle h, GridArgs &a, int64_t k0, int64_t K, int32_t *user) {
    int32_t *dst = user;
    if (!dst) {
        if (K > h->idx_cap) {
            if (h->idxbuf) cudaFree(h->idxbuf);
            h->idxbuf = nullptr;
            h->idx_cap = 0;
            const int64_t cap = std::max<int64_t>(K, 65536);
            CK(cudaMalloc(&h->idxbuf, sizeof(int32_t) * 2 * cap));
            h->idx_cap = cap;
        }
        dst = h->idxbuf;
    }
    LK(h, sample_blocks(a.seed, a.stream, k0, K, h->cdf_r, h->s, h->cdf_c, h->t, h->fb[0], h->fb[1],
                        dst, h->stream));
    a.idx = dst;
    a.k0 = k0;
    a.iters = K;
    return REBK_OK;
}

// One launch of the persistent kernel (a.idx, a.k0, a.iters set); returns the
// device status and the iterations it ran.
rebk_status run_grid(rebk_handle h, Mode mode, GridArgs a, int G, int *dev_status, int64_t *done,
                     cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr) {
    const cudaStream_t st = h->stream;
    (void)G;
    CK(cudaMemsetAsync(h->acc, 0, sizeof(double) * 6 * (size_t)h->acc_r * h->acc_w, st));
    CK(cudaMemsetAsync(h->ws, 0, sizeof(Workspace), st));
    if (!e0) {
        e0 = h->kev0;
        e1 = h->kev1;
    }
    CK(cudaEventRecord(e0, st));
    CK(launch_grid(mode, a, G, st));
    CK(cudaEventRecord(e1, st));
    ++h->launches;
    ++h->grid_launches;
    Workspace w;
    CK(cudaMemcpyAsync(&w, h->ws, sizeof(Workspace), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float kms = 0.f;
    CK(cudaEventElapsedTime(&kms, e0, e1));
    h->kernel_ms += kms;
    *dev_status = w.status;
    *done = w.iters_done;
    return REBK_OK;
}

int pick_ctas(rebk_handle h, Mode mode);

rebk_status check_smem(rebk_handle h, Mode mode, int G) {
    GridArgs a = base_args(h, mode, G);
    const size_t smem = grid_smem_bytes(mode, a);
    if (smem > kSmemLimit)
        return fail(REBK_EUNSUPPORTED, "problem too large for the persistent kernel's shared memory "
                                       "(owned slices of m + n per CTA)");
    return REBK_OK;
}

// CTA count of the persistent kernel: the caller's, else the fastest of a few
// candidates on a short timed run over zero data (same work as a real run).
int pick_ctas(rebk_handle h, Mode mode) {
    const int mi = mode_index(mode);
    if (h->G[mi] > 0) return h->G[mi];
    int maxG = grid_max_ctas(mode, grid_smem_bytes(mode, base_args(h, mode, 16)));
    if (maxG <= 0) maxG = 1;
    if (h->num_ctas_opt > 0) {
        h->G[mi] = std::min(h->num_ctas_opt, maxG);
        return h->G[mi];
    }
    std::vector<int> cands;
    for (int c : {8, 16, 32, 48, 64, 96, 128}) if (c < maxG) cands.push_back(c);
    cands.push_back(maxG);
    // zero state and right-hand side in scratch buffers
    const cudaStream_t st = h->stream;
    void *zs = mode == Mode::PlainF64 ? (void *)h->zbuf : (void *)h->dz;
    void *xs = mode == Mode::PlainF64 ? (void *)h->yn : (void *)h->dx;
    cudaMemsetAsync(h->ym, 0, sizeof(double) * h->m, st);
    cudaMemsetAsync(h->g, 0, sizeof(double) * h->n, st);
    cudaMemsetAsync(zs, 0, (mode == Mode::PlainF64 ? 8 : 4) * h->m, st);
    cudaMemsetAsync(xs, 0, (mode == Mode::PlainF64 ? 8 : 4) * h->n, st);
    cudaMemsetAsync(h->sd, 0, 4 * h->n, st);
    cudaMemsetAsync(h->vd, 0, 4 * h->m, st);
    const int64_t iters = 48;
    float best = 1e30f;
    int bestG = cands.back();
    for (int G : cands) {
        if (check_smem(h, mode, G) != REBK_OK) continue;
        GridArgs a = base_args(h, mode, G);
        a.seed = 1;
        if (sample_into(h, a, 0, iters, nullptr) != REBK_OK) break;
        a.z = zs;
        a.x = xs;
        a.beta = h->ym;
        a.gamma = mode == Mode::PlainF64 ? nullptr : h->g;
        a.sdual = h->sd;
        a.vdual = h->vd;
        float tbest = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            int ds;
            int64_t done;
            if (run_grid(h, mode, a, G, &ds, &done, h->ev0, h->ev1) != REBK_OK || ds != 0) {
                tbest = 1e30f;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, h->ev0, h->ev1);
            tbest = std::min(tbest, ms);
        }
        if (tbest < best) {
            best = tbest;
            bestG = G;
        }
    }
    cudaGetLastError();
    h->G[mi] = bestG;
    return bestG;
}

void reset_counters(rebk_handle h) {
    h->launches = 0;
    h->grid_launches = 0;
    h->kernel_ms = 0.0;
    h->sweep_used = 0;
}

// FP64 sweep with its CUDA-event time recorded for the stats.
rebk_status timed_sweep(rebk_handle h, const void *p, bool p_f32, const void *q, bool q_f32,
                        double *ym, double *yn) {
    if (h->sweep_used + 2 > h->sweep_ev.size()) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            h->sweep_ev.push_back(e);
        }
    }
    cudaEvent_t e0 = h->sweep_ev[h->sweep_used], e1 = h->sweep_ev[h->sweep_used + 1];
    h->sweep_used += 2;
    CK(cudaEventRecord(e0, h->stream));
    LK(h, dual_sweep(h->A64, h->lda, h->m, h->n, p, p_f32, q, q_f32, ym, yn, h->stream));
    CK(cudaEventRecord(e1, h->stream));
    return REBK_OK;
}

double sweep_time(rebk_handle h) {
    double tot = 0.0;
    for (size_t i = 0; i + 1 < h->sweep_used; i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->sweep_ev[i], h->sweep_ev[i + 1]) == cudaSuccess) tot += ms;
    }
    return tot;
}

rebk_status fetch_small(rebk_handle h, double *host, int count) {
    CK(cudaMemcpyAsync(host, h->ws->small, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return REBK_OK;
}

// ||b - z - A x|| / ||b|| and ||A^T z|| / (||A||_F ||b||) in FP64.
rebk_status residuals(rebk_handle h, const double *b, const double *x, const double *z, double *rf,
                      double *rg) {
    const cudaStream_t st = h->stream;
    rebk_status ts = timed_sweep(h, x, false, z, false, h->ym, h->yn);
    if (ts != REBK_OK) return ts;
    LK(h, form_f(b, z, h->ym, h->f, h->m, st));
    LK(h, sum_sq(h->f, h->m, h->ws->small, st));
    LK(h, sum_sq(h->yn, h->n, h->ws->small + 2, st));
    LK(h, sum_sq(b, h->m, h->ws->small + 4, st));
    double v[6];
    rebk_status s = fetch_small(h, v, 6);
    if (s != REBK_OK) return s;
    const double nb = std::sqrt(v[5]);
    *rf = nb > 0 ? std::sqrt(v[1]) / nb : 0.0;
    *rg = nb > 0 ? std::sqrt(v[3]) / (std::sqrt(h->fro2) * nb) : 0.0;
    return REBK_OK;
}

rebk_status rel_error(rebk_handle h, const double *x, const double *xref, double *rel) {
    LK(h, err_norms(nullptr, x, xref, h->n, h->ws->small, h->stream));
    double v[2];
    rebk_status s = fetch_small(h, v, 2);
    if (s != REBK_OK) return s;
    *rel = v[1] > 0 ? std::sqrt(v[0] / v[1]) : std::sqrt(v[0]);
    return REBK_OK;
}

void fill_stats(rebk_handle h, rebk_stats *st, int64_t iters, int outer, rebk_status status,
                double rel, double rf, double rg, double ms) {
    if (!st) return;
    st->kernel_ms = h->kernel_ms;
    st->sweep_ms = sweep_time(h);
    st->launches = h->launches;
    st->grid_launches = h->grid_launches;
    st->iterations = iters;
    st->outer = outer;
    st->status = status;
    st->rel_err = rel;
    st->resid_f = rf;
    st->resid_g = rg;
    st->device_ms = ms;
}

// Checks one side of a partition: off[0] = 0 < off[1] < ... < off[nb] = size,
// every block at most 512 long.  Fills the host copy and the largest block.
rebk_status check_offsets(const int64_t *off, int64_t nb, int64_t size, const char *what,
                          std::vector<int64_t> *copy, int64_t *tau) {
    if (nb < 1 || nb > ((int64_t)1 << 30)) return fail(REBK_EINVAL, std::string(what) + ": block count out of range");
    if (off[0] != 0 || off[nb] != size)
        return fail(REBK_EINVAL, std::string(what) + ": offsets must run from 0 to the dimension");
    int64_t big = 0;
    for (int64_t b = 0; b < nb; ++b) {
        if (off[b + 1] <= off[b]) return fail(REBK_EINVAL, std::string(what) + ": offsets must increase strictly");
        big = std::max(big, off[b + 1] - off[b]);
    }
    if (big > 512) return fail(REBK_EUNSUPPORTED, std::string(what) + ": a block larger than 512");
    copy->assign(off, off + nb + 1);
    *tau = big;
    return REBK_OK;
}


// Launch geometry of the multi-right-hand-side kernel: every SM (or the
// handle's CTA count), the owned slices and TMA tiles of the one-right-hand-side
// kernel, and the largest group (8, else 4; or `want`) whose tiles fit in shared
// memory, with the rest of shared memory as the reduction scratch.
rebk_status multi_setup(rebk_handle h, Mode mode, int want, MultiArgs *Mout, int *Gout, int *nrout) {
    const bool bf16 = mode == Mode::CorrBF16;
    int dev = 0, sms = 1;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int G = h->num_ctas_opt > 0 ? std::min(sms, h->num_ctas_opt) : sms;
    MultiArgs M;
    memset(&M, 0, sizeof(M));
    GridArgs &a = M.geo;
    a.A = bf16 ? (const void *)h->A16 : (const void *)h->A32;
    a.lda = h->lda;
    a.m = h->m;
    a.n = h->n;
    a.tau_r = h->tau_r;
    a.tau_c = h->tau_c;
    a.s = h->s;
    a.t = h->t;
    a.row_off = h->d_row_off;
    a.col_off = h->d_col_off;
    a.col_align = h->col_align;
    a.coef_r = h->coef_r32;
    a.coef_c = h->coef_c32;
    a.nrow_cap = (int)((h->m + G - 1) / G);
    a.ncol_cap = (int)std::min<int64_t>(8 * (((h->n + 7) / 8 + G - 1) / G), h->n);
    a.bar = &h->ws->bar;
    a.status = &h->ws->status;
    a.iters_done = &h->ws->iters_done;
    a.timeout_ns = kBarrierTimeoutNs;
    if (!tma_geometry(mode, a))
        return fail(REBK_EUNSUPPORTED, "multi-right-hand-side form: a tile is wider or taller than 256 "
                                       "(tau or the owned column slice)");
    a.use_tma = 1;
    const GridArgs plain = a;
    // Tensor-core geometry (FP32 storage, groups of 8): column-tile rows 4 floats off a
    // multiple of 32 bytes and row-tile rows 8 floats off a multiple of 64 bytes, so
    // the fragment loads of the products hit distinct banks; each tile buffer keeps
    // slack for the reads past the box that the 16 x 8 fragments make.
    auto mma_geometry = [&](GridArgs &g) {
        if (g.bw_c % 8 == 0) g.bw_c += 4;
        if (g.bw_r % 8 != 0) g.bw_r += 8 - g.bw_r % 8;
        if (g.bw_r % 16 == 0) g.bw_r += 8;
        if (g.bw_c > 256 || g.bw_r > 256) return false;
        const int64_t es = 4;
        g.tile_c_bytes_tx = (int64_t)g.nbox_c * g.bh_c * g.bw_c * es;
        g.tile_r_bytes_tx = (int64_t)g.tau_r * g.bw_r * es;
        const int64_t rows_c = std::max<int64_t>((int64_t)g.nbox_c * g.bh_c, (g.nrow_cap + 15) / 16 * 16);
        const int64_t rows_r = (g.tau_r + 15) / 16 * 16;
        g.tile_c_bytes = (rows_c * g.bw_c * es + 256 + 127) / 128 * 128;
        g.tile_r_bytes = (rows_r * g.bw_r * es + 256 + 127) / 128 * 128;
        return true;
    };
    struct Cand { int nr; bool mma; };
    const Cand cands[] = {{8, true}, {8, false}, {4, false}};
    int nr = 0;
    for (const Cand &c : cands) {
        if (want != 0 && c.nr != want) continue;
        if (c.mma && bf16) continue;
        a = plain;
        M.mma = 0;
        if (c.mma) {
            if (!mma_geometry(a)) continue;
            M.mma = 1;
        }
        if (tma_encode(mode, a) != cudaSuccess) continue;
        M.scr_floats = 0;
        const size_t base = multi_smem_bytes(M, c.nr);
        if (base + 128 > kSmemLimit) continue;
        M.scr_floats = (int)std::min<size_t>((kSmemLimit - base - 128) / 4 / 32 * 32, (size_t)512 * c.nr);
        // the two products of a stage accumulate side by side in the scratch
        auto r16 = [](int v) { return (v + 15) / 16 * 16; };
        if (c.mma && M.scr_floats < 8 * std::max(r16(a.ncol_cap) + r16(a.nrow_cap), r16(a.tau_r) + r16(a.tau_c)))
            continue;
        const size_t smem = multi_smem_bytes(M, c.nr);
        if (smem > kSmemLimit || multi_max_ctas(bf16, c.nr, c.mma, smem) < G) continue;
        nr = c.nr;
        break;
    }
    if (nr == 0)
        return fail(REBK_EUNSUPPORTED, "multi-right-hand-side form: no tensor map, or the tiles do not fit in "
                                       "shared memory");
    *Mout = M;
    *Gout = G;
    *nrout = nr;
    return REBK_OK;
}
}  // namespace

namespace rebk {
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace rebk

// ===========================================================================
extern "C" {

const char *rebk_last_error(void) { return g_last_error.c_str(); }

const char *rebk_version(void) { return "rebk-gb300 0.1 (sm_103a)"; }

void rebk_destroy(rebk_handle h) { free_handle(h); }

rebk_status rebk_create(rebk_handle *out, const double *A, int64_t m, int64_t n, int64_t lda,
                                   int A_on_device, const rebk_partition *part, double alpha,
                                   const rebk_options *opt) {
    g_last_error.clear();
    if (!out) return fail(REBK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!A) return fail(REBK_EINVAL, "A is NULL");
    if (m < 1 || n < 1) return fail(REBK_EINVAL, "m and n must be >= 1");
    if (lda < n) return fail(REBK_EINVAL, "lda must be >= n");
    if (m > (int64_t)1 << 30 || n > (int64_t)1 << 30) return fail(REBK_EUNSUPPORTED, "m, n > 2^30");
    if (!std::isfinite(alpha)) return fail(REBK_EINVAL, "alpha is not finite");
    rebk_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.tau_row < 0 || o.tau_col < 0) return fail(REBK_EINVAL, "tau must be >= 1 (0 = default)");
    if (o.tau_row == 0) o.tau_row = std::min<int64_t>(m, 64);
    if (o.tau_col == 0) o.tau_col = std::min<int64_t>(n, 64);
    o.tau_row = std::min(o.tau_row, m);
    o.tau_col = std::min(o.tau_col, n);
    std::vector<int64_t> roff, coff;
    if (part && part->row_off) {
        rebk_status ps = check_offsets(part->row_off, part->s, m, "row partition", &roff, &o.tau_row);
        if (ps != REBK_OK) return ps;
    }
    if (part && part->col_off) {
        rebk_status ps = check_offsets(part->col_off, part->t, n, "column partition", &coff, &o.tau_col);
        if (ps != REBK_OK) return ps;
    }
    if (o.tau_row > 512 || o.tau_col > 512) return fail(REBK_EUNSUPPORTED, "tau > 512");
    if (o.check_every < 0) return fail(REBK_EINVAL, "check_every < 0");
    if (o.num_ctas < 0) return fail(REBK_EINVAL, "num_ctas < 0");
    if (o.storage_mask & ~((1 << REBK_FP32) | (1 << REBK_BF16) | 1))
        return fail(REBK_EINVAL, "unknown bits in storage_mask");

    rebk_handle h = new rebk_handle_s();
    h->stream = static_cast<cudaStream_t>(o.stream);
    h->m = m;
    h->n = n;
    h->lda = round_up(n, 64);
    h->tau_r = (int)o.tau_row;
    h->tau_c = (int)o.tau_col;
    h->s = roff.empty() ? (int)((m + h->tau_r - 1) / h->tau_r) : (int)(roff.size() - 1);
    h->t = coff.empty() ? (int)((n + h->tau_c - 1) / h->tau_c) : (int)(coff.size() - 1);
    if (roff.empty())
        for (int64_t b = 0; b <= h->s; ++b) h->row_off.push_back(std::min<int64_t>(m, b * h->tau_r));
    else
        h->row_off = roff;
    if (coff.empty())
        for (int64_t b = 0; b <= h->t; ++b) h->col_off.push_back(std::min<int64_t>(n, b * h->tau_c));
    else
        h->col_off = coff;
    if (!coff.empty()) {  // largest power of two (<= 16) dividing every column-block start
        int al = 16;
        for (int64_t v : coff)
            while (al > 1 && v % al != 0) al >>= 1;
        h->col_align = al;
    }
    h->check_every = o.check_every;
    h->num_ctas_opt = o.num_ctas;
    h->acc_w = (int)round_up(std::max(h->tau_c, h->tau_r + 1), 32);
    const cudaStream_t st = h->stream;

#define CKH(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess) {                                                                  \
            rebk_status s__ = cuda_fail(e__, #call);                                               \
            free_handle(h);                                                                        \
            return s__;                                                                            \
        }                                                                                          \
    } while (0)

    CKH(cudaGetDevice(&h->device));
    if (!roff.empty()) {
        CKH(cudaMalloc(&h->d_row_off, sizeof(int64_t) * roff.size()));
        CKH(cudaMemcpy(h->d_row_off, roff.data(), sizeof(int64_t) * roff.size(), cudaMemcpyHostToDevice));
    }
    if (!coff.empty()) {
        CKH(cudaMalloc(&h->d_col_off, sizeof(int64_t) * coff.size()));
        CKH(cudaMemcpy(h->d_col_off, coff.data(), sizeof(int64_t) * coff.size(), cudaMemcpyHostToDevice));
    }
    CKH(cudaEventCreate(&h->ev0));
    CKH(cudaEventCreate(&h->ev1));
    CKH(cudaEventCreate(&h->kev0));
    CKH(cudaEventCreate(&h->kev1));
    const size_t nA = (size_t)m * h->lda;
    CKH(cudaMalloc(&h->A64, nA * sizeof(double)));
    CKH(cudaMemcpy2DAsync(h->A64, h->lda * sizeof(double), A, lda * sizeof(double), n * sizeof(double),
                          m, A_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (h->lda > n)
        CKH(cudaMemset2DAsync(h->A64 + n, h->lda * sizeof(double), 0, (h->lda - n) * sizeof(double), m,
                              st));
    if (o.storage_mask & (1 << REBK_FP32)) {
        CKH(cudaMalloc(&h->A32, nA * sizeof(float)));
        CKH(convert_storage(h->A64, h->lda, h->A32, h->lda, m, n, 1, st));
    }
    if (o.storage_mask & (1 << REBK_BF16)) {
        CKH(cudaMalloc(&h->A16, nA * sizeof(__nv_bfloat16)));
        CKH(convert_storage(h->A64, h->lda, h->A16, h->lda, m, n, 2, st));
    }
    CKH(cudaMalloc(&h->nr, sizeof(double) * h->s));
    CKH(cudaMalloc(&h->cdf_r, sizeof(double) * h->s));
    CKH(cudaMalloc(&h->nc, sizeof(double) * h->t));
    CKH(cudaMalloc(&h->cdf_c, sizeof(double) * h->t));
    CKH(cudaMalloc(&h->d_fallback, sizeof(int) * 2));
    {
        double *scratch = nullptr;
        CKH(cudaMalloc(&scratch, sizeof(double) * (size_t)(m + n + 64 * n)));
        cudaError_t e = block_tables(h->A64, h->lda, m, n, h->tau_r, h->tau_c, h->s, h->t, h->nr, h->nc,
                                     h->cdf_r, h->cdf_c, h->d_fallback, scratch, st, h->d_row_off, h->d_col_off);
        cudaError_t e2 = cudaStreamSynchronize(st);
        cudaFree(scratch);
        CKH(e);
        CKH(e2);
    }
    CKH(cudaMemcpy(h->fb, h->d_fallback, sizeof(int) * 2, cudaMemcpyDeviceToHost));
    CKH(cudaMemcpy(&h->fro2, h->cdf_r + (h->s - 1), sizeof(double), cudaMemcpyDeviceToHost));
    CKH(cudaMalloc(&h->acc, sizeof(double) * 6 * (size_t)h->acc_r * h->acc_w));
    CKH(cudaMalloc(&h->coef_r64, sizeof(double) * h->s));
    CKH(cudaMalloc(&h->coef_c64, sizeof(double) * h->t));
    CKH(cudaMalloc(&h->coef_r32, sizeof(float) * h->s));
    CKH(cudaMalloc(&h->coef_c32, sizeof(float) * h->t));
    CKH(cudaMalloc(&h->ws, sizeof(Workspace)));
    CKH(cudaMalloc(&h->zbuf, sizeof(double) * m));
    CKH(cudaMalloc(&h->f, sizeof(double) * m));
    CKH(cudaMalloc(&h->ym, sizeof(double) * m));
    CKH(cudaMalloc(&h->g, sizeof(double) * n));
    CKH(cudaMalloc(&h->yn, sizeof(double) * n));
    CKH(cudaMalloc(&h->dz, sizeof(float) * m));
    CKH(cudaMalloc(&h->vd, sizeof(float) * m));
    CKH(cudaMalloc(&h->dx, sizeof(float) * n));
    CKH(cudaMalloc(&h->sd, sizeof(float) * n));
#undef CKH
    if (alpha > 0.0) {
        h->alpha = alpha;
    } else if (h->fro2 > 0.0) {
        double br, bc;
        rebk_status s = rebk_beta_max(h, &br, &bc);
        if (s != REBK_OK) {
            free_handle(h);
            return s;
        }
        h->alpha = 1.75 / std::max(br, bc);
    } else {
        h->alpha = 1.0;
    }
    {
        cudaError_t e1 = step_coefficients(h->nr, h->s, h->alpha, h->coef_r64, h->coef_r32, st);
        cudaError_t e2 = step_coefficients(h->nc, h->t, h->alpha, h->coef_c64, h->coef_c32, st);
        cudaError_t e3 = cudaStreamSynchronize(st);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            rebk_status s = cuda_fail(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "step coefficients");
            free_handle(h);
            return s;
        }
    }
    *out = h;
    return REBK_OK;
}

rebk_status rebk_beta_max(rebk_handle h, double *beta_row, double *beta_col) {
    if (!h) return fail(REBK_EINVAL, "handle is NULL");
    if (!h->beta_done) {
        const cudaStream_t st = h->stream;
        const size_t gsz = std::max((size_t)h->s * h->tau_r * h->tau_r, (size_t)h->t * h->tau_c * h->tau_c);
        double *gram = nullptr, *br = nullptr, *bc = nullptr;
        CK(cudaMalloc(&gram, sizeof(double) * gsz));
        CK(cudaMalloc(&br, sizeof(double) * h->s));
        CK(cudaMalloc(&bc, sizeof(double) * h->t));
        cudaError_t e = beta_max_device(h->A64, h->lda, h->m, h->n, h->tau_r, h->tau_c, h->s, h->t, h->nr,
                                        h->nc, gram, br, bc, st, h->d_row_off, h->d_col_off);
        std::vector<double> hr(h->s), hc(h->t);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hr.data(), br, sizeof(double) * h->s, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), bc, sizeof(double) * h->t, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(gram);
        cudaFree(br);
        cudaFree(bc);
        if (e != cudaSuccess) return cuda_fail(e, "beta_max");
        h->beta_r = *std::max_element(hr.begin(), hr.end());
        h->beta_c = *std::max_element(hc.begin(), hc.end());
        h->beta_done = true;
    }
    if (beta_row) *beta_row = h->beta_r;
    if (beta_col) *beta_col = h->beta_c;
    return REBK_OK;
}

rebk_status rebk_get_alpha(rebk_handle h, double *alpha) {
    if (!h || !alpha) return fail(REBK_EINVAL, "NULL argument");
    *alpha = h->alpha;
    return REBK_OK;
}

rebk_status rebk_set_alpha(rebk_handle h, double alpha) {
    g_last_error.clear();
    if (!h) return fail(REBK_EINVAL, "handle is NULL");
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(REBK_EINVAL, "alpha must be finite and > 0");
    const cudaStream_t st = h->stream;
    cudaError_t e = step_coefficients(h->nr, h->s, alpha, h->coef_r64, h->coef_r32, st);
    if (e == cudaSuccess) e = step_coefficients(h->nc, h->t, alpha, h->coef_c64, h->coef_c32, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "step coefficients");
    h->alpha = alpha;
    for (int i = 0; i < 3; ++i) h->prepG[i] = 0;  // launch arguments carry alpha
    return REBK_OK;
}

rebk_status rebk_spectral_estimates(rebk_handle h, int32_t steps, uint64_t seed, rebk_spectrum *out) {
    g_last_error.clear();
    if (!h || !out) return fail(REBK_EINVAL, "NULL argument");
    if (steps < 1 || steps > 2048) return fail(REBK_EINVAL, "steps must be in [1, 2048]");
    memset(out, 0, sizeof(*out));
    out->fro2 = h->fro2;
    if (h->fro2 == 0.0) return REBK_OK;  // A = 0: no nonzero singular value
    double s1 = 0.0, sr = 0.0;
    int done = 0;
    cudaError_t e = lanczos_extremes(h->A64, h->lda, h->m, h->n, steps, seed, h->stream, &s1, &sr, &done);
    if (e != cudaSuccess) return cuda_fail(e, "Lanczos bidiagonalisation");
    double br = 0.0, bc = 0.0;
    rebk_status s = rebk_beta_max(h, &br, &bc);
    if (s != REBK_OK) return s;
    const double F = h->fro2, a = h->alpha;
    out->sigma1_sq = s1;
    out->sigma_r_sq = sr;
    out->steps = done;
    out->alpha_mean_opt = 2.0 * F / (s1 + sr);
    out->delta_opt = (s1 - sr) / (s1 + sr);
    out->alpha = a;
    out->delta = std::max(std::fabs(1.0 - a * s1 / F), std::fabs(1.0 - a * sr / F));
    out->beta_row = br;
    out->beta_col = bc;
    out->eta = 1.0 - (2.0 * a - a * a * br) * sr / F;
    out->rho = 1.0 - (2.0 * a - a * a * bc) * sr / F;
    return REBK_OK;
}

rebk_status rebk_get_blocks(rebk_handle h, int64_t *s, int64_t *t) {
    if (!h) return fail(REBK_EINVAL, "handle is NULL");
    if (s) *s = h->s;
    if (t) *t = h->t;
    return REBK_OK;
}

rebk_status rebk_get_partition(rebk_handle h, int64_t *row_off, int64_t *col_off, int64_t *tau_row,
                               int64_t *tau_col) {
    if (!h) return fail(REBK_EINVAL, "handle is NULL");
    if (row_off) std::copy(h->row_off.begin(), h->row_off.end(), row_off);
    if (col_off) std::copy(h->col_off.begin(), h->col_off.end(), col_off);
    if (tau_row) *tau_row = h->tau_r;
    if (tau_col) *tau_col = h->tau_c;
    return REBK_OK;
}

rebk_status rebk_get_tables(rebk_handle h, double *nr, double *nc, double *cdf_r, double *cdf_c) {
    if (!h) return fail(REBK_EINVAL, "handle is NULL");
    if (nr) CK(cudaMemcpy(nr, h->nr, sizeof(double) * h->s, cudaMemcpyDeviceToHost));
    if (nc) CK(cudaMemcpy(nc, h->nc, sizeof(double) * h->t, cudaMemcpyDeviceToHost));
    if (cdf_r) CK(cudaMemcpy(cdf_r, h->cdf_r, sizeof(double) * h->s, cudaMemcpyDeviceToHost));
    if (cdf_c) CK(cudaMemcpy(cdf_c, h->cdf_c, sizeof(double) * h->t, cudaMemcpyDeviceToHost));
    return REBK_OK;
}

rebk_status rebk_export_storage(rebk_handle h, int32_t storage, void *host_out) {
    if (!h || !host_out) return fail(REBK_EINVAL, "NULL argument");
    const void *src = storage == REBK_FP64 ? (const void *)h->A64
                      : storage == REBK_FP32 ? (const void *)h->A32
                      : storage == REBK_BF16 ? (const void *)h->A16 : nullptr;
    if (!src) return fail(REBK_EINVAL, "storage not kept by this handle");
    const size_t es = storage == REBK_FP64 ? 8 : (storage == REBK_FP32 ? 4 : 2);
    CK(cudaMemcpy2D(host_out, h->n * es, src, h->lda * es, h->n * es, h->m, cudaMemcpyDeviceToHost));
    return REBK_OK;
}

rebk_status rebk_solve_ex(rebk_handle h, const double *b, double *x, double tol, int64_t max_iter,
                          uint64_t seed, const rebk_solve_ext *ext, rebk_stats *stats) {
    g_last_error.clear();
    if (!h) return fail(REBK_EINVAL, "handle is NULL");
    if (!b || !x) return fail(REBK_EINVAL, "b and x must be device pointers");
    if (max_iter < 0) return fail(REBK_EINVAL, "max_iter < 0");
    if (!std::isfinite(tol)) return fail(REBK_EINVAL, "tol is not finite");
    rebk_solve_ext e;
    memset(&e, 0, sizeof(e));
    if (ext) e = *ext;
    if (e.k0 < 0) return fail(REBK_EINVAL, "k0 < 0");
    const cudaStream_t st = h->stream;
    double *z = e.z_out ? e.z_out : h->zbuf;
    const Mode mode = Mode::PlainF64;
    // the CTA-count choice runs timed launches on scratch buffers: before any state is set
    const int G = (h->fro2 == 0.0 || max_iter == 0) ? 1 : pick_ctas(h, mode);
    reset_counters(h);

    CK(cudaEventRecord(h->ev0, st));
    if (e.z0) {
        if (e.z0 != z) CK(cudaMemcpyAsync(z, e.z0, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    } else {
        CK(cudaMemcpyAsync(z, b, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    }
    if (e.x0) {
        if (e.x0 != x) CK(cudaMemcpyAsync(x, e.x0, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, st));
    } else {
        CK(cudaMemsetAsync(x, 0, sizeof(double) * h->n, st));
    }
    if (h->fro2 == 0.0 || max_iter == 0) {
        // A = 0: A^+ b = 0 and Algorithm 1 cannot move.
        CK(cudaStreamSynchronize(st));
        double rel = -1;
        if (e.x_ref) {
            rebk_status s = rel_error(h, x, e.x_ref, &rel);
            if (s != REBK_OK) return s;
        }
        fill_stats(h, stats, 0, 0, REBK_OK, rel, -1, -1, 0.0);
        return REBK_OK;
    }
    rebk_status s = check_smem(h, mode, G);
    if (s != REBK_OK) return s;

    GridArgs a = base_args(h, mode, G);
    a.seed = seed;
    a.stream = e.stream_id;
    a.z = z;
    a.x = x;
    a.beta = b;
    a.gamma = nullptr;

    double ref2 = 0.0;
    const bool use_ref = e.x_ref != nullptr;
    int64_t check = h->check_every;
    if (use_ref) {
        LK(h, sum_sq(e.x_ref, h->n, h->ws->small, st));
        double v[2];
        s = fetch_small(h, v, 2);
        if (s != REBK_OK) return s;
        ref2 = v[1];
        if (check <= 0) check = 10;
        a.x_ref = tol > 0 ? e.x_ref : nullptr;
        a.x_base = nullptr;
        a.tol2_abs = tol * tol * ref2;
        a.check_every = check;
    } else if (tol > 0) {
        if (check <= 0) {
            const double per_iter = (double)h->tau_r * h->n + (double)h->tau_c * h->m;
            check = std::max<int64_t>(50, (int64_t)(20.0 * (double)h->m * h->n / per_iter));
        }
    }

    int64_t total = 0;
    int dev_status = 0;
    rebk_status result = REBK_MAX_ITER;
    double rf = -1, rg = -1, rel = -1;
    int64_t grow = 16384;
    while (total < max_iter) {
        int64_t chunk = max_iter - total;
        if (!use_ref && tol > 0) chunk = std::min(chunk, check);
        chunk = std::min(chunk, e.idx_out ? kMaxItersPerLaunch : kIdxChunkMax);
        if (use_ref && tol > 0) {  // early stop likely: sample in growing chunks
            chunk = std::min(chunk, grow);
            grow = std::min<int64_t>(grow * 2, kIdxChunkMax);
        }
        s = sample_into(h, a, e.k0 + total, chunk, e.idx_out ? e.idx_out + 2 * total : nullptr);
        if (s != REBK_OK) return s;
        a.check_offset = total;
        int64_t done = 0;
        s = run_grid(h, mode, a, G, &dev_status, &done);
        if (s != REBK_OK) return s;
        total += done;
        if (dev_status == 6) {
            fill_stats(h, stats, total, 0, REBK_BARRIER_TIMEOUT, -1, -1, -1, 0);
            return fail(REBK_BARRIER_TIMEOUT, "device-wide barrier timed out");
        }
        if (dev_status == 5) {
            result = REBK_DIVERGED;
            break;
        }
        if (use_ref) {
            if (done < chunk) {  // stopped by the error test
                result = REBK_OK;
                break;
            }
            // the kernel does not test the last iterate of a launch: do it here
            if (tol > 0 && total % check == 0) {
                s = rel_error(h, x, e.x_ref, &rel);
                if (s != REBK_OK) return s;
                if (rel <= tol) {
                    result = REBK_OK;
                    break;
                }
            }
        } else if (tol > 0) {
            s = residuals(h, b, x, z, &rf, &rg);
            if (s != REBK_OK) return s;
            if (std::max(rf, rg) <= tol) {
                result = REBK_OK;
                break;
            }
        }
    }
    CK(cudaEventRecord(h->ev1, st));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    if (use_ref) {
        s = rel_error(h, x, e.x_ref, &rel);
        if (s != REBK_OK) return s;
        if (result == REBK_MAX_ITER && tol > 0 && rel <= tol) result = REBK_OK;
    }
    if (tol <= 0 && result == REBK_MAX_ITER) result = REBK_OK;
    fill_stats(h, stats, total, 0, result, rel, rf, rg, ms);
    if (result == REBK_DIVERGED) return fail(REBK_DIVERGED, "iteration diverged (Inf/NaN)");
    return result;
}

rebk_status rebk_warm_start(rebk_handle h, rebk_mlp net, const double *b, double *x0, double *z0) {
    g_last_error.clear();
    if (!h || !net || !b || !x0 || !z0) return fail(REBK_EINVAL, "NULL argument");
    int64_t nm = 0, nn = 0;
    rebk_status s = rebk_mlp_shape(net, &nm, &nn);
    if (s != REBK_OK) return s;
    if (nm != h->m || nn != h->n) return fail(REBK_EINVAL, "network shape does not match the solver's A");
    const cudaStream_t st = h->stream;
    CK(cudaStreamSynchronize(st));
    s = rebk_mlp_forward(net, b, 1, h->ym);  // y (length m) in the handle's scratch
    if (s != REBK_OK) return s;
    // x0 = A^T y and A x0 with the FP64 copy of A; z0 = b - A x0
    CK(dual_sweep(h->A64, h->lda, h->m, h->n, nullptr, false, h->ym, false, nullptr, x0, st));
    CK(dual_sweep(h->A64, h->lda, h->m, h->n, x0, false, nullptr, false, h->f, nullptr, st));
    CK(vec_sub(b, h->f, z0, h->m, st));
    CK(cudaStreamSynchronize(st));
    return REBK_OK;
}

rebk_status rebk_warm_start_batch(rebk_handle h, rebk_mlp net, const double *B, int64_t count, int32_t group,
                                  double *X0, double *Z0) {
    g_last_error.clear();
    if (!h || !net || !B || !X0 || !Z0) return fail(REBK_EINVAL, "NULL argument");
    if (count < 1 || group < 1 || count % group != 0) return fail(REBK_EINVAL, "count must be a positive multiple of group");
    int64_t nm = 0, nn = 0;
    rebk_status s = rebk_mlp_shape(net, &nm, &nn);
    if (s != REBK_OK) return s;
    if (nm != h->m || nn != h->n) return fail(REBK_EINVAL, "network shape does not match the solver's A");
    const int64_t cap = mlp_batch_capacity(net);
    const cudaStream_t st = h->stream;
    const int64_t chunk = std::min<int64_t>(cap, count);
    double *Bc = nullptr, *Yc = nullptr, *Xc = nullptr;
    cudaError_t ae = cudaMalloc(&Bc, sizeof(double) * chunk * h->m);
    if (ae == cudaSuccess) ae = cudaMalloc(&Yc, sizeof(double) * chunk * h->m);
    if (ae == cudaSuccess) ae = cudaMalloc(&Xc, sizeof(double) * chunk * h->n);
    auto release = [&]() {
        if (Bc) cudaFree(Bc);
        if (Yc) cudaFree(Yc);
        if (Xc) cudaFree(Xc);
    };
    if (ae != cudaSuccess) {
        release();
        return fail(ae == cudaErrorMemoryAllocation ? REBK_ENOMEM : REBK_ECUDA, cudaGetErrorString(ae));
    }
    rebk_status out = REBK_OK;
    for (int64_t j0 = 0; j0 < count && out == REBK_OK; j0 += chunk) {
        const int64_t cnt = std::min(chunk, count - j0);
        cudaError_t e = group_gather(B, j0, cnt, group, h->m, Bc, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the network may run on another stream
        if (e == cudaSuccess) {
            out = rebk_mlp_forward(net, Bc, cnt, Yc);  // y for the chunk (rows of m)
            if (out != REBK_OK) break;
        }
        // x0 = A^T y (rows: X0c = Yc A) and A x0 (rows: Yc <- X0c A^T) with the FP64 copy of A,
        // then z0 = b - A x0, stored in the grouped layouts
        if (e == cudaSuccess) e = dgemm((int)cnt, (int)h->n, (int)h->m, Yc, h->m, 1, h->A64, h->lda, 1, Xc, h->n, st);
        if (e == cudaSuccess) e = dgemm((int)cnt, (int)h->m, (int)h->n, Xc, h->n, 1, h->A64, 1, h->lda, Yc, h->m, st);
        if (e == cudaSuccess) e = group_store_xz_many(Xc, h->n, Bc, Yc, h->m, j0, cnt, group, X0, Z0, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) out = fail(REBK_ECUDA, cudaGetErrorString(e));
    }
    release();
    return out;
}

rebk_status rebk_solve(rebk_handle h, const double *b, double *x, double tol, int64_t max_iter,
                       uint64_t seed, rebk_stats *stats) {
    return rebk_solve_ex(h, b, x, tol, max_iter, seed, nullptr, stats);
}

rebk_status rebk_solve_refined(rebk_handle h, const double *b, double *x, double tol,
                               int64_t max_iter, uint64_t seed, const rebk_refine_opts *ropt,
                               const rebk_solve_ext *ext, rebk_stats *stats) {
    g_last_error.clear();
    if (!h) return fail(REBK_EINVAL, "handle is NULL");
    if (!b || !x) return fail(REBK_EINVAL, "b and x must be device pointers");
    if (max_iter < 0) return fail(REBK_EINVAL, "max_iter < 0");
    if (!std::isfinite(tol)) return fail(REBK_EINVAL, "tol is not finite");
    rebk_refine_opts ro;
    memset(&ro, 0, sizeof(ro));
    ro.storage = REBK_FP32;
    if (ropt) ro = *ropt;
    Mode mode;
    if (ro.storage == REBK_FP32) {
        if (!h->A32) return fail(REBK_EINVAL, "FP32 copy not kept (storage_mask)");
        mode = Mode::CorrF32;
    } else if (ro.storage == REBK_BF16) {
        if (!h->A16) return fail(REBK_EINVAL, "BF16 copy not kept (storage_mask)");
        mode = Mode::CorrBF16;
    } else {
        return fail(REBK_EINVAL, "refinement storage must be REBK_FP32 or REBK_BF16");
    }
    if (ro.max_outer < 0 || ro.inner_iters < 0 || ro.inner_reduction < 0)
        return fail(REBK_EINVAL, "negative refinement option");
    const int max_outer = ro.max_outer > 0 ? ro.max_outer : 30;
    const double red = ro.inner_reduction > 0 ? ro.inner_reduction : (mode == Mode::CorrF32 ? 1e-4 : 1e-2);
    rebk_solve_ext e;
    memset(&e, 0, sizeof(e));
    if (ext) e = *ext;
    if (e.k0 < 0) return fail(REBK_EINVAL, "k0 < 0");
    const cudaStream_t st = h->stream;
    double *z = e.z_out ? e.z_out : h->zbuf;
    const int G = (h->fro2 == 0.0 || max_iter == 0) ? 1 : pick_ctas(h, mode);
    reset_counters(h);

    CK(cudaEventRecord(h->ev0, st));
    if (e.z0) {
        if (e.z0 != z) CK(cudaMemcpyAsync(z, e.z0, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    } else {
        CK(cudaMemcpyAsync(z, b, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    }
    if (e.x0) {
        if (e.x0 != x) CK(cudaMemcpyAsync(x, e.x0, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, st));
    } else {
        CK(cudaMemsetAsync(x, 0, sizeof(double) * h->n, st));
    }
    if (h->fro2 == 0.0 || max_iter == 0) {
        CK(cudaStreamSynchronize(st));
        double rel = -1;
        if (e.x_ref) {
            rebk_status s = rel_error(h, x, e.x_ref, &rel);
            if (s != REBK_OK) return s;
        }
        fill_stats(h, stats, 0, 0, REBK_OK, rel, -1, -1, 0.0);
        return REBK_OK;
    }
    rebk_status s = check_smem(h, mode, G);
    if (s != REBK_OK) return s;

    const bool use_ref = e.x_ref != nullptr;
    double refn = 0.0;
    if (use_ref) {
        LK(h, sum_sq(e.x_ref, h->n, h->ws->small, st));
        double v[2];
        s = fetch_small(h, v, 2);
        if (s != REBK_OK) return s;
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
    int64_t check = h->check_every > 0 ? h->check_every : 10;

    GridArgs a = base_args(h, mode, G);
    a.seed = seed;
    a.stream = e.stream_id;
    a.z = h->dz;
    a.x = h->dx;
    a.beta = h->f;
    a.gamma = h->g;
    a.sdual = h->sd;
    a.vdual = h->vd;

    int64_t total = 0;
    int outer = 0;
    rebk_status result = REBK_MAX_ITER;
    double rel = -1, rf = -1, rg = -1, prev_res = -1;
    bool x_zero = e.x0 == nullptr;  // x^0 = 0: A x vanishes in the first residual
    for (outer = 0; outer < max_outer; ++outer) {
        double e0 = 0.0;
        if (use_ref) {  // the error test needs x only: before the sweep, which a converged x skips
            LK(h, err_norms(nullptr, x, e.x_ref, h->n, h->ws->small, st));
            double v[2];
            s = fetch_small(h, v, 2);
            if (s != REBK_OK) return s;
            e0 = std::sqrt(v[0]);
            rel = refn > 0 ? e0 / refn : e0;
            if (rel <= tol) {
                result = REBK_OK;
                break;
            }
        }
        // f = b - z - A x, g = A^T z (FP64)
        if (x_zero) CK(cudaMemsetAsync(h->ym, 0, sizeof(double) * h->m, st));
        s = timed_sweep(h, x_zero ? nullptr : x, false, z, false, h->ym, h->g);
        if (s != REBK_OK) return s;
        x_zero = false;
        LK(h, form_f(b, z, h->ym, h->f, h->m, st));
        if (!use_ref) {
            LK(h, sum_sq(h->f, h->m, h->ws->small, st));
            LK(h, sum_sq(h->g, h->n, h->ws->small + 2, st));
            LK(h, sum_sq(b, h->m, h->ws->small + 4, st));
            double v[6];
            s = fetch_small(h, v, 6);
            if (s != REBK_OK) return s;
            const double nb = std::sqrt(v[5]);
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
        LK(h, fill_zero_f32(h->dz, h->m, st));
        LK(h, fill_zero_f32(h->vd, h->m, st));
        LK(h, fill_zero_f32(h->dx, h->n, st));
        LK(h, fill_zero_f32(h->sd, h->n, st));
        const int64_t iters = std::min(inner_max, max_iter - total);
        int64_t ran = 0;
        int64_t grow = mode == Mode::CorrBF16 ? 2048 : 4096;  // chunks of g, g, 2g, 4g, ... iterations
        int chunks = 0;
        // A pass ends when its error test passes, or (with a reference) when its
        // error stops falling: after a chunk without the test, the error of
        // x + dx is measured; a chunk that did not lower it, or whose rate
        // (log-reduction per iteration) fell below a tenth of the previous
        // chunk's, means the inner iteration reached the floor that the rounded
        // matrix sets, and a new FP64 residual is the way on.
        double e_prev = e0, rate_prev = -1.0;
        while (ran < iters) {
            int64_t chunk = std::min(iters - ran, e.idx_out ? kMaxItersPerLaunch : kIdxChunkMax);
            if (use_ref) {
                chunk = std::min(chunk, grow);
                if (++chunks >= 2) grow = std::min<int64_t>(grow * 2, kIdxChunkMax);
            }
            s = sample_into(h, a, e.k0 + total + ran, chunk,
                            e.idx_out ? e.idx_out + 2 * (total + ran) : nullptr);
            if (s != REBK_OK) return s;
            a.check_offset = ran;
            if (use_ref) {
                const double thr = std::max(tol * refn, red * e0);
                a.x_ref = e.x_ref;
                a.x_base = x;
                a.tol2_abs = thr * thr;
                a.check_every = check;
            }
            int dev_status = 0;
            int64_t done = 0;
            s = run_grid(h, mode, a, G, &dev_status, &done);
            if (s != REBK_OK) return s;
            ran += done;
            if (dev_status == 6) {
                fill_stats(h, stats, total + ran, outer + 1, REBK_BARRIER_TIMEOUT, -1, -1, -1, 0);
                return fail(REBK_BARRIER_TIMEOUT, "device-wide barrier timed out");
            }
            if (dev_status == 5) {
                fill_stats(h, stats, total + ran, outer + 1, REBK_DIVERGED, -1, -1, -1, 0);
                return fail(REBK_DIVERGED, "inner iteration diverged (Inf/NaN)");
            }
            if (done < chunk) break;  // error test met
            if (use_ref && ran < iters) {
                LK(h, err_norms_f32(x, h->dx, e.x_ref, h->n, h->ws->small, st));
                double v[2];
                s = fetch_small(h, v, 2);
                if (s != REBK_OK) return s;
                const double e_now = std::sqrt(v[0]);
                if (!(e_now < e_prev)) break;
                const double rate = std::log(e_prev / e_now) / (double)done;
                if (rate_prev > 0.0 && rate < 0.1 * rate_prev) break;
                rate_prev = rate;
                e_prev = e_now;
            }
        }
        total += ran;
        // z <- z - A s, x <- x + A^T v (FP64 A); the FP32 duals are widened first into
        // g and f, which the next pass recomputes
        LK(h, widen_f32(h->sd, h->g, h->n, st));
        LK(h, widen_f32(h->vd, h->f, h->m, st));
        s = timed_sweep(h, h->g, false, h->f, false, h->ym, h->yn);
        if (s != REBK_OK) return s;
        LK(h, apply_update(x, h->yn, h->n, z, h->ym, h->m, st));
    }
    if (result != REBK_OK) {
        // final test after the last pass
        if (use_ref) {
            s = rel_error(h, x, e.x_ref, &rel);
            if (s != REBK_OK) return s;
            if (rel <= tol) result = REBK_OK;
        } else {
            s = residuals(h, b, x, z, &rf, &rg);
            if (s != REBK_OK) return s;
            if (std::max(rf, rg) <= tol) result = REBK_OK;
        }
    }
    CK(cudaEventRecord(h->ev1, st));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    fill_stats(h, stats, total, outer, result, rel, rf, rg, ms);
    return result;
}

rebk_status rebk_solve_free(rebk_handle h, int64_t tau_row, int64_t tau_col, double alpha, const double *b,
                            double *x, double tol, int64_t max_iter, uint64_t seed, const rebk_solve_ext *ext,
                            rebk_stats *stats) {
    g_last_error.clear();
    if (!h) return fail(REBK_EINVAL, "handle is NULL");
    if (!b || !x) return fail(REBK_EINVAL, "b and x must be device pointers");
    if (tau_row < 1 || tau_col < 1) return fail(REBK_EINVAL, "tau_row and tau_col must be >= 1");
    if (tau_row > 512 || tau_col > 512) return fail(REBK_EUNSUPPORTED, "tau > 512");
    if (max_iter < 0) return fail(REBK_EINVAL, "max_iter < 0");
    if (!std::isfinite(tol) || !std::isfinite(alpha)) return fail(REBK_EINVAL, "tol or alpha not finite");
    rebk_solve_ext e;
    memset(&e, 0, sizeof(e));
    if (ext) e = *ext;
    if (e.k0 < 0) return fail(REBK_EINVAL, "k0 < 0");
    const cudaStream_t st = h->stream;
    const int tr = (int)tau_row, tc = (int)tau_col, W = tr + tc;
    const double a_step = alpha > 0.0 ? alpha : h->alpha;
    reset_counters(h);
    // per-row / per-column squared norms and prefix sums (tables with blocks of one)
    if (!h->fr_rn) {
        double *scratch = nullptr;
        int *fb = nullptr;
        CK(cudaMalloc(&h->fr_rn, sizeof(double) * h->m));
        CK(cudaMalloc(&h->fr_cdf_r, sizeof(double) * h->m));
        CK(cudaMalloc(&h->fr_cn, sizeof(double) * h->n));
        CK(cudaMalloc(&h->fr_cdf_c, sizeof(double) * h->n));
        CK(cudaMalloc(&scratch, sizeof(double) * (size_t)(h->m + h->n + 64 * h->n)));
        CK(cudaMalloc(&fb, sizeof(int) * 2));
        cudaError_t ce = block_tables(h->A64, h->lda, h->m, h->n, 1, 1, (int)h->m, (int)h->n, h->fr_rn, h->fr_cn,
                                      h->fr_cdf_r, h->fr_cdf_c, fb, scratch, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(h->fr_fb, fb, sizeof(int) * 2, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        cudaFree(scratch);
        cudaFree(fb);
        CK(ce);
    }
    // the drawn columns are read as rows of a transposed FP64 copy (contiguous), built once
    if (!h->fr_AT) {
        const int64_t ldt = round_up(h->m, 32);
        CK(cudaMalloc(&h->fr_AT, sizeof(double) * (size_t)h->n * ldt));
        h->fr_ldt = ldt;
        CK(cudaMemsetAsync(h->fr_AT, 0, sizeof(double) * (size_t)h->n * ldt, st));
        LK(h, transpose_f64(h->A64, h->lda, h->m, h->n, h->fr_AT, ldt, st));
    }
    const int acc_w = (int)round_up(W + 1, 32);
    if (acc_w > h->fr_acc_w) {
        if (h->fr_acc) cudaFree(h->fr_acc);
        h->fr_acc = nullptr;
        h->fr_acc_w = 0;
        CK(cudaMalloc(&h->fr_acc, sizeof(double) * 3 * (size_t)acc_w));
        h->fr_acc_w = acc_w;
    }
    double *z = e.z_out ? e.z_out : h->zbuf;
    CK(cudaEventRecord(h->ev0, st));
    if (e.z0) {
        if (e.z0 != z) CK(cudaMemcpyAsync(z, e.z0, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    } else {
        CK(cudaMemcpyAsync(z, b, sizeof(double) * h->m, cudaMemcpyDeviceToDevice, st));
    }
    if (e.x0) {
        if (e.x0 != x) CK(cudaMemcpyAsync(x, e.x0, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, st));
    } else {
        CK(cudaMemsetAsync(x, 0, sizeof(double) * h->n, st));
    }
    double rel = -1.0;
    if (h->fro2 == 0.0 || max_iter == 0) {
        CK(cudaStreamSynchronize(st));
        if (e.x_ref) {
            rebk_status s = rel_error(h, x, e.x_ref, &rel);
            if (s != REBK_OK) return s;
        }
        fill_stats(h, stats, 0, 0, REBK_OK, rel, -1, -1, 0.0);
        return REBK_OK;
    }
    int G = free_max_ctas(tr, tc);
    if (G < 1) return fail(REBK_EUNSUPPORTED, "the partition-free kernel does not fit on this GPU");
    G = (int)std::min<int64_t>(G, std::max<int64_t>(1, std::max(h->m, h->n) / 32));
    if (h->num_ctas_opt > 0) G = std::min(G, h->num_ctas_opt);
    const bool use_ref = e.x_ref != nullptr && tol > 0;
    int64_t check = h->check_every > 0 ? h->check_every : 10;
    double ref2 = 0.0;
    if (use_ref) {
        LK(h, sum_sq(e.x_ref, h->n, h->ws->small, st));
        double v[2];
        rebk_status s = fetch_small(h, v, 2);
        if (s != REBK_OK) return s;
        ref2 = v[1];
    }
    FreeArgs a;
    memset(&a, 0, sizeof(a));
    a.A = h->A64;
    a.AT = h->fr_AT;
    a.ldt = h->fr_ldt;
    a.lda = h->lda;
    a.m = h->m;
    a.n = h->n;
    a.tau_r = tr;
    a.tau_c = tc;
    a.rn = h->fr_rn;
    a.cn = h->fr_cn;
    a.alpha = a_step;
    a.z = z;
    a.x = x;
    a.b = b;
    a.acc = h->fr_acc;
    a.acc_w = acc_w;
    a.bar = &h->ws->bar;
    a.status = &h->ws->status;
    a.iters_done = &h->ws->iters_done;
    a.x_ref = use_ref ? e.x_ref : nullptr;
    a.tol2_abs = tol * tol * ref2;
    a.check_every = check;
    a.timeout_ns = kBarrierTimeoutNs;
    // draws of one launch: at most 2^22 entries in the handle's buffer
    const int64_t chunk_cap = std::max<int64_t>(1, ((int64_t)1 << 22) / W);
    int64_t total = 0, grow = 4096;
    rebk_status result = REBK_MAX_ITER;
    while (total < max_iter) {
        int64_t chunk = std::min(max_iter - total, e.idx_out ? kMaxItersPerLaunch : chunk_cap);
        if (use_ref) {
            chunk = std::min(chunk, grow);
            grow = std::min<int64_t>(grow * 2, chunk_cap);
        }
        int32_t *dst = e.idx_out ? e.idx_out + (size_t)W * total : nullptr;
        if (!dst) {
            if (chunk * W > h->fr_idx_cap) {
                if (h->fr_idx) cudaFree(h->fr_idx);
                h->fr_idx = nullptr;
                h->fr_idx_cap = 0;
                CK(cudaMalloc(&h->fr_idx, sizeof(int32_t) * (size_t)chunk * W));
                h->fr_idx_cap = chunk * W;
            }
            dst = h->fr_idx;
        }
        LK(h, free_sample(seed, e.stream_id, e.k0 + total, chunk, h->fr_cdf_r, h->m, h->fr_cdf_c, h->n, tr, tc,
                          h->fr_fb[0], h->fr_fb[1], dst, st));
        a.idx = dst;
        a.iters = chunk;
        a.check_offset = total;
        CK(cudaMemsetAsync(h->fr_acc, 0, sizeof(double) * 3 * (size_t)acc_w, st));
        CK(cudaMemsetAsync(h->ws, 0, sizeof(Workspace), st));
        CK(cudaEventRecord(h->kev0, st));
        CK(launch_free(a, G, st));
        CK(cudaEventRecord(h->kev1, st));
        ++h->launches;
        ++h->grid_launches;
        Workspace w;
        CK(cudaMemcpyAsync(&w, h->ws, sizeof(Workspace), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        float kms = 0.f;
        CK(cudaEventElapsedTime(&kms, h->kev0, h->kev1));
        h->kernel_ms += kms;
        total += w.iters_done;
        if (w.status == 6) {
            fill_stats(h, stats, total, 0, REBK_BARRIER_TIMEOUT, -1, -1, -1, 0);
            return fail(REBK_BARRIER_TIMEOUT, "device-wide barrier timed out");
        }
        if (w.status == 5) {
            result = REBK_DIVERGED;
            break;
        }
        if (use_ref) {
            if (w.iters_done < chunk) {  // stopped by the error test
                result = REBK_OK;
                break;
            }
            if (total % check == 0) {  // the last iterate of a launch is tested here
                rebk_status s = rel_error(h, x, e.x_ref, &rel);
                if (s != REBK_OK) return s;
                if (rel <= tol) {
                    result = REBK_OK;
                    break;
                }
            }
        }
    }
    CK(cudaEventRecord(h->ev1, st));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    if (e.x_ref) {
        rebk_status s = rel_error(h, x, e.x_ref, &rel);
        if (s != REBK_OK) return s;
        if (result == REBK_MAX_ITER && use_ref && rel <= tol) result = REBK_OK;
    }
    if (!use_ref && result == REBK_MAX_ITER) result = REBK_OK;
    fill_stats(h, stats, total, 0, result, rel, -1, -1, ms);
    if (result == REBK_DIVERGED) return fail(REBK_DIVERGED, "iteration diverged (Inf/NaN)");
    return result;
}


rebk_status rebk_multi_group(rebk_handle h, int32_t storage, int32_t *group) {
    g_last_error.clear();
    if (!h || !group) return fail(REBK_EINVAL, "handle or group is NULL");
    Mode mode;
    if (storage == REBK_FP32 && h->A32) mode = Mode::CorrF32;
    else if (storage == REBK_BF16 && h->A16) mode = Mode::CorrBF16;
    else return fail(REBK_EINVAL, "storage must be REBK_FP32 or REBK_BF16 and kept by the handle");
    MultiArgs M;
    int G = 0, nr = 0;
    rebk_status s = multi_setup(h, mode, 0, &M, &G, &nr);
    if (s != REBK_OK) return s;
    *group = nr;
    return REBK_OK;
}

rebk_status rebk_solve_multi(rebk_handle h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                             double tol, int64_t max_iter, uint64_t seed, const rebk_multi_opts *opt,
                             const double *X_ref, int64_t ldxr, double *rel_out, rebk_stats *stats) {
    g_last_error.clear();
    if (!h) return fail(REBK_EINVAL, "handle is NULL");
    if (nrhs < 0) return fail(REBK_EINVAL, "nrhs < 0");
    if (nrhs > 0 && (!B || !X)) return fail(REBK_EINVAL, "B and X must be device pointers");
    if (nrhs > 0 && (ldb < h->m || ldx < h->n || (X_ref && ldxr < h->n)))
        return fail(REBK_EINVAL, "a leading dimension is below the vector length");
    if (max_iter < 0) return fail(REBK_EINVAL, "max_iter < 0");
    if (!std::isfinite(tol)) return fail(REBK_EINVAL, "tol is not finite");
    rebk_multi_opts o;
    memset(&o, 0, sizeof(o));
    o.storage = REBK_FP32;
    if (opt) o = *opt;
    Mode mode;
    if (o.storage == REBK_FP32) {
        if (!h->A32) return fail(REBK_EINVAL, "FP32 copy not kept (storage_mask)");
        mode = Mode::CorrF32;
    } else if (o.storage == REBK_BF16) {
        if (!h->A16) return fail(REBK_EINVAL, "BF16 copy not kept (storage_mask)");
        mode = Mode::CorrBF16;
    } else {
        return fail(REBK_EINVAL, "storage must be REBK_FP32 or REBK_BF16");
    }
    const bool bf16 = mode == Mode::CorrBF16;
    if (o.group != 0 && o.group != 4 && o.group != 8) return fail(REBK_EINVAL, "group must be 0, 4 or 8");
    if (o.max_outer < 0 || o.inner_iters < 0 || o.inner_reduction < 0 || o.reserved != 0)
        return fail(REBK_EINVAL, "negative or reserved option set");
    const int max_outer = o.max_outer > 0 ? o.max_outer : 30;
    const double red = o.inner_reduction > 0 ? o.inner_reduction : (bf16 ? 1e-2 : 1e-4);
    const cudaStream_t st = h->stream;
    const int64_t m = h->m, n = h->n;
    const bool use_ref = X_ref != nullptr;
    reset_counters(h);
    if (nrhs == 0) {
        fill_stats(h, stats, 0, 0, REBK_OK, -1, -1, -1, 0.0);
        return REBK_OK;
    }

    MultiArgs M;
    int G = 0, nr = 0;
    rebk_status ms_ = multi_setup(h, mode, o.group, &M, &G, &nr);
    if (ms_ != REBK_OK) return ms_;
    GridArgs &a = M.geo;
    const int aw = (int)round_up((int64_t)(a.tau_r + a.tau_c) * nr, 4);

    // device buffers (one allocation kept by the handle)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o0 = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o0;
    };
    const size_t mv = (size_t)m * nr, nv = (size_t)n * nr;
    const size_t oB = take(8 * mv), oZ = take(8 * mv), oX = take(8 * nv), oXr = take(8 * nv), oYm = take(8 * mv),
                 oYn = take(8 * nv), oSm = take(8 * 64), oF = take(4 * mv), oG = take(4 * nv), odZ = take(4 * mv),
                 oV = take(4 * mv), odX = take(4 * nv), oS = take(4 * nv), oSd = take(8 * nv), oVd = take(8 * mv),
                 oAcc = take(sizeof(float) * 3 * kMultiReplicas * (size_t)aw);
    if (off > h->mr_bytes) {
        if (h->mr_buf) cudaFree(h->mr_buf);
        h->mr_buf = nullptr;
        h->mr_bytes = 0;
        CK(cudaMalloc(&h->mr_buf, off));
        h->mr_bytes = off;
    }
    char *base = static_cast<char *>(h->mr_buf);
    double *Bq = (double *)(base + oB), *Zq = (double *)(base + oZ), *Xq = (double *)(base + oX);
    double *Xr = (double *)(base + oXr), *Ym = (double *)(base + oYm), *Yn = (double *)(base + oYn);
    double *small = (double *)(base + oSm);
    float *F = (float *)(base + oF), *Gf = (float *)(base + oG), *dZ = (float *)(base + odZ);
    float *V = (float *)(base + oV), *dX = (float *)(base + odX), *S = (float *)(base + oS);
    float *acc = (float *)(base + oAcc);
    double *Sd = (double *)(base + oSd), *Vd = (double *)(base + oVd);
    M.dZ = dZ;
    M.dX = dX;
    M.S = S;
    M.V = V;
    M.F = F;
    M.G = Gf;
    a.acc = acc;
    a.acc_w = aw;
    auto fetch = [&](double *host, int count) -> rebk_status {
        CK(cudaMemcpyAsync(host, small, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return REBK_OK;
    };
    // FP64 products of the refinement loop, timed like the one-right-hand-side sweeps
    auto products = [&](const void *P, bool p_f32, const void *Q, bool q_f32) -> rebk_status {
        if (h->sweep_used + 2 > h->sweep_ev.size()) {
            for (int i = 0; i < 2; ++i) {
                cudaEvent_t ev;
                CK(cudaEventCreate(&ev));
                h->sweep_ev.push_back(ev);
            }
        }
        cudaEvent_t e0 = h->sweep_ev[h->sweep_used], e1 = h->sweep_ev[h->sweep_used + 1];
        h->sweep_used += 2;
        CK(cudaEventRecord(e0, st));
        if (P) LK(h, multi_ap(h->A64, h->lda, m, n, nr, P, p_f32, Ym, st));
        else CK(cudaMemsetAsync(Ym, 0, 8 * mv, st));
        LK(h, multi_atq(h->A64, h->lda, m, n, nr, Q, q_f32, Yn, st));
        CK(cudaEventRecord(e1, st));
        return REBK_OK;
    };
    int64_t inner_default = o.inner_iters;
    if (inner_default <= 0) {
        if (use_ref) {
            inner_default = 1000000;
        } else {
            const double per_iter = (double)h->tau_r * n + (double)h->tau_c * m;
            inner_default = std::max<int64_t>(200, (int64_t)(40.0 * (double)m * n / per_iter));
        }
    }

    CK(cudaEventRecord(h->ev0, st));
    const int64_t ngroups = (nrhs + nr - 1) / nr;
    int64_t all_iters = 0;
    int outer_max_seen = 0;
    double worst = -1.0;
    rebk_status result = REBK_OK;
    for (int64_t gi = 0; gi < ngroups; ++gi) {
        const int64_t j0 = gi * nr;
        const int cnt = (int)std::min<int64_t>(nr, nrhs - j0);
        LK(h, multi_gather(B + j0 * ldb, ldb, cnt, m, nr, Bq, st));
        CK(cudaMemcpyAsync(Zq, Bq, 8 * mv, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(Xq, 0, 8 * nv, st));
        double v[4 * 8];
        double refn[8] = {0}, bn[8] = {0}, rel[8], res[8];
        for (int q = 0; q < 8; ++q) rel[q] = res[q] = -1.0;
        if (use_ref) {
            LK(h, multi_gather(X_ref + j0 * ldxr, ldxr, cnt, n, nr, Xr, st));
            LK(h, multi_norms(nullptr, nullptr, Xr, n, nr, small, st));
        } else {
            LK(h, multi_norms(nullptr, nullptr, Bq, m, nr, small, st));
        }
        rebk_status s = fetch(v, 2 * nr);
        if (s != REBK_OK) return s;
        for (int q = 0; q < nr; ++q) (use_ref ? refn : bn)[q] = std::sqrt(v[nr + q]);
        // residual test of every member (after a sweep that left F and G current)
        auto residual_test = [&](double *worst_res) -> rebk_status {
            LK(h, multi_norms(nullptr, F, nullptr, m, nr, small, st));
            LK(h, multi_norms(nullptr, Gf, nullptr, n, nr, small + 2 * nr, st));
            rebk_status s2 = fetch(v, 4 * nr);
            if (s2 != REBK_OK) return s2;
            *worst_res = 0.0;
            for (int q = 0; q < cnt; ++q) {
                const double rf = bn[q] > 0 ? std::sqrt(v[q]) / bn[q] : 0.0;
                const double rg = bn[q] > 0 ? std::sqrt(v[2 * nr + q]) / (std::sqrt(h->fro2) * bn[q]) : 0.0;
                res[q] = std::max(rf, rg);
                *worst_res = std::max(*worst_res, res[q]);
            }
            return REBK_OK;
        };
        auto error_test = [&](const float *corr, double *e) -> rebk_status {
            LK(h, multi_norms(Xq, corr, Xr, n, nr, small, st));
            rebk_status s2 = fetch(v, nr);
            if (s2 != REBK_OK) return s2;
            for (int q = 0; q < nr; ++q) e[q] = std::sqrt(v[q]);
            return REBK_OK;
        };
        bool converged = false, x_zero = true;
        int64_t total = 0, inner_max = inner_default;
        double prev_res = -1.0;
        int outer = 0;
        if (h->fro2 == 0.0) converged = true;  // x = 0 is A^+ b
        for (; !converged && outer < max_outer; ++outer) {
            double e0[8] = {0};
            if (use_ref) {
                s = error_test(nullptr, e0);
                if (s != REBK_OK) return s;
                bool all = true;
                for (int q = 0; q < cnt; ++q) {
                    rel[q] = refn[q] > 0 ? e0[q] / refn[q] : e0[q];
                    all = all && rel[q] <= tol;
                }
                if (all) {
                    converged = true;
                    break;
                }
            }
            // F = b - z - A x, G = A^T z (FP64)
            s = products(x_zero ? nullptr : Xq, false, Zq, false);
            if (s != REBK_OK) return s;
            x_zero = false;
            LK(h, multi_form(Bq, Zq, Ym, F, m, Yn, Gf, n, nr, st));
            if (!use_ref) {
                double wr = 0.0;
                s = residual_test(&wr);
                if (s != REBK_OK) return s;
                if (wr <= tol) {
                    converged = true;
                    break;
                }
                if (prev_res > 0 && wr > 0.1 * prev_res) inner_max = std::min<int64_t>(inner_max * 2, 1 << 24);
                prev_res = wr;
            }
            if (total >= max_iter) break;
            CK(cudaMemsetAsync(dZ, 0, 4 * mv, st));
            CK(cudaMemsetAsync(V, 0, 4 * mv, st));
            CK(cudaMemsetAsync(dX, 0, 4 * nv, st));
            CK(cudaMemsetAsync(S, 0, 4 * nv, st));
            const int64_t iters = std::min(inner_max, max_iter - total);
            int64_t ran = 0, chunk_next = use_ref ? 512 : iters;
            // A pass ends (with a reference) once every member's error x + dx is below
            // its threshold or has stopped falling, as in rebk_solve_refined; the next
            // chunk is sized from the slowest member's observed rate.
            double e_prev[8], rate_prev[8];
            bool fin[8];
            for (int q = 0; q < 8; ++q) {
                e_prev[q] = e0[q];
                rate_prev[q] = -1.0;
                fin[q] = q >= cnt;
            }
            while (ran < iters) {
                const int64_t chunk = std::min(std::min(iters - ran, chunk_next), kMaxItersPerLaunch);
                int32_t *dst = (gi == 0 && o.idx_out) ? o.idx_out + 2 * (total + ran) : nullptr;
                if (!dst) {
                    if (chunk > h->idx_cap) {
                        if (h->idxbuf) cudaFree(h->idxbuf);
                        h->idxbuf = nullptr;
                        h->idx_cap = 0;
                        const int64_t cap = std::max<int64_t>(chunk, 65536);
                        CK(cudaMalloc(&h->idxbuf, sizeof(int32_t) * 2 * cap));
                        h->idx_cap = cap;
                    }
                    dst = h->idxbuf;
                }
                LK(h, sample_blocks(seed, o.stream_id + (uint64_t)gi, total + ran, chunk, h->cdf_r, h->s, h->cdf_c,
                                    h->t, h->fb[0], h->fb[1], dst, st));
                a.idx = dst;
                a.k0 = total + ran;
                a.iters = chunk;
                CK(cudaMemsetAsync(acc, 0, sizeof(float) * 3 * kMultiReplicas * (size_t)aw, st));
                CK(cudaMemsetAsync(h->ws, 0, sizeof(Workspace), st));
                CK(cudaEventRecord(h->kev0, st));
                CK(launch_multi(M, bf16, nr, G, st));
                CK(cudaEventRecord(h->kev1, st));
                ++h->launches;
                ++h->grid_launches;
                Workspace w;
                CK(cudaMemcpyAsync(&w, h->ws, sizeof(Workspace), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                float kms = 0.f;
                CK(cudaEventElapsedTime(&kms, h->kev0, h->kev1));
                h->kernel_ms += kms;
                ran += w.iters_done;
                if (w.status == 6) {
                    fill_stats(h, stats, all_iters + total + ran, outer + 1, REBK_BARRIER_TIMEOUT, -1, -1, -1, 0);
                    return fail(REBK_BARRIER_TIMEOUT, "device-wide barrier or tile copy timed out");
                }
                if (w.status == 5) {
                    fill_stats(h, stats, all_iters + total + ran, outer + 1, REBK_DIVERGED, -1, -1, -1, 0);
                    return fail(REBK_DIVERGED, "inner iteration diverged (Inf/NaN)");
                }
                if (w.status != 0 || w.iters_done != chunk)
                    return fail(REBK_ECUDA, "multi-right-hand-side kernel ran fewer iterations than launched");
                if (!use_ref || ran >= iters) continue;
                double e_now[8];
                s = error_test(dX, e_now);
                if (s != REBK_OK) return s;
                bool all = true;
                double need = 0.0;
                for (int q = 0; q < cnt; ++q) {
                    if (fin[q]) continue;
                    const double thr = std::max(tol * refn[q], red * e0[q]);
                    const double rate = e_now[q] > 0 ? std::log(e_prev[q] / e_now[q]) / (double)chunk : 1.0;
                    if (e_now[q] <= thr || !(e_now[q] < e_prev[q]) || (rate_prev[q] > 0.0 && rate < 0.1 * rate_prev[q])) {
                        fin[q] = true;
                        continue;
                    }
                    all = false;
                    rate_prev[q] = rate;
                    e_prev[q] = e_now[q];
                    need = std::max(need, std::log(e_now[q] / thr) / rate);
                }
                if (all) break;
                chunk_next = std::min<int64_t>(std::max<int64_t>((int64_t)(need * 1.06) + 32, 128), (int64_t)1 << 20);
            }
            total += ran;
            // z <- z - A s, x <- x + A^T v (FP64 A)
            LK(h, widen_f32(S, Sd, (int64_t)nv, st));
            LK(h, widen_f32(V, Vd, (int64_t)mv, st));
            s = products(Sd, false, Vd, false);
            if (s != REBK_OK) return s;
            LK(h, multi_apply(Xq, Yn, n, Zq, Ym, m, nr, st));
        }
        if (!converged) {  // the test after the last pass
            if (use_ref) {
                double e[8];
                s = error_test(nullptr, e);
                if (s != REBK_OK) return s;
                converged = true;
                for (int q = 0; q < cnt; ++q) {
                    rel[q] = refn[q] > 0 ? e[q] / refn[q] : e[q];
                    converged = converged && rel[q] <= tol;
                }
            } else {
                s = products(Xq, false, Zq, false);
                if (s != REBK_OK) return s;
                LK(h, multi_form(Bq, Zq, Ym, F, m, Yn, Gf, n, nr, st));
                double wr = 0.0;
                s = residual_test(&wr);
                if (s != REBK_OK) return s;
                converged = wr <= tol;
            }
        } else if (use_ref && h->fro2 == 0.0) {
            double e[8];
            s = error_test(nullptr, e);
            if (s != REBK_OK) return s;
            for (int q = 0; q < cnt; ++q) rel[q] = refn[q] > 0 ? e[q] / refn[q] : e[q];
        }
        LK(h, multi_scatter(Xq, cnt, n, nr, X + j0 * ldx, ldx, st));
        for (int q = 0; q < cnt; ++q) {
            const double r = use_ref ? rel[q] : res[q];
            if (rel_out) rel_out[j0 + q] = r;
            worst = std::max(worst, r);
        }
        all_iters += total;
        outer_max_seen = std::max(outer_max_seen, outer);
        if (!converged) result = REBK_MAX_ITER;
    }
    CK(cudaEventRecord(h->ev1, st));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    fill_stats(h, stats, all_iters, outer_max_seen, result, use_ref ? worst : -1.0, use_ref ? -1.0 : worst, -1.0, ms);
    return result;
}

}  // extern "C"
