"""Python face of the REBK solver: a handle around the C ABI with torch tensors
for device memory and streams.  Every computation runs in librebk.so."""
from __future__ import annotations

import ctypes
import math
from typing import Optional, Sequence

import numpy as np

from . import rebk as _r


def _torch():
    import torch
    return torch


def _dptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _require_cuda_f64(t, n: int, name: str):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
            and t.numel() == n):
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {n} elements")


class Solver:
    """REBK solver for one matrix A (Algorithm 1 of arXiv:2001.04179).

    A: torch CUDA float64 tensor (m x n, row-major) or a numpy float64 array.
    tau_row / tau_col: block sizes of the contiguous partitions (Section 3).
    row_off / col_off: any partitions instead (Section 2's I_1..I_s and
    J_1..J_t): int64 offsets 0 = off[0] < ... < off[-1] = m (n), blocks of at
    most 512; the tau of a side given by offsets is ignored.
    alpha: step size; <= 0 picks 1.75 / beta_max.
    storage: reduced-precision copies to keep for solve_refined ("fp32", "bf16").
    """

    def __init__(self, A, tau_row: int = 0, tau_col: int = 0, alpha: float = 0.0,
                 storage: Sequence[str] = ("fp32",), num_ctas: int = 0, check_every: int = 0,
                 stream=None, row_off=None, col_off=None):
        torch = _torch()
        lib = _r.load()
        mask = 0
        for s in storage:
            mask |= 1 << _r.STORAGE[s]
        self._stream = stream
        opt = _r.RebkOptions(tau_row, tau_col, mask, num_ctas, check_every,
                             None if stream is None else ctypes.c_void_p(stream.cuda_stream))
        part = None
        if row_off is not None or col_off is not None:
            self._ro = None if row_off is None else np.ascontiguousarray(row_off, dtype=np.int64)
            self._co = None if col_off is None else np.ascontiguousarray(col_off, dtype=np.int64)
            part = _r.RebkPartition(None if self._ro is None else self._ro.ctypes.data,
                                    0 if self._ro is None else self._ro.size - 1,
                                    None if self._co is None else self._co.ctypes.data,
                                    0 if self._co is None else self._co.size - 1)
        pp = None if part is None else ctypes.byref(part)
        h = ctypes.c_void_p()
        if isinstance(A, torch.Tensor):
            if not (A.is_cuda and A.dtype == torch.float64 and A.dim() == 2 and A.stride(1) == 1):
                raise ValueError("A must be a CUDA float64 matrix with unit column stride")
            m, n = A.shape
            st = lib.rebk_create(ctypes.byref(h), ctypes.c_void_p(A.data_ptr()), m, n, A.stride(0), 1, pp,
                                 float(alpha), ctypes.byref(opt))
        else:
            An = np.ascontiguousarray(A, dtype=np.float64)
            m, n = An.shape
            st = lib.rebk_create(ctypes.byref(h), An.ctypes.data_as(ctypes.c_void_p), m, n, n, 0, pp,
                                 float(alpha), ctypes.byref(opt))
        _r.check(st)
        self._h = h
        self.m, self.n = int(m), int(n)
        ro, co = self.partition()
        self.tau_row, self.tau_col = int(np.max(np.diff(ro))), int(np.max(np.diff(co)))

    def partition(self):
        """(row_off, col_off): the partitions in use, as int64 offset arrays."""
        s, t = self.blocks()
        ro, co = np.zeros(s + 1, dtype=np.int64), np.zeros(t + 1, dtype=np.int64)
        _r.check(_r.load().rebk_get_partition(self._h, ro.ctypes.data_as(ctypes.c_void_p),
                                              co.ctypes.data_as(ctypes.c_void_p), None, None))
        return ro, co

    @classmethod
    def rek(cls, A, **kw) -> "Solver":
        """The randomized extended Kaczmarz special case of Algorithm 1 (single rows
        and columns, alpha = 1; the remark after Algorithm 1)."""
        kw.setdefault("storage", ())
        return cls(A, 1, 1, alpha=1.0, **kw)

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _r.load().rebk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    @property
    def alpha(self) -> float:
        a = ctypes.c_double()
        _r.check(_r.load().rebk_get_alpha(self._h, ctypes.byref(a)))
        return a.value

    @alpha.setter
    def alpha(self, value: float):
        """Replace the step size (block coefficients are rebuilt on the device)."""
        _r.check(_r.load().rebk_set_alpha(self._h, float(value)))

    def spectrum(self, steps: int = 200, seed: int = 0) -> dict:
        """sigma_1^2, sigma_r^2 (device Lanczos) and the step-size quantities of
        Remark alpha, Theorem ner and Theorem main (rebk_spectral_estimates)."""
        out = _r.RebkSpectrum()
        _r.check(_r.load().rebk_spectral_estimates(self._h, int(steps), int(seed), ctypes.byref(out)))
        return out.as_dict()

    def use_mean_optimal_alpha(self, steps: int = 200, seed: int = 0) -> float:
        """Set alpha to Remark alpha's 2 ||A||_F^2 / (sigma_1^2 + sigma_r^2), the
        minimiser of Theorem ner's rate for the mean error.  It usually exceeds
        2 / beta_max, where Theorem main gives no mean-square convergence."""
        a = self.spectrum(steps, seed)["alpha_mean_opt"]
        self.alpha = a
        return a

    def blocks(self):
        s, t = ctypes.c_int64(), ctypes.c_int64()
        _r.check(_r.load().rebk_get_blocks(self._h, ctypes.byref(s), ctypes.byref(t)))
        return s.value, t.value

    def tables(self):
        s, t = self.blocks()
        nr, nc, cr, cc = np.zeros(s), np.zeros(t), np.zeros(s), np.zeros(t)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _r.check(_r.load().rebk_get_tables(self._h, p(nr), p(nc), p(cr), p(cc)))
        return nr, nc, cr, cc

    def beta_max(self):
        br, bc = ctypes.c_double(), ctypes.c_double()
        _r.check(_r.load().rebk_beta_max(self._h, ctypes.byref(br), ctypes.byref(bc)))
        return br.value, bc.value

    def export_storage(self, storage: str) -> np.ndarray:
        dt = {"fp64": np.float64, "fp32": np.float32, "bf16": np.uint16}[storage]
        out = np.zeros((self.m, self.n), dtype=dt)
        _r.check(_r.load().rebk_export_storage(self._h, _r.STORAGE[storage],
                                               out.ctypes.data_as(ctypes.c_void_p)))
        return out

    # ------------------------------------------------------------------
    def _ext(self, x_ref, x0, z0, z_out, idx_out, k0, stream_id):
        for t, n, name in [(x_ref, self.n, "x_ref"), (x0, self.n, "x0"), (z0, self.m, "z0"),
                           (z_out, self.m, "z_out")]:
            if t is not None:
                _require_cuda_f64(t, n, name)
        return _r.RebkSolveExt(_dptr(x_ref), _dptr(x0), _dptr(z0), _dptr(z_out), _dptr(idx_out),
                               int(k0), int(stream_id))

    def solve(self, b, tol: float = 0.0, max_iter: int = 1000, seed: int = 0, x_ref=None, x0=None,
              z0=None, k0: int = 0, stream_id: int = 0, record: bool = False, return_z: bool = False,
              x=None, allow=(_r.REBK_OK, _r.REBK_MAX_ITER)):
        """Plain FP64 Algorithm 1.  Returns dict(x, stats[, z][, idx])."""
        torch = _torch()
        _require_cuda_f64(b, self.m, "b")
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=b.device)
        z = torch.empty(self.m, dtype=torch.float64, device=b.device) if return_z else None
        idx = torch.zeros(max(2 * max_iter, 2), dtype=torch.int32, device=b.device) if record else None
        ext = self._ext(x_ref, x0, z0, z, idx, k0, stream_id)
        stats = _r.RebkStats()
        st = _r.load().rebk_solve_ex(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                     float(tol), int(max_iter), int(seed), ctypes.byref(ext),
                                     ctypes.byref(stats))
        _r.check(st, allow)
        out = {"x": x, "stats": stats.as_dict(), "status": st}
        if return_z:
            out["z"] = z
        if record:
            out["idx"] = idx[: 2 * stats.iterations].view(-1, 2)
        return out

    def solve_free(self, b, tau_row: int, tau_col: int, alpha: float = 0.0, tol: float = 0.0,
                   max_iter: int = 1000, seed: int = 0, x_ref=None, x0=None, z0=None, k0: int = 0,
                   stream_id: int = 0, record: bool = False, return_z: bool = False, x=None,
                   allow=(_r.REBK_OK, _r.REBK_MAX_ITER)):
        """Algorithm 1 with index sets drawn without a partition (rebk_solve_free):
        tau_col columns and tau_row rows drawn independently with probabilities
        proportional to their squared norms per iteration.  alpha <= 0 uses the
        handle's.  Returns dict(x, stats[, z][, idx]); idx is (iterations,
        tau_col + tau_row): the column draws, then the row draws."""
        torch = _torch()
        _require_cuda_f64(b, self.m, "b")
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=b.device)
        z = torch.empty(self.m, dtype=torch.float64, device=b.device) if return_z else None
        W = int(tau_row) + int(tau_col)
        idx = torch.zeros(max(W * max_iter, 1), dtype=torch.int32, device=b.device) if record else None
        ext = self._ext(x_ref, x0, z0, z, idx, k0, stream_id)
        stats = _r.RebkStats()
        st = _r.load().rebk_solve_free(self._h, int(tau_row), int(tau_col), float(alpha),
                                       ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), float(tol),
                                       int(max_iter), int(seed), ctypes.byref(ext), ctypes.byref(stats))
        _r.check(st, allow)
        out = {"x": x, "stats": stats.as_dict(), "status": st}
        if return_z:
            out["z"] = z
        if record:
            out["idx"] = idx[: W * stats.iterations].view(-1, W)
        return out

    def solve_multi(self, B, tol: float = 1e-8, max_iter: int = 10**7, seed: int = 0, storage: str = "fp32",
                    group: int = 0, X_ref=None, max_outer: int = 0, inner_iters: int = 0,
                    inner_reduction: float = 0.0, stream_id: int = 0, record: bool = False, X=None,
                    allow=(_r.REBK_OK, _r.REBK_MAX_ITER)):
        """Several right-hand sides at once (rebk_solve_multi): B is a CUDA
        float64 (nrhs, m) tensor with unit column stride; each row is solved as
        solve_refined solves one, in groups of `group` (4 or 8, 0 = library
        choice) that share one block sequence.  Returns dict(X (nrhs, n), rel
        (per right-hand side: error with X_ref, else residual), stats[, idx of
        the first group])."""
        torch = _torch()
        if not (B.is_cuda and B.dtype == torch.float64 and B.dim() == 2 and B.shape[1] == self.m
                and B.stride(1) == 1):
            raise ValueError(f"B must be a CUDA float64 (nrhs, {self.m}) tensor with unit column stride")
        nrhs = B.shape[0]
        if X is None:
            X = torch.empty(nrhs, self.n, dtype=torch.float64, device=B.device)
        if X_ref is not None and not (X_ref.is_cuda and X_ref.dtype == torch.float64 and X_ref.dim() == 2
                                      and tuple(X_ref.shape) == (nrhs, self.n) and X_ref.stride(1) == 1):
            raise ValueError(f"X_ref must be a CUDA float64 ({nrhs}, {self.n}) tensor with unit column stride")
        idx = torch.zeros(max(2 * min(max_iter, 10**7), 2), dtype=torch.int32, device=B.device) if record else None
        opt = _r.RebkMultiOpts(_r.STORAGE[storage], int(group), int(max_outer), 0, int(inner_iters),
                               float(inner_reduction), _dptr(idx), int(stream_id))
        rel = (ctypes.c_double * max(nrhs, 1))()
        stats = _r.RebkStats()
        st = _r.load().rebk_solve_multi(self._h, nrhs, _dptr(B), B.stride(0) if nrhs else self.m, _dptr(X),
                                        X.stride(0) if nrhs else self.n, float(tol), int(max_iter), int(seed),
                                        ctypes.byref(opt), _dptr(X_ref),
                                        X_ref.stride(0) if X_ref is not None else 0,
                                        ctypes.cast(rel, ctypes.c_void_p), ctypes.byref(stats))
        _r.check(st, allow)
        out = {"X": X, "rel": np.array(rel[:nrhs]), "stats": stats.as_dict(), "status": st}
        if record:
            out["idx"] = idx
        return out

    def multi_group(self, storage: str = "fp32") -> int:
        """Group size solve_multi picks for `storage` (rebk_multi_group)."""
        g = ctypes.c_int32()
        _r.check(_r.load().rebk_multi_group(self._h, _r.STORAGE[storage], ctypes.byref(g)))
        return g.value

    def solve_rabk(self, b, **kw):
        """The RABK special case (the remark after Algorithm 1): z^0 = 0 keeps every
        z^k = 0, so each step is the weighted block average of eq. (rabk) on A x = b
        (consistent systems).  Arguments as solve()."""
        torch = _torch()
        _require_cuda_f64(b, self.m, "b")
        kw["z0"] = torch.zeros(self.m, dtype=torch.float64, device=b.device)
        return self.solve(b, **kw)

    def solve_refined(self, b, tol: float = 1e-8, max_iter: int = 10**7, seed: int = 0,
                      storage: str = "fp32", x_ref=None, x0=None, z0=None, k0: int = 0,
                      stream_id: int = 0, max_outer: int = 0, inner_iters: int = 0,
                      inner_reduction: float = 0.0, record: bool = False, return_z: bool = False,
                      x=None, allow=(_r.REBK_OK, _r.REBK_MAX_ITER)):
        """Mixed precision (FP32/BF16 inner sweeps, FP64 refinement).  Returns dict(x, stats, ...)."""
        torch = _torch()
        _require_cuda_f64(b, self.m, "b")
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=b.device)
        z = torch.empty(self.m, dtype=torch.float64, device=b.device) if return_z else None
        idx = torch.zeros(max(2 * min(max_iter, 10**7), 2), dtype=torch.int32, device=b.device) if record else None
        ext = self._ext(x_ref, x0, z0, z, idx, k0, stream_id)
        ro = _r.RebkRefineOpts(_r.STORAGE[storage], int(max_outer), int(inner_iters), float(inner_reduction))
        stats = _r.RebkStats()
        st = _r.load().rebk_solve_refined(self._h, ctypes.c_void_p(b.data_ptr()),
                                          ctypes.c_void_p(x.data_ptr()), float(tol), int(max_iter),
                                          int(seed), ctypes.byref(ro), ctypes.byref(ext),
                                          ctypes.byref(stats))
        _r.check(st, allow)
        out = {"x": x, "stats": stats.as_dict(), "status": st}
        if return_z:
            out["z"] = z
        if record:
            out["idx"] = idx[: 2 * stats.iterations].view(-1, 2)
        return out


def tune_tau(A, b, taus: Sequence[int], x_ref=None, alpha_factor: float = 1.75, storage: str = "fp64",
             tol: float = 1e-8, max_iter: int = 10**7, seed: int = 0, trials: int = 1, num_ctas: int = 0,
             check_every: int = 0, stream=None):
    """Block-size autotuner (rebk_tune_tau): time to tolerance for each tau.

    A: CUDA float64 tensor or numpy array (m x n); b, x_ref: CUDA float64.
    Returns (best_tau, [dict(tau, beta_max, alpha, iterations, device_ms, status)]);
    best_tau is 0 when no candidate reached tol.
    """
    torch = _torch()
    lib = _r.load()
    taus = [int(t) for t in taus]
    arr = (ctypes.c_int64 * len(taus))(*taus)
    pts = (_r.RebkTunePoint * len(taus))()
    best = ctypes.c_int64()
    opt = _r.RebkOptions(0, 0, 0, num_ctas, check_every,
                         None if stream is None else ctypes.c_void_p(stream.cuda_stream))
    if isinstance(A, torch.Tensor):
        if not (A.is_cuda and A.dtype == torch.float64 and A.dim() == 2 and A.stride(1) == 1):
            raise ValueError("A must be a CUDA float64 matrix with unit column stride")
        m, n = A.shape
        ptr, ld, on_dev = A.data_ptr(), A.stride(0), 1
        keep = A
    else:
        keep = np.ascontiguousarray(A, dtype=np.float64)
        m, n = keep.shape
        ptr, ld, on_dev = keep.ctypes.data, n, 0
    _require_cuda_f64(b, m, "b")
    if x_ref is not None:
        _require_cuda_f64(x_ref, n, "x_ref")
    st = lib.rebk_tune_tau(ctypes.c_void_p(ptr), m, n, ld, on_dev, ctypes.c_void_p(b.data_ptr()),
                           _dptr(x_ref), ctypes.cast(arr, ctypes.c_void_p), len(taus), float(alpha_factor),
                           _r.STORAGE[storage], float(tol), int(max_iter), int(seed), int(trials),
                           ctypes.byref(opt), ctypes.cast(pts, ctypes.c_void_p), ctypes.byref(best))
    del keep
    _r.check(st, (_r.REBK_OK, _r.REBK_MAX_ITER))
    return best.value, [p.as_dict() for p in pts]


class SparseSolver:
    """REBK on a sparse m x n matrix in CSR form (Algorithm 1 of
    arXiv:2001.04179 with row blocks over CSR and column blocks over a CSC copy
    the library builds).  indptr: int64 (m + 1); indices: int32, increasing
    within each row; data: float64.  alpha <= 0 picks 1.75 / beta_max."""

    def __init__(self, m: int, n: int, indptr, indices, data, tau_row: int, tau_col: int, alpha: float = 0.0,
                 num_ctas: int = 0, check_every: int = 0, power_iters: int = 0, stream=None):
        lib = _r.load()
        self._arrays = (np.ascontiguousarray(indptr, dtype=np.int64), np.ascontiguousarray(indices, dtype=np.int32),
                        np.ascontiguousarray(data, dtype=np.float64))
        if self._arrays[0].shape != (m + 1,):
            raise ValueError("indptr must have m + 1 entries")
        opt = _r.RebkSparseOptions(num_ctas, check_every, power_iters,
                                   None if stream is None else ctypes.c_void_p(stream.cuda_stream))
        h = ctypes.c_void_p()
        p = [a.ctypes.data_as(ctypes.c_void_p) for a in self._arrays]
        _r.check(lib.rebk_sparse_create(ctypes.byref(h), int(m), int(n), p[0], p[1], p[2], int(tau_row),
                                        int(tau_col), float(alpha), ctypes.byref(opt)))
        self._h = h
        self.m, self.n = int(m), int(n)

    def close(self):
        if getattr(self, "_h", None):
            _r.load().rebk_sparse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        a, bm, s, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32()
        _r.check(_r.load().rebk_sparse_info(self._h, ctypes.byref(a), ctypes.byref(bm), ctypes.byref(s),
                                            ctypes.byref(t)))
        return {"alpha": a.value, "beta_max": bm.value, "row_blocks": s.value, "col_blocks": t.value}

    @property
    def alpha(self) -> float:
        return self.info()["alpha"]

    def solve(self, b, tol: float = 0.0, max_iter: int = 1000, seed: int = 0, x_ref=None, x0=None, z0=None,
              k0: int = 0, stream_id: int = 0, record: bool = False, return_z: bool = False, x=None,
              allow=(_r.REBK_OK, _r.REBK_MAX_ITER)):
        """Plain FP64 Algorithm 1 (as Solver.solve).  Returns dict(x, stats[, z][, idx])."""
        torch = _torch()
        _require_cuda_f64(b, self.m, "b")
        for t, nn, name in [(x_ref, self.n, "x_ref"), (x0, self.n, "x0"), (z0, self.m, "z0")]:
            if t is not None:
                _require_cuda_f64(t, nn, name)
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=b.device)
        z = torch.empty(self.m, dtype=torch.float64, device=b.device) if return_z else None
        idx = torch.zeros(max(2 * max_iter, 2), dtype=torch.int32, device=b.device) if record else None
        ext = _r.RebkSolveExt(_dptr(x_ref), _dptr(x0), _dptr(z0), _dptr(z), _dptr(idx), int(k0), int(stream_id))
        stats = _r.RebkStats()
        st = _r.load().rebk_sparse_solve(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                         float(tol), int(max_iter), int(seed), ctypes.byref(ext),
                                         ctypes.byref(stats))
        _r.check(st, allow)
        out = {"x": x, "stats": stats.as_dict(), "status": st}
        if return_z:
            out["z"] = z
        if record:
            out["idx"] = idx[: 2 * stats.iterations].view(-1, 2)
        return out

    def solve_refined(self, b, tol: float = 1e-8, max_iter: int = 10**7, seed: int = 0, x_ref=None, x0=None,
                      z0=None, k0: int = 0, stream_id: int = 0, max_outer: int = 0, inner_iters: int = 0,
                      inner_reduction: float = 0.0, record: bool = False, return_z: bool = False, x=None,
                      allow=(_r.REBK_OK, _r.REBK_MAX_ITER)):
        """Mixed precision (FP32 values and inner sweeps, FP64 refinement).  Returns dict(x, stats, ...)."""
        torch = _torch()
        _require_cuda_f64(b, self.m, "b")
        for t, nn, name in [(x_ref, self.n, "x_ref"), (x0, self.n, "x0"), (z0, self.m, "z0")]:
            if t is not None:
                _require_cuda_f64(t, nn, name)
        if x is None:
            x = torch.empty(self.n, dtype=torch.float64, device=b.device)
        z = torch.empty(self.m, dtype=torch.float64, device=b.device) if return_z else None
        idx = torch.zeros(max(2 * min(max_iter, 10**7), 2), dtype=torch.int32, device=b.device) if record else None
        ext = _r.RebkSolveExt(_dptr(x_ref), _dptr(x0), _dptr(z0), _dptr(z), _dptr(idx), int(k0), int(stream_id))
        ro = _r.RebkRefineOpts(_r.REBK_FP32, int(max_outer), int(inner_iters), float(inner_reduction))
        stats = _r.RebkStats()
        st = _r.load().rebk_sparse_solve_refined(self._h, ctypes.c_void_p(b.data_ptr()),
                                                 ctypes.c_void_p(x.data_ptr()), float(tol), int(max_iter),
                                                 int(seed), ctypes.byref(ro), ctypes.byref(ext), ctypes.byref(stats))
        _r.check(st, allow)
        out = {"x": x, "stats": stats.as_dict(), "status": st}
        if return_z:
            out["z"] = z
        if record:
            out["idx"] = idx[: 2 * stats.iterations].view(-1, 2)
        return out


class BatchSolver:
    """Many independent systems A_i x = b_i, each with up to eight right-hand
    sides, solved together (mixed precision with FP64 refinement, one
    persistent launch per refinement pass, one CUDA graph per solve).

    As: list of float64 numpy arrays (m_i x n_i).  tau: block size (0 =
    autotune at the first solve with reference solutions).  alpha: per-system
    step sizes or None (1.75 / beta_max each).  col_path: column-step tile shape
    for blocks of 16 / 32 columns (0: 16-byte row vectors, 1: lane per column;
    autotuned with tau = 0).  cluster: CTAs per thread-block cluster for the
    systems predicted to run longest (1: one CTA per system; 0: library
    choice, 2); joint_frac: their threshold as a fraction of the mean load per
    CTA (0: 0.25, and no clusters when every system qualifies)."""

    def __init__(self, As, nrhs: int = 8, tau: int = 0, alpha=None, max_outer: int = 0,
                 check_every: int = 0, inner_reduction: float = 0.0, stream=None, col_path: int = 0,
                 cluster: int = 0, joint_frac: float = 0.0):
        lib = _r.load()
        self.count = len(As)
        self._As = [np.ascontiguousarray(A, dtype=np.float64) for A in As]
        self.m = np.array([A.shape[0] for A in self._As], dtype=np.int64)
        self.n = np.array([A.shape[1] for A in self._As], dtype=np.int64)
        ptrs = (ctypes.c_void_p * self.count)(*[A.ctypes.data for A in self._As])
        al = None
        if alpha is not None:
            self._alpha = np.ascontiguousarray(alpha, dtype=np.float64)
            al = self._alpha.ctypes.data_as(ctypes.c_void_p)
        opt = _r.RebkBatchOptions(tau, nrhs, max_outer, check_every, inner_reduction,
                                  None if stream is None else ctypes.c_void_p(stream.cuda_stream), int(col_path),
                                  int(cluster), float(joint_frac))
        h = ctypes.c_void_p()
        st = lib.rebk_batch_create(ctypes.byref(h), self.count, self.m.ctypes.data_as(ctypes.c_void_p),
                                   self.n.ctypes.data_as(ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p), 0,
                                   al, ctypes.byref(opt))
        _r.check(st)
        self._h = h
        self.nrhs = nrhs
        self.mrow = np.concatenate([[0], np.cumsum(self.m)])
        self.nrow = np.concatenate([[0], np.cumsum(self.n)])

    def close(self):
        if getattr(self, "_h", None):
            _r.load().rebk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stack_rhs(self, blocks, rows) -> "torch.Tensor":
        """Concatenate per-system (rows_i x nrhs) blocks into one CUDA tensor."""
        torch = _torch()
        cat = np.concatenate([np.asarray(b, dtype=np.float64).reshape(r, self.nrhs)
                              for b, r in zip(blocks, rows)], axis=0)
        return torch.from_numpy(np.ascontiguousarray(cat)).cuda()

    def split_x(self, X):
        Xn = X.cpu().numpy() if hasattr(X, "cpu") else np.asarray(X)
        return [Xn[self.nrow[i]:self.nrow[i + 1]] for i in range(self.count)]

    def solve(self, B, X_ref=None, tol: float = 1e-8, max_iter: int = 200000, inner_iters: int = 0,
              seed: int = 0, X0=None, Z0=None, record_iters: int = 0, return_z: bool = False):
        """B: CUDA float64 (sum m_i) x nrhs; X_ref: (sum n_i) x nrhs or None;
        X0 / Z0: starting points laid out like X / B, or None (x = 0, z = b).
        record_iters > 0: also return "idx", a (count, record_iters, 2) int32
        tensor of each system's block draws (j_k, i_k) for iterations
        1..record_iters (entries past a system's last iteration are -1);
        return_z: also return "z", the final z laid out like B
        (rebk_batch_record).  Returns dict(x, status (per system), stats)."""
        torch = _torch()
        lib = _r.load()
        X = torch.empty((int(self.nrow[-1]), self.nrhs), dtype=torch.float64, device=B.device)
        status = torch.zeros(self.count, dtype=torch.int32, device=B.device)
        stats = _r.RebkBatchStats()
        ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        idx = torch.full((self.count, record_iters, 2), -1, dtype=torch.int32, device=B.device) \
            if record_iters > 0 else None
        Z = torch.empty((int(self.mrow[-1]), self.nrhs), dtype=torch.float64, device=B.device) if return_z else None
        recording = idx is not None or Z is not None
        if recording:
            _r.check(lib.rebk_batch_record(self._h, ptr(idx), int(record_iters), ptr(Z)))
        try:
            st = lib.rebk_batch_solve_ex(self._h, ptr(B), ptr(X), ptr(X_ref), ptr(X0), ptr(Z0),
                                         float(tol), int(max_iter), int(inner_iters), int(seed),
                                         ctypes.c_void_p(status.data_ptr()), ctypes.byref(stats))
        finally:
            if recording:
                lib.rebk_batch_record(self._h, None, 0, None)
        _r.check(st)
        out = {"x": X, "status": status.cpu().numpy(), "stats": stats.as_dict()}
        if idx is not None:
            out["idx"] = idx
        if Z is not None:
            out["z"] = Z
        return out


class WarmStartNet:
    """The learned warm start y = W3 relu(W2 relu(W1 b)) for a fixed A (m x n):
    x0 = A^T y and z0 = b - A x0 start the solve (see rebk.h)."""

    def __init__(self, A, hidden: int = 512, batch_capacity: int = 256, init_weights=None, seed: int = 0,
                 stream=None):
        lib = _r.load()
        An = np.ascontiguousarray(A, dtype=np.float64)
        self.m, self.n = An.shape
        self.hidden = hidden
        self.shapes = [(hidden, self.m), (hidden, hidden), (self.m, hidden)]
        arr = None
        if init_weights is not None:
            self._init = [np.ascontiguousarray(w, dtype=np.float32) for w in init_weights]
            arr = (ctypes.c_void_p * 3)(*[w.ctypes.data for w in self._init])
        h = ctypes.c_void_p()
        st = lib.rebk_mlp_create(ctypes.byref(h), An.ctypes.data_as(ctypes.c_void_p), self.m, self.n, 0, hidden,
                                 batch_capacity, None if arr is None else ctypes.cast(arr, ctypes.c_void_p),
                                 seed, None if stream is None else ctypes.c_void_p(stream.cuda_stream))
        _r.check(st)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _r.load().rebk_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, Bm):
        """Bm: CUDA float64 (batch x m).  Returns Y (batch x m)."""
        torch = _torch()
        Y = torch.empty_like(Bm)
        _r.check(_r.load().rebk_mlp_forward(self._h, ctypes.c_void_p(Bm.data_ptr()), Bm.shape[0],
                                            ctypes.c_void_p(Y.data_ptr())))
        return Y

    LOSSES = {"x": 0, "y_rel": 1}

    def set_loss(self, loss: str = "x", out_scale: float = 1.0):
        """loss "x": mean ||A^T y - x_ls||^2 (targets x_ls, N x n); "y_rel": mean
        ||y - y*||^2 / ||y*||^2 (targets y* = (A^T)^+ x_ls, N x m).  out_scale
        multiplies the network output (see rebk_mlp_set_loss)."""
        _r.check(_r.load().rebk_mlp_set_loss(self._h, self.LOSSES[loss], float(out_scale)))
        self.loss, self.out_scale = loss, float(out_scale)

    def fit(self, Bm, T, steps: int, lr: float = 1e-3, batch: int = 256) -> list:
        """Adam over `steps` minibatches of `batch` consecutive rows of Bm (CUDA,
        N x m) and T (the targets of the selected loss), cycling through the
        rows in the caller's order, with the learning rate on a cosine schedule
        from lr to 0.  Returns the minibatch losses."""
        N = int(Bm.shape[0])
        if N < batch:
            raise ValueError("fewer training rows than one minibatch")
        nb = N // batch
        losses = []
        for k in range(steps):
            i = (k % nb) * batch
            lr_k = lr * 0.5 * (1.0 + math.cos(math.pi * k / steps))
            losses.append(self.train_step(Bm[i:i + batch], T[i:i + batch], lr=lr_k))
        return losses

    def gradients(self, Bm, Xls):
        grads = [np.zeros(s, dtype=np.float32) for s in self.shapes]
        arr = (ctypes.c_void_p * 3)(*[g.ctypes.data for g in grads])
        loss = ctypes.c_double()
        _r.check(_r.load().rebk_mlp_gradients(self._h, ctypes.c_void_p(Bm.data_ptr()),
                                              ctypes.c_void_p(Xls.data_ptr()), Bm.shape[0], ctypes.byref(loss),
                                              ctypes.cast(arr, ctypes.c_void_p)))
        return loss.value, grads

    def train_step(self, Bm, Xls, lr: float = 1e-3) -> float:
        loss = ctypes.c_double()
        _r.check(_r.load().rebk_mlp_train_step(self._h, ctypes.c_void_p(Bm.data_ptr()),
                                               ctypes.c_void_p(Xls.data_ptr()), Bm.shape[0], float(lr),
                                               ctypes.byref(loss)))
        return loss.value

    def weights(self):
        ws = [np.zeros(s, dtype=np.float32) for s in self.shapes]
        arr = (ctypes.c_void_p * 3)(*[w.ctypes.data for w in ws])
        _r.check(_r.load().rebk_mlp_get_weights(self._h, ctypes.cast(arr, ctypes.c_void_p)))
        return ws

    def warm_start_batch(self, solver: "Solver", B, count: int, group: int = 1):
        """(X0, Z0) for `count` right-hand sides in the grouped layout of B
        (CUDA float64; right-hand side j = column j % group of block j // group,
        blocks of m x group), e.g. BatchSolver.solve's X0 / Z0 for systems sharing A."""
        torch = _torch()
        X0 = torch.empty((count // group * self.n, group), dtype=torch.float64, device=B.device)
        Z0 = torch.empty((count // group * self.m, group), dtype=torch.float64, device=B.device)
        _r.check(_r.load().rebk_warm_start_batch(solver._h, self._h, ctypes.c_void_p(B.data_ptr()), int(count),
                                                 int(group), ctypes.c_void_p(X0.data_ptr()),
                                                 ctypes.c_void_p(Z0.data_ptr())))
        return X0, Z0

    def warm_start(self, solver: "Solver", b):
        """(x0, z0) for solver.solve / solve_refined."""
        torch = _torch()
        x0 = torch.empty(solver.n, dtype=torch.float64, device=b.device)
        z0 = torch.empty(solver.m, dtype=torch.float64, device=b.device)
        _r.check(_r.load().rebk_warm_start(solver._h, self._h, ctypes.c_void_p(b.data_ptr()),
                                           ctypes.c_void_p(x0.data_ptr()), ctypes.c_void_p(z0.data_ptr())))
        return x0, z0
