"""Python face of the FP64 REBK oracle (TEST INFRASTRUCTURE ONLY).

The iteration itself (Algorithm 1 of Du, Si, Sun, arXiv:2001.04179) runs in
the plain C file ``rebk_oracle.c`` next to this one, compiled with
-ffp-contract=off.  The rest is numpy, one library call per mathematical step:

* ``pinv_solve``: A^+ b from the SVD (the paper's target, Section 1).
* ``mean_closed_form``: E[z^k] and E[x^k] from the proof of Theorem ner
  (the recursions for E[z^k] and E[x^k - A^+ b]).
* ``beta_max``: beta^I_max and beta^J_max of Section 2.2 from the exact
  spectral norms of the block Gram matrices.
* ``bound_ner`` / ``bound_estz`` / ``bound_main``: right-hand sides of
  Theorem ner, Lemma estz and Theorem main.
* ``refine``: the mixed-precision outer loop (a reading of ours, the paper is
  silent): FP64 residuals f = b - z - A x, g = A^T z, Algorithm 1 on
  corrections with the reduced-precision matrix, FP64 update of x and z
  through the duals.
* ``mlp_forward`` / ``mlp_backward``: the warm-start network in FP64.
* ``rebk_sparse``: Algorithm 1 over the stored entries of a CSR matrix, for
  matrices whose dense form does not fit (numpy, the same draws as ``rebk``).
* ``rebk_free``: the iteration with index sets drawn without a partition (a
  reading of Section 4's variants), in C next to Algorithm 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build_oracle", "lib",
    "philox", "uniform", "pick",
    "block_norms", "cdf", "tables",
    "rebk", "rebk_correction", "rebk_sparse", "rebk_free", "uniform_slot",
    "pinv_solve", "mean_closed_form", "beta_max",
    "bound_ner", "bound_estz", "bound_main",
    "round_fp32", "round_bf16",
    "dual_residuals", "refine",
    "mlp_init", "mlp_forward", "mlp_backward", "mlp_loss",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rebk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


# Builds of the same C file.  "parity" is the reference every test uses (no FMA
# contraction).  The other two exist only to time the oracle as a CPU baseline:
# "fast" lets the compiler contract products into FMAs at -O3; "omp" adds
# -fopenmp, which splits the block products over all host threads (the pragmas
# in rebk_oracle.c keep each value's summation order).  Host code here is
# built for the generic target of the machine's compiler (no -march flag), so
# the same commands work on x86-64 and on Arm.
_VARIANTS = {
    "parity": (["-O2", "-ffp-contract=off", "-fno-fast-math"], "liborc.so"),
    "fast": (["-O3", "-ffp-contract=fast"], "liborc_fast.so"),
    "omp": (["-O3", "-ffp-contract=fast", "-fopenmp"], "liborc_omp.so"),
}


def build_oracle(force: bool = False, variant: str = "parity") -> str:
    """Compile rebk_oracle.c with gcc into _build/<lib>.so (see _VARIANTS)."""
    flags, name = _VARIANTS[variant]
    so = os.path.join(_BUILD, name)
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc"] + flags + ["-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


_variant_libs = {}


def _declare(L):
    L.orc_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
    L.orc_philox4x64_10.restype = None
    L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
    L.orc_uniform.restype = ctypes.c_double
    L.orc_pick.argtypes = [_f64p, ctypes.c_int64, ctypes.c_double]
    L.orc_pick.restype = ctypes.c_int64
    L.orc_block_norms.argtypes = [ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_int64,
                                  ctypes.c_int64, _i64p, ctypes.c_int64, _i64p, _f64p, _f64p]
    L.orc_block_norms.restype = None
    L.orc_cdf.argtypes = [_f64p, ctypes.c_int64, _f64p]
    L.orc_cdf.restype = None
    L.orc_rebk.argtypes = [ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_int64,
                           ctypes.c_int64, _i64p, ctypes.c_int64, _i64p,
                           _f64p, _f64p, _f64p, _f64p,
                           ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                           _f64p, _f64p, _f64p,
                           ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_double,
                           _i32p, _f64p]
    L.orc_rebk.restype = ctypes.c_int64
    L.orc_rebk_correction.argtypes = [ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_int64,
                                      ctypes.c_int64, _i64p, ctypes.c_int64, _i64p,
                                      _f64p, _f64p, _f64p, _f64p,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                      _f64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                      ctypes.c_int64, ctypes.c_int64, _f64p, _f64p, ctypes.c_double,
                                      _i32p, _f64p]
    L.orc_rebk_correction.restype = ctypes.c_int64
    L.orc_uniform_slot.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
    L.orc_uniform_slot.restype = ctypes.c_double
    L.orc_rebk_free.argtypes = [ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_int64,
                                _f64p, _f64p, _f64p, _f64p, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                _f64p, _f64p, _f64p,
                                ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_double,
                                _i32p, _i64p, _i64p, _f64p]
    L.orc_rebk_free.restype = ctypes.c_int64
    return L


def lib(variant: str = "parity"):
    global _lib
    with _lock:
        if variant == "parity":
            if _lib is None:
                _lib = _declare(ctypes.CDLL(build_oracle()))
            return _lib
        if variant not in _variant_libs:
            _variant_libs[variant] = _declare(ctypes.CDLL(build_oracle(variant=variant)))
        return _variant_libs[variant]


def _p(a, t=_f64p):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Sampling (Algorithm 1, "pick j with probability ...")
# --------------------------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    """Philox4x64-10 block for a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c, _u64p), _p(k, _u64p), _p(out, _u64p))
    return out


def uniform(seed: int, stream: int, d: int) -> float:
    return lib().orc_uniform(seed, stream, d)


def pick(cdf_table: np.ndarray, u: float) -> int:
    c = _f64(cdf_table)
    return int(lib().orc_pick(_p(c), c.size, u))


def block_norms(A: np.ndarray, row_off: np.ndarray, col_off: np.ndarray):
    """(nr, nc): squared Frobenius norms of the row blocks A_{I_i,:} and of the
    column blocks A_{:,J_j}."""
    A = _f64(A)
    ro = np.ascontiguousarray(row_off, dtype=np.int64)
    co = np.ascontiguousarray(col_off, dtype=np.int64)
    s, t = ro.size - 1, co.size - 1
    nr = np.zeros(s)
    nc = np.zeros(t)
    lib().orc_block_norms(A.shape[0], A.shape[1], _p(A), A.shape[1], s, _p(ro, _i64p), t,
                          _p(co, _i64p), _p(nr), _p(nc))
    return nr, nc


def cdf(w: np.ndarray) -> np.ndarray:
    w = _f64(w)
    out = np.zeros_like(w)
    lib().orc_cdf(_p(w), w.size, _p(out))
    return out


def tables(A, row_off, col_off):
    nr, nc = block_norms(A, row_off, col_off)
    return nr, nc, cdf(nr), cdf(nc)


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------

def rebk(A, b, row_off, col_off, alpha, seed, iters, stream=0, k0=0, z0=None, x0=None,
         check_every=0, x_ref=None, tol=0.0, record=False, norms=None, variant="parity"):
    """Run iterations k0+1 .. k0+iters of Algorithm 1.

    z0 defaults to b and x0 to 0 (Section 3).  ``norms`` may pass the block
    norms of another matrix (used for the sampling table and the step sizes);
    by default they are those of A.  Returns dict(x, z, iters, idx) where idx
    is an (iters, 2) array of (j_k, i_k) when ``record``.  ``variant`` picks
    the build (see _VARIANTS; only "parity" is a reference).
    """
    A = _f64(A)
    m, n = A.shape
    ro = np.ascontiguousarray(row_off, dtype=np.int64)
    co = np.ascontiguousarray(col_off, dtype=np.int64)
    if norms is None:
        nr, nc, cr, cc = tables(A, ro, co)
    else:
        nr, nc = _f64(norms[0]), _f64(norms[1])
        cr, cc = cdf(nr), cdf(nc)
    b = _f64(b)
    z = _f64(b.copy() if z0 is None else z0).copy()
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    idx = np.zeros((max(iters, 1), 2), dtype=np.int32) if record else None
    xr = None if x_ref is None else _f64(x_ref)
    work = np.zeros(max(np.max(np.diff(ro)), np.max(np.diff(co))) + 1)
    done = lib(variant).orc_rebk(m, n, _p(A), n, ro.size - 1, _p(ro, _i64p), co.size - 1, _p(co, _i64p),
                          _p(nr), _p(nc), _p(cr), _p(cc), float(alpha), seed, stream, k0,
                          _p(b), _p(z), _p(x), iters, check_every, _p(xr), float(tol),
                          _p(idx, _i32p), _p(work))
    return {"x": x, "z": z, "iters": int(done), "idx": None if idx is None else idx[:done]}


def uniform_slot(seed: int, stream: int, d: int, q: int) -> float:
    """u of slot q of draw d (Philox counter (d, q, 0, 0)); slot 0 is ``uniform``."""
    return lib().orc_uniform_slot(seed, stream, d, q)


def rebk_free(A, b, tau_r, tau_c, alpha, seed, iters, stream=0, k0=0, z0=None, x0=None,
              check_every=0, x_ref=None, tol=0.0, record=False):
    """Iterations k0+1 .. k0+iters of Algorithm 1 with index sets drawn without a
    partition (see orc_rebk_free in rebk_oracle.c: tau_c columns and tau_r rows
    drawn independently with probabilities proportional to their squared norms,
    the step of Algorithm 1 on the drawn submatrices).  Row and column norms
    come from ``block_norms`` with blocks of one row / column.  Returns
    dict(x, z, iters, idx) with idx an (iters, tau_c + tau_r) array (column
    draws, then row draws) when ``record``."""
    A = _f64(A)
    m, n = A.shape
    rn, cn = block_norms(A, np.arange(m + 1), np.arange(n + 1))
    cr, cc = cdf(rn), cdf(cn)
    b = _f64(b)
    z = _f64(b.copy() if z0 is None else z0).copy()
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    idx = np.zeros((max(iters, 1), tau_c + tau_r), dtype=np.int32) if record else None
    xr = None if x_ref is None else _f64(x_ref)
    jset = np.zeros(tau_c, dtype=np.int64)
    iset = np.zeros(tau_r, dtype=np.int64)
    work = np.zeros(tau_c + tau_r)
    done = lib().orc_rebk_free(m, n, _p(A), n, _p(rn), _p(cn), _p(cr), _p(cc), tau_r, tau_c, float(alpha),
                               seed, stream, k0, _p(b), _p(z), _p(x), iters, check_every, _p(xr), float(tol),
                               _p(idx, _i32p), _p(jset, _i64p), _p(iset, _i64p), _p(work))
    return {"x": x, "z": z, "iters": int(done), "idx": None if idx is None else idx[:done]}


def rebk_correction(Alo, f, g, row_off, col_off, norms, alpha, seed, iters, stream=0, k0=0,
                    state=None, check_every=0, xbase=None, x_ref=None, err_abs=0.0, record=False):
    """Algorithm 1 on corrections (see rebk_oracle.c): returns dict(dz, dx, s, v, iters, idx)."""
    Alo = _f64(Alo)
    m, n = Alo.shape
    ro = np.ascontiguousarray(row_off, dtype=np.int64)
    co = np.ascontiguousarray(col_off, dtype=np.int64)
    nr, nc = _f64(norms[0]), _f64(norms[1])
    cr, cc = cdf(nr), cdf(nc)
    f, g = _f64(f), _f64(g)
    if state is None:
        dz, dx, s, v = np.zeros(m), np.zeros(n), np.zeros(n), np.zeros(m)
    else:
        dz, dx, s, v = (_f64(a).copy() for a in state)
    idx = np.zeros((max(iters, 1), 2), dtype=np.int32) if record else None
    work = np.zeros(max(np.max(np.diff(ro)), np.max(np.diff(co))) + 1)
    xb = None if xbase is None else _f64(xbase)
    xr = None if x_ref is None else _f64(x_ref)
    done = lib().orc_rebk_correction(m, n, _p(Alo), n, ro.size - 1, _p(ro, _i64p), co.size - 1,
                                     _p(co, _i64p), _p(nr), _p(nc), _p(cr), _p(cc), float(alpha),
                                     seed, stream, k0, _p(f), _p(g), _p(dz), _p(dx), _p(s), _p(v),
                                     iters, check_every, _p(xb), _p(xr), float(err_abs),
                                     _p(idx, _i32p), _p(work))
    return {"dz": dz, "dx": dx, "s": s, "v": v, "iters": int(done),
            "idx": None if idx is None else idx[:done]}


def rebk_sparse(m, n, indptr, indices, data, b, row_off, col_off, alpha, seed, iters, stream=0, k0=0,
                record=False):
    """Iterations k0+1 .. k0+iters of Algorithm 1 on a matrix given in CSR form
    (indptr (m + 1), indices, data), from z^0 = b, x^0 = 0, for matrices whose
    dense form is too large for ``rebk``.  The same steps with the products
    written over the stored entries: the squared block norms are sums of the
    squared entries of each block; w = A_J^T z adds data * z[row] into the
    entry's column, z -= c_J A_J w subtracts c_J data w[column] from the entry's
    row; r = A_I x - b_I + z_I and x -= c_I A_I^T r likewise over the row block.
    Block picks use the same Philox draws and table search as ``rebk``.
    Returns dict(x, z, idx)."""
    indptr = np.asarray(indptr, dtype=np.int64)
    cols = np.asarray(indices, dtype=np.int64)
    vals = _f64(data)
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(indptr))
    ro = np.asarray(row_off, dtype=np.int64)
    co = np.asarray(col_off, dtype=np.int64)
    s, t = ro.size - 1, co.size - 1
    rblk = np.searchsorted(ro, rows, side="right") - 1   # row block of each entry
    cblk = np.searchsorted(co, cols, side="right") - 1   # column block of each entry
    nr = np.bincount(rblk, weights=vals * vals, minlength=s)
    nc = np.bincount(cblk, weights=vals * vals, minlength=t)
    cr, cc = cdf(nr), cdf(nc)
    b = _f64(b)
    z = b.copy()
    x = np.zeros(n)
    idx = np.zeros((max(iters, 1), 2), dtype=np.int32)
    for kk in range(iters):
        k = k0 + kk + 1
        j = pick(cc, uniform(seed, stream, 2 * (k - 1)))
        i = pick(cr, uniform(seed, stream, 2 * (k - 1) + 1))
        idx[kk] = (j, i)
        # column step on the entries of A_{:,J_j}
        e = np.nonzero(cblk == j)[0]
        w = np.bincount(cols[e] - co[j], weights=vals[e] * z[rows[e]], minlength=co[j + 1] - co[j])
        cJ = alpha / nc[j] if nc[j] > 0 else 0.0
        z = z - np.bincount(rows[e], weights=cJ * vals[e] * w[cols[e] - co[j]], minlength=m)
        # row step on the entries of A_{I_i,:}
        e = np.arange(indptr[ro[i]], indptr[ro[i + 1]])
        h = ro[i + 1] - ro[i]
        r = np.bincount(rows[e] - ro[i], weights=vals[e] * x[cols[e]], minlength=h) - b[ro[i]:ro[i + 1]] \
            + z[ro[i]:ro[i + 1]]
        cI = alpha / nr[i] if nr[i] > 0 else 0.0
        x = x - np.bincount(cols[e], weights=cI * vals[e] * r[rows[e] - ro[i]], minlength=n)
    return {"x": x, "z": z, "idx": idx[:iters] if record else None}


# --------------------------------------------------------------------------
# Closed forms and bounds (Section 2)
# --------------------------------------------------------------------------

def pinv_solve(A, b, rcond=1e-12):
    """A^+ b through the SVD (numpy.linalg.pinv)."""
    return np.linalg.pinv(_f64(A), rcond=rcond) @ _f64(b)


def mean_closed_form(A, b, alpha, k, z0=None, x0=None):
    """E[z^k] = (I - alpha A A^T/||A||_F^2)^k z^0 and
    E[x^k] = A^+ b + (I - alpha A^T A/||A||_F^2)^k (x^0 - A^+ b)
             - alpha k (I - alpha A^T A/||A||_F^2)^k A^T z^0 / ||A||_F^2
    (proof of Theorem ner)."""
    A = _f64(A)
    m, n = A.shape
    fro2 = float(np.sum(A * A))
    z0 = _f64(b) if z0 is None else _f64(z0)
    x0 = np.zeros(n) if x0 is None else _f64(x0)
    xs = pinv_solve(A, b)
    Pz = np.linalg.matrix_power(np.eye(m) - alpha * (A @ A.T) / fro2, k)
    Px = np.linalg.matrix_power(np.eye(n) - alpha * (A.T @ A) / fro2, k)
    Ez = Pz @ z0
    Ex = xs + Px @ (x0 - xs) - alpha * k * (Px @ (A.T @ z0)) / fro2
    return Ex, Ez


def beta_max(A, row_off, col_off):
    """(beta^I_max, beta^J_max) of Section 2.2: the largest ||block||_2^2 /
    ||block||_F^2 over row blocks and over column blocks, spectral norms from
    the eigenvalues of the block Gram matrices (numpy.linalg.eigvalsh).
    Blocks of zero norm are skipped."""
    A = _f64(A)
    bi = 0.0
    for i in range(len(row_off) - 1):
        B = A[row_off[i]:row_off[i + 1], :]
        f2 = float(np.sum(B * B))
        if f2 > 0:
            bi = max(bi, float(np.linalg.eigvalsh(B @ B.T)[-1]) / f2)
    bj = 0.0
    for j in range(len(col_off) - 1):
        B = A[:, col_off[j]:col_off[j + 1]]
        f2 = float(np.sum(B * B))
        if f2 > 0:
            bj = max(bj, float(np.linalg.eigvalsh(B.T @ B)[-1]) / f2)
    return bi, bj


def _sv(A):
    s = np.linalg.svd(_f64(A), compute_uv=False)
    r = int(np.sum(s > s[0] * 1e-12)) if s.size and s[0] > 0 else 0
    return s[:r]


def bound_ner(A, b, alpha, k, z0=None, x0=None):
    """Theorem ner: delta^k (||x^0 - A^+ b|| + alpha k ||A^T z^0|| / ||A||_F^2)."""
    A = _f64(A)
    sv = _sv(A)
    fro2 = float(np.sum(A * A))
    delta = float(np.max(np.abs(1.0 - alpha * sv ** 2 / fro2)))
    z0 = _f64(b) if z0 is None else _f64(z0)
    x0 = np.zeros(A.shape[1]) if x0 is None else _f64(x0)
    xs = pinv_solve(A, b)
    return delta ** k * (np.linalg.norm(x0 - xs) + alpha * k * np.linalg.norm(A.T @ z0) / fro2)


def _eta_rho(A, alpha, row_off, col_off):
    A = _f64(A)
    sv = _sv(A)
    fro2 = float(np.sum(A * A))
    bI, bJ = beta_max(A, row_off, col_off)
    sr2 = sv[-1] ** 2
    eta = 1.0 - (2 * alpha - alpha ** 2 * bI) * sr2 / fro2
    rho = 1.0 - (2 * alpha - alpha ** 2 * bJ) * sr2 / fro2
    return eta, rho, bI, bJ, fro2


def bound_estz(A, b, alpha, k, row_off, col_off, z0=None):
    """Lemma estz: rho^k ||z^0 - b_perp||^2, b_perp = (I - A A^+) b."""
    A = _f64(A)
    eta, rho, bI, bJ, fro2 = _eta_rho(A, alpha, row_off, col_off)
    z0 = _f64(b) if z0 is None else _f64(z0)
    bperp = _f64(b) - A @ pinv_solve(A, b)
    return rho ** k * float(np.sum((z0 - bperp) ** 2))


def bound_main(A, b, alpha, k, row_off, col_off, eps=1.0, z0=None, x0=None):
    """Theorem main: (1+eps)^k eta^k ||x^0 - A^+ b||^2
    + (1 + 1/eps) alpha^2 beta^I_max ||z^0 - b_perp||^2 / ||A||_F^2
      * sum_{l<k} rho^{k-l} (1+eps)^l eta^l."""
    A = _f64(A)
    eta, rho, bI, bJ, fro2 = _eta_rho(A, alpha, row_off, col_off)
    z0 = _f64(b) if z0 is None else _f64(z0)
    x0 = np.zeros(A.shape[1]) if x0 is None else _f64(x0)
    xs = pinv_solve(A, b)
    bperp = _f64(b) - A @ xs
    tail = sum(rho ** (k - l) * (1 + eps) ** l * eta ** l for l in range(k))
    return ((1 + eps) ** k * eta ** k * float(np.sum((x0 - xs) ** 2))
            + (1 + 1 / eps) * alpha ** 2 * bI * float(np.sum((z0 - bperp) ** 2)) / fro2 * tail)


# --------------------------------------------------------------------------
# Reduced-precision storage and the refinement loop (our reading)
# --------------------------------------------------------------------------

def round_fp32(A):
    """FP64 -> FP32, round to nearest even, as FP64 values."""
    return _f64(A).astype(np.float32).astype(np.float64)


def round_bf16(A):
    """FP64 -> FP32 -> BF16, each round to nearest even, as FP64 values.
    (Inf/NaN inputs are not expected.)"""
    f = _f64(A).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def dual_residuals(A, b, z, x):
    """f = b - z - A x and g = A^T z in FP64.  Both vanish exactly at
    (x, z) = (A^+ b, (I - A A^+) b)."""
    A = _f64(A)
    return _f64(b) - _f64(z) - A @ _f64(x), A.T @ _f64(z)


def refine(A, b, Alo, row_off, col_off, alpha, seed, inner_iters, outer_max=50,
           x_ref=None, tol=1e-8, stream=0, x0=None, z0=None, inner_reduction=None):
    """Mixed-precision REBK with FP64 refinement (our reading; the paper is silent).

    State (x, z) in FP64 with x0 = 0, z0 = b unless given.  Each outer pass:
      f = b - z - A x, g = A^T z                  (FP64, A)
      Algorithm 1 on corrections with Alo          (rebk_correction)
      z <- z - A s,  x <- x + A^T v                (FP64, A)
    The random stream continues across passes (k0 advances).  A pass ends
    after ``inner_iters`` iterations, or earlier when x_ref is given and
    ||x + dx - x_ref|| <= max(tol ||x_ref||, inner_reduction * err_at_pass_start).
    Stops when ||x - x_ref|| <= tol ||x_ref|| (x_ref given) or after outer_max
    passes.  Block norms (sampling table, step sizes) are those of FP64 A.
    Returns dict(x, z, outer, inner_total, history).
    """
    A = _f64(A)
    m, n = A.shape
    nr, nc = block_norms(A, row_off, col_off)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    z = _f64(b).copy() if z0 is None else _f64(z0).copy()
    k0 = 0
    hist = []
    xr = None if x_ref is None else _f64(x_ref)
    refn = None if xr is None else float(np.linalg.norm(xr))
    for outer in range(1, outer_max + 1):
        f, g = dual_residuals(A, b, z, x)
        err_abs = 0.0
        check = 0
        if xr is not None:
            e0 = float(np.linalg.norm(x - xr))
            if e0 <= tol * refn:
                return {"x": x, "z": z, "outer": outer - 1, "inner_total": k0, "history": hist}
            red = inner_reduction if inner_reduction is not None else 0.0
            err_abs = max(tol * refn, red * e0)
            check = 10
        r = rebk_correction(Alo, f, g, row_off, col_off, (nr, nc), alpha, seed, inner_iters,
                            stream=stream, k0=k0, check_every=check, xbase=x, x_ref=xr,
                            err_abs=err_abs)
        k0 += r["iters"]
        z = z - A @ r["s"]
        x = x + A.T @ r["v"]
        hist.append({"outer": outer, "inner": r["iters"],
                     "err": None if xr is None else float(np.linalg.norm(x - xr) / refn)})
    return {"x": x, "z": z, "outer": outer_max, "inner_total": k0, "history": hist}


# --------------------------------------------------------------------------
# Learned warm start network (FP64 reference)
# --------------------------------------------------------------------------

def mlp_init(sizes, seed):
    """Weights W_l (out x in) with N(0, 2/in) entries (He initialisation)."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((sizes[i + 1], sizes[i])) * np.sqrt(2.0 / sizes[i])
            for i in range(len(sizes) - 1)]


def mlp_forward(W, Bm, out_scale=1.0):
    """y = s W_L relu(... relu(W_1 b)) with output scale s: columns of Bm are
    inputs.  Returns (y, cache) with cache = pre-activations and activations
    per layer (the last pre-activation unscaled)."""
    acts = [_f64(Bm)]
    pres = []
    h = acts[0]
    for l, Wl in enumerate(W):
        p = Wl @ h
        pres.append(p)
        h = out_scale * p if l == len(W) - 1 else np.maximum(p, 0.0)
        acts.append(h)
    return h, (pres, acts)


def mlp_loss(W, A, Bm, T, loss="x", out_scale=1.0):
    """Mean over columns of the training loss of the warm start x^0 = A^T y:
    loss "x": ||A^T y - x_ls||^2 (T = x_ls, n x B);
    loss "y_rel": ||y - y*||^2 / ||y*||^2 (T = y* = (A^T)^+ x_ls, m x B)."""
    y, _ = mlp_forward(W, Bm, out_scale)
    if loss == "x":
        R = _f64(A).T @ y - _f64(T)
        return float(np.sum(R * R)) / Bm.shape[1]
    T = _f64(T)
    nt = np.sum(T * T, axis=0)
    d = np.sum((y - T) ** 2, axis=0)
    return float(np.sum(np.where(nt > 0, d / np.where(nt > 0, nt, 1.0), 0.0))) / Bm.shape[1]


def mlp_backward(W, A, Bm, T, loss="x", out_scale=1.0):
    """Gradients of mlp_loss w.r.t. each W_l by the chain rule.  dL/dy:
    loss "x": (2/B) A (A^T y - x_ls); loss "y_rel": (2/B) (y - y*) / ||y*||^2
    per column (0 for a zero target).  The output scale s multiplies the
    signal entering the last layer; then back through the linear layers and
    the ReLU masks (derivative 0 at 0)."""
    y, (pres, acts) = mlp_forward(W, Bm, out_scale)
    B = Bm.shape[1]
    if loss == "x":
        A = _f64(A)
        G = (2.0 / B) * (A @ (A.T @ y - _f64(T)))
    else:
        T = _f64(T)
        nt = np.sum(T * T, axis=0)
        G = (2.0 / B) * (y - T) * np.where(nt > 0, 1.0 / np.where(nt > 0, nt, 1.0), 0.0)
    G = out_scale * G
    grads = [None] * len(W)
    for l in range(len(W) - 1, -1, -1):
        if l < len(W) - 1:
            G = G * (pres[l] > 0)
        grads[l] = G @ acts[l].T
        G = W[l].T @ G
    return grads
