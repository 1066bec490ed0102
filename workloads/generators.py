"""Seeded synthetic problems A x = b with a known A^+ b.

Matrix families follow Section 3.1 of Du, Si, Sun (arXiv:2001.04179):

* Type I:  A = U D V^T, U (m x r) and V (n x r) with orthonormal columns from
  QR of Gaussian matrices, D = diag of values uniform on (1, kappa).
* Type II: A = randn(m, n).

Inconsistent right-hand sides follow Section 3: b = A x + r with r in
null(A^T).  The remaining families (a Gaussian product G1 G2 of lower rank, a
prescribed-spectrum U diag(sigma) V^T, batches of uneven systems) are the
shapes the benchmark configurations name.

Every generator also returns x_ref = A^+ b computed from the factors it built
(a closed form of the construction), never from an iterative solver.  All
randomness comes from ``numpy.random.default_rng(seed)`` so results are the
same on every machine.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

__all__ = [
    "Problem",
    "contiguous_offsets",
    "gaussian_problem",
    "type1_problem",
    "product_problem",
    "spectrum_problem",
    "batched_problems",
    "small_cases",
    "SparseProblem",
    "sparse_problem",
]


@dataclasses.dataclass
class Problem:
    """One least-squares problem A x = b with its known minimum-norm solution."""

    A: np.ndarray          # m x n, float64, row-major
    b: np.ndarray          # m or m x nrhs
    x_ref: np.ndarray      # n or n x nrhs, = A^+ b
    rank: int
    name: str
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]


def contiguous_offsets(size: int, tau: int) -> np.ndarray:
    """Block offsets of the paper's contiguous partition (Section 3): blocks
    [0, tau), [tau, 2 tau), ..., the last one holding what is left."""
    if size <= 0 or tau <= 0:
        raise ValueError("size and tau must be positive")
    nb = -(-size // tau)
    off = np.minimum(np.arange(nb + 1, dtype=np.int64) * tau, size)
    return off


def _orth(mat: np.ndarray) -> np.ndarray:
    q, _ = np.linalg.qr(mat, mode="reduced")
    return q


def _null_residual(Q: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Component of g orthogonal to range(Q) (Q has orthonormal columns)."""
    return g - Q @ (Q.T @ g)


def gaussian_problem(m: int, n: int, seed: int, resid_ratio: float = 0.1,
                     nrhs: int = 0) -> Problem:
    """Type II A = randn(m, n), full rank almost surely.

    For m >= n: b = A x* + r with r in null(A^T), ||r|| = resid_ratio ||A x*||,
    so A^+ b = x*.  For m < n the system is consistent and underdetermined:
    b = A x*, A^+ b = A^T (A A^T)^{-1} b.
    """
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    k = max(nrhs, 1)
    xs = rng.standard_normal((n, k))
    if m >= n:
        Q = _orth(A)
        Ax = A @ xs
        g = rng.standard_normal((m, k))
        r = _null_residual(Q, g)
        scale = resid_ratio * np.linalg.norm(Ax, axis=0) / np.maximum(np.linalg.norm(r, axis=0), 1e-300)
        b = Ax + r * scale
        x_ref = xs
    else:
        b = A @ xs
        x_ref = A.T @ np.linalg.solve(A @ A.T, b)
    if nrhs == 0:
        b, x_ref = b[:, 0].copy(), x_ref[:, 0].copy()
    return Problem(A, b, x_ref, min(m, n), f"gaussian_{m}x{n}", {"seed": seed, "resid_ratio": resid_ratio})


def type1_problem(m: int, n: int, r: int, kappa: float, seed: int,
                  resid_ratio: float = 0.1) -> Problem:
    """Type I A = U D V^T (Section 3.1), rank r, inconsistent b = A x + r_perp.

    A^+ = V D^{-1} U^T, so A^+ b = V D^{-1} U^T b exactly by construction.
    """
    rng = np.random.default_rng(seed)
    U = _orth(rng.standard_normal((m, r)))
    V = _orth(rng.standard_normal((n, r)))
    d = 1.0 + (kappa - 1.0) * rng.random(r)
    A = (U * d) @ V.T
    x = rng.standard_normal(n)
    Ax = A @ x
    g = rng.standard_normal(m)
    rp = _null_residual(U, g)
    b = Ax + rp * (resid_ratio * np.linalg.norm(Ax) / max(np.linalg.norm(rp), 1e-300))
    x_ref = V @ ((U.T @ b) / d)
    return Problem(A, b, x_ref, r, f"type1_{m}x{n}_r{r}_k{kappa:g}", {"seed": seed, "kappa": kappa})


def product_problem(m: int, n: int, r: int, seed: int, noise: float = 0.01,
                    matmul: Optional[Callable] = None, nrhs: int = 0) -> Problem:
    """Rank-r A = G1 G2, G1 = randn(m, r), G2 = randn(r, n), b = A x* + N(0, noise^2).

    G1 has full column rank and G2 full row rank (almost surely, r <= m, n),
    so A^+ = G2^+ G1^+ = G2^T (G2 G2^T)^{-1} (G1^T G1)^{-1} G1^T.
    ``matmul`` may supply a faster product for large sizes (same result up to
    rounding); it defaults to numpy.
    """
    if not (r <= m and r <= n):
        raise ValueError("product_problem needs r <= min(m, n)")
    mm = matmul or (lambda a, b: a @ b)
    rng = np.random.default_rng(seed)
    G1 = rng.standard_normal((m, r))
    G2 = rng.standard_normal((r, n))
    k = max(nrhs, 1)
    xs = rng.standard_normal((n, k))
    A = np.ascontiguousarray(mm(G1, G2))
    b = mm(A, xs) + noise * rng.standard_normal((m, k))
    y = np.linalg.solve(mm(G1.T, G1), mm(G1.T, b))          # G1^+ b
    x_ref = mm(G2.T, np.linalg.solve(mm(G2, G2.T), y))       # G2^+ (G1^+ b)
    if nrhs == 0:
        b, x_ref = b[:, 0].copy(), x_ref[:, 0].copy()
    return Problem(A, b, x_ref, r, f"product_{m}x{n}_r{r}", {"seed": seed, "noise": noise})


def spectrum_problem(m: int, n: int, seed: int, latent: int = 32, noise: float = 1e-3,
                     nrhs: int = 1, sigma: Optional[np.ndarray] = None) -> Problem:
    """A = U diag(sigma) V^T with sigma_i = i^{-1/2} (m >= n, full column rank)
    and right-hand sides b = A (M c) + N(0, noise^2), M = randn(n, latent),
    c ~ N(0, I): a stream of related problems for the learned warm start.

    A^+ = V diag(1/sigma) U^T, so A^+ b follows from the factors.
    """
    if m < n:
        raise ValueError("spectrum_problem builds m >= n")
    rng = np.random.default_rng(seed)
    U = _orth(rng.standard_normal((m, n)))
    V = _orth(rng.standard_normal((n, n)))
    s = sigma if sigma is not None else 1.0 / np.sqrt(np.arange(1, n + 1, dtype=np.float64))
    A = (U * s) @ V.T
    M = rng.standard_normal((n, latent))
    C = rng.standard_normal((latent, nrhs))
    B = A @ (M @ C) + noise * rng.standard_normal((m, nrhs))
    X = V @ ((U.T @ B) / s[:, None])
    return Problem(A, B, X, n, f"spectrum_{m}x{n}", {"seed": seed, "latent": latent,
                                                      "noise": noise, "U": U, "V": V, "sigma": s, "M": M})


def batched_problems(count: int, seed: int, m_range=(200, 6000), n_range=(50, 2000),
                     deficient_frac: float = 0.3, nrhs: int = 8, noise: float = 0.01,
                     scale_down: int = 1) -> list:
    """Uneven independent systems: m ~ U[m_range], n ~ U[n_range]; a fraction
    built rank-deficient as P Q with inner dimension ceil(n/4); nrhs
    right-hand sides b = A X* + N(0, noise^2) each.  ``scale_down`` divides the
    size ranges (for tests).

    A^+ B is formed from the factors: (A^T A)^{-1} A^T B for full column rank,
    A^T (A A^T)^{-1} B for full row rank, Q^+ P^+ B for a product with full-rank
    factors (P^+ = (P^T P)^{-1} P^T, Q^+ = Q^T (Q Q^T)^{-1}).
    """
    rng = np.random.default_rng(seed)
    out = []
    for sid in range(count):
        m = int(rng.integers(m_range[0] // scale_down, m_range[1] // scale_down + 1))
        n = int(rng.integers(max(n_range[0] // scale_down, 2), n_range[1] // scale_down + 1))
        deficient = bool(rng.random() < deficient_frac)
        X = rng.standard_normal((n, nrhs))
        if deficient:
            k = -(-n // 4)
            P = rng.standard_normal((m, k))
            Qm = rng.standard_normal((k, n))
            A = P @ Qm
            B = A @ X + noise * rng.standard_normal((m, nrhs))
            if m >= k:
                y = np.linalg.solve(P.T @ P, P.T @ B)
                x_ref = Qm.T @ np.linalg.solve(Qm @ Qm.T, y)
                rank = k
            else:  # A = P Q has full row rank m
                x_ref = A.T @ np.linalg.solve(A @ A.T, B)
                rank = m
        else:
            A = rng.standard_normal((m, n))
            B = A @ X + noise * rng.standard_normal((m, nrhs))
            if m >= n:
                x_ref = np.linalg.solve(A.T @ A, A.T @ B)
            else:
                x_ref = A.T @ np.linalg.solve(A @ A.T, B)
            rank = min(m, n)
        out.append(Problem(np.ascontiguousarray(A), B, x_ref, rank, f"batch{sid}_{m}x{n}",
                           {"seed": seed, "sid": sid, "deficient": deficient}))
    return out


def small_cases(seed: int = 0) -> list:
    """The four kinds of system the paper's introduction lists (consistent or
    not, full rank or rank-deficient), over- and underdetermined, small enough
    for a dense SVD."""
    rng = np.random.default_rng(seed)
    cases = []

    def finish(A, b, name):
        x_ref = np.linalg.pinv(A, rcond=1e-12) @ b
        cases.append(Problem(A, b, x_ref, int(np.linalg.matrix_rank(A)), name, {}))

    # (1) consistent, full column rank, overdetermined
    A = rng.standard_normal((40, 12)); finish(A, A @ rng.standard_normal(12), "consistent_fullcol")
    # (2) consistent, rank-deficient, underdetermined
    A = rng.standard_normal((18, 5)) @ rng.standard_normal((5, 30)); finish(A, A @ rng.standard_normal(30), "consistent_deficient_under")
    # (3) inconsistent, full column rank
    A = rng.standard_normal((50, 10)); finish(A, rng.standard_normal(50), "inconsistent_fullcol")
    # (4) inconsistent, rank-deficient, overdetermined and underdetermined
    A = rng.standard_normal((36, 6)) @ rng.standard_normal((6, 20)); finish(A, rng.standard_normal(36), "inconsistent_deficient_over")
    A = rng.standard_normal((16, 5)) @ rng.standard_normal((5, 28)); finish(A, rng.standard_normal(16), "inconsistent_deficient_under")
    return cases


@dataclasses.dataclass
class SparseProblem:
    """A sparse least-squares problem in CSR form (row pointers int64, column
    indices int32 sorted within each row, FP64 values) with x_ref = A^+ b."""
    m: int
    n: int
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray
    b: np.ndarray
    x_ref: Optional[np.ndarray]
    name: str
    meta: dict

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def dense(self) -> np.ndarray:
        A = np.zeros((self.m, self.n))
        for i in range(self.m):
            lo, hi = self.indptr[i], self.indptr[i + 1]
            A[i, self.indices[lo:hi]] = self.data[lo:hi]
        return A


def sparse_problem(m: int, n: int, nnz_row: int, seed: int, noise: float = 0.01, decades: float = 1.0,
                   x_ref: str = "normal") -> SparseProblem:
    """Tomography-like sparse A: every row has nnz_row distinct columns drawn
    uniformly, values U(0, 1) * 10^{u_i} with u_i ~ U(0, decades) per row (row
    norms spread over `decades` decades); b = A x* + e, x* ~ N(0, I), e Gaussian
    with ||e|| ~ noise ||A x*||.

    x_ref = A^+ b by a direct method: "normal" solves A^T A x = A^T b by a dense
    Cholesky factorisation (A of full column rank, m >= n; forward error about
    kappa(A)^2 eps), "lstsq" uses a dense SVD least-squares solve (small cases,
    any shape), None skips it.
    """
    rng = np.random.default_rng(seed)
    if nnz_row > n:
        raise ValueError("nnz_row > n")
    indptr = np.arange(m + 1, dtype=np.int64) * nnz_row
    indices = np.empty(m * nnz_row, dtype=np.int32)
    for i in range(m):
        indices[i * nnz_row:(i + 1) * nnz_row] = np.sort(rng.choice(n, nnz_row, replace=False))
    scale = 10.0 ** rng.uniform(0.0, decades, m)
    data = rng.uniform(0.0, 1.0, m * nnz_row) * np.repeat(scale, nnz_row)
    xs = rng.standard_normal(n)
    rows = np.repeat(np.arange(m), nnz_row)
    ax = np.bincount(rows, weights=data * xs[indices], minlength=m)
    e = rng.standard_normal(m)
    b = ax + noise * np.linalg.norm(ax) / np.linalg.norm(e) * e
    p = SparseProblem(m, n, indptr, indices, data, b, None, f"sparse_{m}x{n}_{nnz_row}",
                      {"seed": seed, "noise": noise, "decades": decades, "x_star": xs})
    if x_ref == "lstsq":
        p.x_ref = np.linalg.lstsq(p.dense(), b, rcond=None)[0]
    elif x_ref == "normal":
        import scipy.linalg
        import scipy.sparse
        A = scipy.sparse.csr_matrix((data, indices, indptr), shape=(m, n))
        G = (A.T @ A).toarray()
        c = A.T @ b
        L = scipy.linalg.cho_factor(G, lower=True)
        p.x_ref = scipy.linalg.cho_solve(L, c)
    return p
