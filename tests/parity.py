"""Comparison helpers of the GPU parity tests (no GPU needed to import).

``assert_close(got, ref, tol)`` holds when both
  ||got - ref||_2   <= tol * ||ref||_2     (the vector as a whole), and
  max_i |got_i - ref_i| <= tol * max_i |ref_i|   (every entry),
so a few wrong entries cannot hide inside a small norm of the difference.
That is the bar for parity: the same iterations on both sides.

``assert_converged(x, x_ref, tol)`` is the bar of a solve stopped by the
paper's rule, ||x - x_ref||_2 <= tol ||x_ref||_2: a statement about the norm,
which is what the stop rule tested."""
import numpy as np


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_inf(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def assert_close(got, ref, tol, what=""):
    r2, ri = rel(got, ref), rel_inf(got, ref)
    assert r2 <= tol, f"{what} relative 2-norm difference {r2:.3e} > {tol:.1e}"
    assert ri <= tol, f"{what} largest entry difference {ri:.3e} > {tol:.1e} of the largest entry"


def assert_converged(x, x_ref, tol, what=""):
    r2 = rel(x, x_ref)
    assert r2 <= tol, f"{what} relative error {r2:.3e} > {tol:.1e}"
