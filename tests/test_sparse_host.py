"""Sparse problems on the host: the generator's reference solution and the
C ABI's argument checks (no GPU work)."""
import ctypes

import numpy as np

from workloads import sparse_problem


def test_reference_solution_solves_the_normal_equations():
    p = sparse_problem(400, 120, 10, seed=3, x_ref="normal")
    A = p.dense()
    r = A.T @ (A @ p.x_ref - p.b)
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(A.T @ p.b)
    q = sparse_problem(400, 120, 10, seed=3, x_ref="lstsq")
    assert np.linalg.norm(q.x_ref - p.x_ref) <= 1e-10 * np.linalg.norm(q.x_ref)


def test_rows_have_distinct_sorted_columns_and_spread_norms():
    p = sparse_problem(300, 80, 12, seed=4, decades=1.0, x_ref=None)
    for i in range(p.m):
        cols = p.indices[p.indptr[i]:p.indptr[i + 1]]
        assert len(cols) == 12 and np.all(np.diff(cols) > 0)
    norms = np.sqrt(np.add.reduceat(p.data ** 2, p.indptr[:-1]))
    assert norms.max() / norms.min() > 4.0


def test_sparse_create_rejects_bad_csr_on_the_host():
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    h = ctypes.c_void_p()
    rp = np.array([0, 2, 3], dtype=np.int64)
    ci = np.array([1, 0, 2], dtype=np.int32)  # row 0 not increasing
    v = np.ones(3)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.rebk_sparse_create(ctypes.byref(h), 2, 3, P(rp), P(ci), P(v), 1, 1, 1.0, None) == R.REBK_EINVAL
    ci2 = np.array([0, 5, 2], dtype=np.int32)  # out of range
    assert lib.rebk_sparse_create(ctypes.byref(h), 2, 3, P(rp), P(ci2), P(v), 1, 1, 1.0, None) == R.REBK_EINVAL
    assert lib.rebk_sparse_create(ctypes.byref(h), 0, 3, P(rp), P(ci), P(v), 1, 1, 1.0, None) == R.REBK_EINVAL
    assert lib.rebk_sparse_solve(None, None, None, 0.0, 1, 0, None, None) == R.REBK_EINVAL
