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


def test_sparse_oracle_equals_the_dense_oracle():
    """The oracle's CSR form of Algorithm 1 (for matrices too large to store
    densely) against its dense form, pinned by the other oracle tests: same block
    picks, iterates equal up to summation order -- with ragged blocks, an offset
    into the random stream, and empty rows and columns."""
    import oracle as O
    from workloads import contiguous_offsets
    p = sparse_problem(300, 120, 8, seed=5, x_ref=None)
    rng = np.random.default_rng(6)
    keep = np.ones(p.nnz, dtype=bool)
    rows = np.repeat(np.arange(p.m), np.diff(p.indptr))
    keep[(rows % 11 == 4) | (p.indices % 13 == 7)] = False  # empty rows and columns
    indptr = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=p.m))]).astype(np.int64)
    indices, data = p.indices[keep], p.data[keep]
    A = np.zeros((p.m, p.n))
    A[rows[keep], indices] = data
    b = rng.standard_normal(p.m)
    for tr, tc, k0 in [(16, 9, 0), (7, 25, 12345)]:
        ro, co = contiguous_offsets(p.m, tr), contiguous_offsets(p.n, tc)
        alpha = 1.3 / max(O.beta_max(A, ro, co))
        sp = O.rebk_sparse(p.m, p.n, indptr, indices, data, b, ro, co, alpha, seed=9, iters=150, k0=k0,
                           record=True)
        de = O.rebk(A, b, ro, co, alpha, seed=9, iters=150, k0=k0, record=True)
        assert np.array_equal(sp["idx"], de["idx"])
        assert np.linalg.norm(sp["x"] - de["x"]) <= 1e-12 * np.linalg.norm(de["x"])
        assert np.linalg.norm(sp["z"] - de["z"]) <= 1e-12 * np.linalg.norm(de["z"])
