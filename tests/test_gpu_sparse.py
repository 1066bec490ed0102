"""Sparse REBK (rebk_sparse_*) against the FP64 oracle on the densified matrix.

Algorithm 1 does not depend on how A is stored: on the same matrix, seed and
step the sparse path draws the same blocks (bit-exact) and its iterates equal
the oracle's up to summation order (FP64 atomic adds), bar 1e-10 relative."""
import numpy as np
import pytest
from parity import assert_close, assert_converged  # noqa: E402

import oracle as O
from workloads import contiguous_offsets, sparse_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2001_04179_gb300 import Solver, SparseSolver  # noqa: E402
from paper_2001_04179_gb300 import rebk as R  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = [
    # m, n, nnz per row, tau_r, tau_c, num_ctas
    (600, 150, 12, 32, 16, 0),
    (333, 97, 9, 25, 10, 7),       # ragged last blocks, few CTAs
    (120, 300, 20, 8, 30, 0),      # underdetermined
    (64, 40, 5, 1, 1, 3),          # single rows / columns
    (500, 64, 64, 64, 8, 152),     # dense rows
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_indices_and_iterates_match_the_dense_oracle(case):
    m, n, k, tr, tc, G = case
    p = sparse_problem(m, n, k, seed=m + n, x_ref=None)
    A = p.dense()
    ro, co = contiguous_offsets(m, tr), contiguous_offsets(n, tc)
    alpha = 1.1 / max(O.beta_max(A, ro, co)) if (tr > 1 or tc > 1) else 1.0
    sol = SparseSolver(m, n, p.indptr, p.indices, p.data, tr, tc, alpha=alpha, num_ctas=G)
    iters = 143
    for seed, k0, sid in [(3, 0, 0), (77, 500, 4)]:
        out = sol.solve(_t(p.b), tol=0.0, max_iter=iters, seed=seed, k0=k0, stream_id=sid, record=True,
                        return_z=True)
        ref = O.rebk(A, p.b, ro, co, alpha, seed=seed, stream=sid, k0=k0, iters=iters, record=True)
        assert out["stats"]["iterations"] == iters
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
        assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
        assert_close(out["z"].cpu().numpy(), ref["z"], 1e-10)


def test_same_blocks_as_the_dense_solver_and_beta_max():
    p = sparse_problem(400, 100, 10, seed=9, x_ref=None)
    A = p.dense()
    sp = SparseSolver(400, 100, p.indptr, p.indices, p.data, 20, 10)
    de = Solver(A, 20, 10, alpha=sp.alpha, storage=())
    a = sp.solve(_t(p.b), max_iter=300, seed=5, record=True)["idx"].cpu().numpy()
    b = de.solve(_t(p.b), max_iter=300, seed=5, record=True)["idx"].cpu().numpy()
    assert np.array_equal(a, b)
    beta = max(O.beta_max(A, contiguous_offsets(400, 20), contiguous_offsets(100, 10)))
    assert sp.info()["beta_max"] == pytest.approx(beta, rel=1e-6)
    assert sp.alpha == pytest.approx(1.75 / beta, rel=1e-6)


@pytest.mark.parametrize("shape", [(800, 200, 12), (150, 400, 30)])
def test_solves_reach_the_pseudoinverse_solution(shape):
    m, n, k = shape
    p = sparse_problem(m, n, k, seed=1, x_ref="lstsq")
    sol = SparseSolver(m, n, p.indptr, p.indices, p.data, 16, 16)
    out = sol.solve(_t(p.b), tol=1e-10, max_iter=2_000_000, seed=2, x_ref=_t(p.x_ref))
    assert out["status"] == R.REBK_OK
    assert_converged(out["x"].cpu().numpy(), p.x_ref, 1e-10)


def test_zero_matrix_gives_zero():
    rp = np.zeros(11, dtype=np.int64)
    sol = SparseSolver(10, 5, rp, np.zeros(0, dtype=np.int32), np.zeros(0), 2, 2, alpha=1.0)
    out = sol.solve(_t(np.ones(10)), tol=1e-8, max_iter=100, seed=1)
    assert np.all(out["x"].cpu().numpy() == 0.0)


def test_empty_rows_and_columns():
    """Rows and columns without entries: their blocks have zero norm, are never
    sampled, and the iterates still match the oracle; the limit is A^+ b."""
    rng = np.random.default_rng(21)
    m, n = 90, 40
    A = np.zeros((m, n))
    for i in range(m):
        if i % 7 == 3:
            continue  # empty row
        cols = rng.choice([c for c in range(n) if c % 9 != 4], 5, replace=False)  # columns 4, 13, ... stay empty
        A[i, np.sort(cols)] = rng.uniform(0.5, 2.0, 5)
    A[:14, :] = 0.0  # a whole empty row block (tau 7: blocks 0 and 1)
    b = rng.standard_normal(m)
    indptr = np.concatenate([[0], np.cumsum((A != 0).sum(1))]).astype(np.int64)
    indices = np.concatenate([np.nonzero(A[i])[0] for i in range(m)]).astype(np.int32)
    data = A[A != 0]
    ro, co = contiguous_offsets(m, 7), contiguous_offsets(n, 5)
    alpha = 1.0 / max(O.beta_max(A, ro, co))
    sol = SparseSolver(m, n, indptr, indices, data, 7, 5, alpha=alpha)
    out = sol.solve(_t(b), tol=0.0, max_iter=200, seed=4, record=True, return_z=True)
    ref = O.rebk(A, b, ro, co, alpha, seed=4, iters=200, record=True)
    idx = out["idx"].cpu().numpy()
    assert np.array_equal(idx, ref["idx"])
    assert not np.any(np.isin(idx[:, 1], [0, 1]))  # zero-norm row blocks never drawn
    assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
    x_ls = O.pinv_solve(A, b)
    full = sol.solve(_t(b), tol=1e-10, max_iter=3_000_000, seed=5, x_ref=_t(x_ls))
    assert full["status"] == R.REBK_OK
    assert_converged(full["x"].cpu().numpy(), x_ls, 1e-10)


PASS_CASES = [
    # m, n, nnz per row, tau_r, tau_c, num_ctas
    (600, 150, 12, 32, 16, 0),
    (333, 97, 9, 25, 10, 7),       # ragged last blocks, few CTAs
    (120, 300, 20, 8, 30, 0),      # underdetermined
]


@pytest.mark.parametrize("case", PASS_CASES, ids=lambda c: "x".join(map(str, c)))
def test_one_mixed_precision_pass_matches_the_oracle_pass(case):
    """One refinement pass of the sparse mixed-precision solve (FP64 residuals
    over CSR / CSC, K inner iterations of the correction form with the FP32
    values, FP64 update) against the oracle's pass on the same rounded values
    (dense form): identical blocks; iterates within the FP32 arithmetic of the
    inner sweeps (the dense path's bar)."""
    m, n, k, tr, tc, G = case
    p = sparse_problem(m, n, k, seed=m + 2 * n, x_ref=None)
    A = p.dense()
    ro, co = contiguous_offsets(m, tr), contiguous_offsets(n, tc)
    alpha = 1.5 / max(O.beta_max(A, ro, co))
    sol = SparseSolver(m, n, p.indptr, p.indices, p.data, tr, tc, alpha=alpha, num_ctas=G)
    K = 200
    out = sol.solve_refined(_t(p.b), tol=0.0, max_iter=K, seed=21, max_outer=1, inner_iters=K, record=True,
                            return_z=True)
    assert out["stats"]["iterations"] == K and out["stats"]["outer"] == 1
    ref = O.refine(A, p.b, O.round_fp32(A), ro, co, alpha, seed=21, inner_iters=K, outer_max=1)
    idx_ref = O.rebk_correction(O.round_fp32(A), *O.dual_residuals(A, p.b, p.b, np.zeros(n)), ro, co,
                                O.block_norms(A, ro, co), alpha, seed=21, iters=K, record=True)["idx"]
    assert np.array_equal(out["idx"].cpu().numpy(), idx_ref)
    assert_close(out["x"].cpu().numpy(), ref["x"], 1e-4)
    assert np.linalg.norm(out["z"].cpu().numpy() - ref["z"]) <= 1e-4 * np.linalg.norm(p.b)


@pytest.mark.parametrize("shape", [(800, 200, 12), (150, 400, 30)])
def test_mixed_precision_reaches_the_pseudoinverse_solution(shape):
    m, n, k = shape
    p = sparse_problem(m, n, k, seed=3, x_ref="lstsq")
    sol = SparseSolver(m, n, p.indptr, p.indices, p.data, 16, 16)
    xr = _t(p.x_ref)
    out = sol.solve_refined(_t(p.b), tol=1e-10, seed=2, x_ref=xr)
    assert out["status"] == R.REBK_OK
    assert_converged(out["x"].cpu().numpy(), p.x_ref, 1e-10)
    assert out["stats"]["outer"] >= 2  # FP32 alone stops near 1e-6: the refinement did the rest
    plain = sol.solve(_t(p.b), tol=1e-10, max_iter=2_000_000, seed=2, x_ref=xr)
    assert out["stats"]["iterations"] <= 2 * plain["stats"]["iterations"] + 8192
    # without a reference solution: the residual stop rule
    out2 = sol.solve_refined(_t(p.b), tol=1e-11, seed=4)
    assert out2["status"] == R.REBK_OK
    assert_converged(out2["x"].cpu().numpy(), p.x_ref, 1e-6)


def test_mixed_precision_options_and_degenerate_cases():
    p = sparse_problem(200, 50, 6, seed=5, x_ref=None)
    sol = SparseSolver(200, 50, p.indptr, p.indices, p.data, 10, 10)
    b = _t(p.b)
    lib = R.load()
    x = torch.empty(50, dtype=torch.float64, device=DEV)
    for storage, want in [(R.REBK_BF16, R.REBK_EUNSUPPORTED), (R.REBK_FP64, R.REBK_EINVAL)]:
        ro = R.RebkRefineOpts(storage, 0, 0, 0.0)
        st = lib.rebk_sparse_solve_refined(sol._h, b.data_ptr(), x.data_ptr(), 1e-8, 100, 0, ro, None, None)
        assert st == want
    # max_iter = 0 leaves x = x0 = 0
    out = sol.solve_refined(b, tol=1e-8, max_iter=0, seed=1)
    assert out["stats"]["iterations"] == 0 and torch.all(out["x"] == 0)
    # A = 0: x = 0 = A^+ b
    rp = np.zeros(11, dtype=np.int64)
    zero = SparseSolver(10, 5, rp, np.zeros(0, dtype=np.int32), np.zeros(0), 2, 2, alpha=1.0)
    out = zero.solve_refined(_t(np.ones(10)), tol=1e-8, seed=1)
    assert out["status"] == R.REBK_OK and torch.all(out["x"] == 0)
