"""Several right-hand sides of one matrix at once (rebk_solve_multi): every
right-hand side runs the mixed-precision solve of rebk_solve_refined (Algorithm
1 of Section 2 on corrections with the FP32 or BF16 copy, FP64 refinement), and
the members of a group share one block sequence, so each member must match the
oracle's `refine` run on its own right-hand side with the group's seed and
stream.

Bars as for the one-right-hand-side mixed path: block indices bit-exact, one
pass of K iterations within 1e-4 entry by entry (FP32 inner arithmetic against
the oracle's FP64 arithmetic on the rounded matrix), full solves to 1e-8 against
A^+ b.  Shapes span many CTAs' slices with ragged tails (m, n not multiples of
the CTA count, blocks of tau with a short last block), groups of 4 and 8, a
right-hand-side count that leaves the last group partly empty, and a ragged
partition."""
import numpy as np
import pytest
from parity import assert_close, assert_converged  # noqa: E402

import oracle as O
from workloads import gaussian_problem, product_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2001_04179_gb300 import Solver  # noqa: E402
from paper_2001_04179_gb300 import rebk as R  # noqa: E402

DEV = torch.device("cuda:0")
LOWER = {"fp32": O.round_fp32, "bf16": O.round_bf16}


def _rhs(p, nrhs, seed):
    """nrhs right-hand sides A x* + noise around the problem's own b."""
    rng = np.random.default_rng(seed)
    B = [p.b]
    for _ in range(nrhs - 1):
        xs = rng.standard_normal(p.A.shape[1])
        B.append(p.A @ xs + 0.01 * rng.standard_normal(p.A.shape[0]))
    return np.array(B)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


CASES = [
    # name, problem, tau_row, tau_col, storage, group, nrhs
    ("gauss_fp32_g8", lambda: gaussian_problem(700, 333, seed=1), 24, 16, "fp32", 8, 8),
    ("gauss_fp32_g4_ragged_count", lambda: gaussian_problem(700, 333, seed=1), 24, 16, "fp32", 4, 6),
    ("product_bf16_g8", lambda: product_problem(640, 500, 160, seed=2), 32, 40, "bf16", 8, 5),
    ("product_fp32_g4", lambda: product_problem(480, 900, 200, seed=3), 40, 24, "fp32", 4, 4),
    # wide blocks: K runs of up to 256 on the tensor-core path, two register segments on the FMA path
    ("wide_blocks_fp32_g8", lambda: product_problem(900, 700, 300, seed=5), 256, 200, "fp32", 8, 8),
    ("wide_blocks_bf16_g4", lambda: gaussian_problem(900, 700, seed=6), 200, 256, "bf16", 4, 4),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_one_pass_matches_oracle_per_member(case):
    name, make, tr, tc, storage, group, nrhs = case
    p = make()
    alpha = 1.5 / max(O.beta_max(p.A, np.append(np.arange(0, p.A.shape[0], tr), p.A.shape[0]),
                                 np.append(np.arange(0, p.A.shape[1], tc), p.A.shape[1])))
    sol = Solver(p.A, tr, tc, alpha=alpha, storage=(storage,))
    ro, co = sol.partition()
    B = _rhs(p, nrhs, 7)
    K = 200
    out = sol.solve_multi(_dev(B), tol=0.0, max_iter=K, seed=13, storage=storage, group=group, max_outer=1,
                          inner_iters=K, record=True)
    assert out["stats"]["iterations"] == K * ((nrhs + group - 1) // group)
    lo = LOWER[storage](p.A)
    idx_ref = O.rebk_correction(lo, *O.dual_residuals(p.A, B[0], B[0], np.zeros(p.A.shape[1])), ro, co,
                                O.block_norms(p.A, ro, co), alpha, seed=13, iters=K, record=True)["idx"]
    assert np.array_equal(out["idx"][: 2 * K].view(-1, 2).cpu().numpy(), idx_ref)
    X = out["X"].cpu().numpy()
    for j in range(nrhs):
        ref = O.refine(p.A, B[j], lo, ro, co, alpha, seed=13, inner_iters=K, outer_max=1, stream=j // group)
        assert_close(X[j], ref["x"], 1e-4)


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_full_solves_reach_tolerance(storage):
    p = product_problem(800, 600, 150, seed=4)
    sol = Solver(p.A, 32, 32, alpha=0.0, storage=(storage,))
    B = _rhs(p, 11, 5)
    Xs = np.array([O.pinv_solve(p.A, b) for b in B])
    out = sol.solve_multi(_dev(B), tol=1e-8, seed=3, storage=storage, X_ref=_dev(Xs))
    assert out["status"] == R.REBK_OK
    assert np.all(out["rel"] <= 1e-8)
    X = out["X"].cpu().numpy()
    for j in range(len(B)):
        assert_converged(X[j], Xs[j], 1e-8)


def test_residual_rule_without_reference():
    """Without X_ref every member stops on the residual test of rebk_solve; the
    solutions are then close to A^+ b (the test bounds the residuals only)."""
    p = gaussian_problem(900, 300, seed=6)
    sol = Solver(p.A, 30, 20, alpha=0.0, storage=("fp32",))
    B = _rhs(p, 8, 9)
    out = sol.solve_multi(_dev(B), tol=1e-10, seed=1, storage="fp32", group=8)
    assert out["status"] == R.REBK_OK
    assert np.all(out["rel"] <= 1e-10)
    X = out["X"].cpu().numpy()
    for j in range(len(B)):
        xs = O.pinv_solve(p.A, B[j])
        assert np.linalg.norm(X[j] - xs) <= 1e-7 * np.linalg.norm(xs)


@pytest.mark.parametrize("group", [4, 8])
def test_ragged_partition_one_pass(group):
    """Blocks of 1 to 150 rows / columns, column starts off every 16-byte boundary;
    group 8 runs the tensor-core products, group 4 the FMA ones."""
    from test_gpu_partitions import ragged
    p = gaussian_problem(640, 500, seed=8)
    ro, co = ragged(640, 3, 150), ragged(500, 4, 120, small=(1, 7))
    alpha = 1.5 / max(O.beta_max(p.A, ro, co))
    sol = Solver(p.A, alpha=alpha, storage=("fp32",), row_off=ro, col_off=co)
    B = _rhs(p, group, 2)
    K = 150
    out = sol.solve_multi(_dev(B), tol=0.0, max_iter=K, seed=21, storage="fp32", group=group, max_outer=1,
                          inner_iters=K, record=True)
    lo = O.round_fp32(p.A)
    idx_ref = O.rebk_correction(lo, *O.dual_residuals(p.A, B[0], B[0], np.zeros(500)), ro, co,
                                O.block_norms(p.A, ro, co), alpha, seed=21, iters=K, record=True)["idx"]
    assert np.array_equal(out["idx"][: 2 * K].view(-1, 2).cpu().numpy(), idx_ref)
    X = out["X"].cpu().numpy()
    for j in range(group):
        ref = O.refine(p.A, B[j], lo, ro, co, alpha, seed=21, inner_iters=K, outer_max=1)
        assert_close(X[j], ref["x"], 1e-4)


def test_members_equal_the_one_rhs_solve():
    """A group member and rebk_solve_refined with the same seed and stream draw
    the same blocks and agree to FP32 rounding after one pass."""
    p = gaussian_problem(500, 260, seed=10)
    sol = Solver(p.A, 20, 20, alpha=0.0, storage=("fp32",))
    B = _rhs(p, 4, 3)
    K = 300
    out = sol.solve_multi(_dev(B), tol=0.0, max_iter=K, seed=5, storage="fp32", group=4, max_outer=1,
                          inner_iters=K, stream_id=2, record=True)
    for j in range(4):
        one = sol.solve_refined(_dev(B[j]), tol=0.0, max_iter=K, seed=5, storage="fp32", max_outer=1,
                                inner_iters=K, stream_id=2, record=True)
        assert np.array_equal(one["idx"].cpu().numpy(), out["idx"][: 2 * K].view(-1, 2).cpu().numpy())
        assert_close(out["X"][j].cpu().numpy(), one["x"].cpu().numpy(), 1e-4)


def test_degenerate_inputs():
    p = gaussian_problem(200, 90, seed=12)
    sol = Solver(p.A, 16, 16, alpha=0.0, storage=("fp32",))
    # no right-hand side
    out = sol.solve_multi(torch.zeros(0, 200, dtype=torch.float64, device=DEV), tol=1e-8)
    assert out["X"].shape == (0, 90)
    # a zero right-hand side: x = 0 at once
    B = _rhs(p, 3, 1)
    B[1] = 0.0
    out = sol.solve_multi(_dev(B), tol=1e-9, seed=2, group=4)
    assert out["status"] == R.REBK_OK
    assert np.all(out["X"][1].cpu().numpy() == 0.0)
    # invalid group
    with pytest.raises(R.RebkError):
        sol.solve_multi(_dev(B), group=6)
