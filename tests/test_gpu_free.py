"""The partition-free variant (rebk_solve_free: index sets drawn
independently per row and column, Algorithm 1's step on the drawn
submatrices) against the oracle's rebk_free on the same Philox stream.

Bars: every drawn index bit-exact; FP64 iterates after the same iterations
1e-10 entry by entry (FMA and tree-order sums on the device, as for the
partition solver); solves stopped at 1e-10 reach A^+ b."""
import numpy as np
import pytest
from parity import assert_close, assert_converged  # noqa: E402

import oracle as O
from workloads import gaussian_problem, product_problem, small_cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2001_04179_gb300 import Solver  # noqa: E402
from paper_2001_04179_gb300 import rebk as R  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


SHAPES = [
    # m, n, tau_r, tau_c, num_ctas
    (1000, 200, 20, 20, 0),
    (37, 23, 5, 4, 3),
    (64, 64, 1, 1, 7),        # REK
    (50, 120, 7, 9, 16),
    (300, 41, 64, 8, 0),      # more draws than columns: repeats certain
    (1, 17, 3, 4, 1),         # single row: every row draw repeats it
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_draws_and_fp64_iterates_match_oracle(shape):
    m, n, tr, tc, G = shape
    p = gaussian_problem(m, n, seed=m * 3 + n)
    sol = Solver(p.A, 4, 4, alpha=1.0, storage=(), num_ctas=G)
    for K in (1, 2, 9, 300):
        out = sol.solve_free(_t(p.b), tr, tc, alpha=1.3, max_iter=K, seed=17, record=True, return_z=True)
        ref = O.rebk_free(p.A, p.b, tr, tc, 1.3, seed=17, iters=K, record=True)
        assert out["stats"]["iterations"] == K
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
        assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
        assert_close(out["z"].cpu().numpy(), ref["z"], 1e-10)


def test_resume_and_stream_id():
    p = gaussian_problem(120, 60, seed=2)
    sol = Solver(p.A, 8, 8, alpha=1.0, storage=())
    a = sol.solve_free(_t(p.b), 6, 5, alpha=1.1, max_iter=50, seed=4, stream_id=3, return_z=True)
    b = sol.solve_free(_t(p.b), 6, 5, alpha=1.1, max_iter=30, seed=4, stream_id=3, k0=50, x0=a["x"],
                       z0=a["z"], record=True, return_z=True)
    full = O.rebk_free(p.A, p.b, 6, 5, 1.1, seed=4, stream=3, iters=80, record=True)
    assert np.array_equal(b["idx"].cpu().numpy(), full["idx"][50:])
    assert_close(b["x"].cpu().numpy(), full["x"], 1e-10)


@pytest.mark.parametrize("case", small_cases(seed=0), ids=lambda c: c.name)
def test_reaches_pseudoinverse_solution(case):
    sol = Solver(case.A, 2, 2, alpha=1.0, storage=())
    xs = O.pinv_solve(case.A, case.b)
    out = sol.solve_free(_t(case.b), 3, 4, alpha=1.0, tol=1e-10, max_iter=2_000_000, seed=11, x_ref=_t(xs))
    assert out["status"] == R.REBK_OK
    assert_converged(out["x"].cpu().numpy(), xs, 1e-10)


def test_rank_deficient_underdetermined_limit_and_stop_iteration():
    """On an inconsistent rank-deficient system the solve stops where the
    oracle's does (check every 10 iterations) and reaches A^+ b."""
    p = product_problem(200, 500, 50, seed=3)
    sol = Solver(p.A, 16, 16, alpha=1.0, storage=(), check_every=10)
    xs = p.x_ref
    out = sol.solve_free(_t(p.b), 16, 16, alpha=1.5, tol=1e-8, max_iter=10**6, seed=5, x_ref=_t(xs))
    ref = O.rebk_free(p.A, p.b, 16, 16, 1.5, seed=5, iters=10**6, check_every=10, x_ref=xs, tol=1e-8)
    assert out["status"] == R.REBK_OK
    assert out["stats"]["iterations"] == ref["iters"]
    assert_converged(out["x"].cpu().numpy(), xs, 1e-8)
