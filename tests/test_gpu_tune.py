"""Step-size replacement and the block-size autotuner, through the C ABI.

* rebk_set_alpha: the iterates after the change match the oracle run with the
  new alpha (relative 1e-10, the plain FP64 bar) and the block indices are
  bit-exact (sampling does not depend on alpha).
* rebk_tune_tau: every candidate reports the Section 2.2 beta_max of its
  partition (against the oracle's exact block spectral norms), alpha =
  c / beta_max, the iteration count a plain solve with that alpha and seed
  needs, and the pick is the candidate with the least measured time.
"""
import numpy as np
import pytest
from parity import assert_close  # noqa: E402

import oracle as O
from workloads import contiguous_offsets, gaussian_problem, product_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2001_04179_gb300 import Solver, tune_tau  # noqa: E402
from paper_2001_04179_gb300 import rebk as R  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("shape", [(300, 80, 12, 7), (45, 130, 4, 16)])
def test_set_alpha_iterates_match_oracle(shape):
    m, n, tr, tc = shape
    p = gaussian_problem(m, n, seed=m + n)
    ro, co = contiguous_offsets(m, tr), contiguous_offsets(n, tc)
    sol = Solver(p.A, tr, tc, alpha=0.0, storage=())
    a_new = 1.3 / max(O.beta_max(p.A, ro, co))
    sol.alpha = a_new
    assert sol.alpha == a_new
    out = sol.solve(_t(p.b), tol=0.0, max_iter=211, seed=5, record=True, return_z=True)
    ref = O.rebk(p.A, p.b, ro, co, a_new, seed=5, iters=211, record=True)
    assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
    assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
    assert_close(out["z"].cpu().numpy(), ref["z"], 1e-10)
    with pytest.raises(R.RebkError):
        sol.alpha = -1.0
    assert sol.alpha == a_new
    sol.close()


def test_tuner_reports_each_candidate_and_picks_the_fastest():
    p = gaussian_problem(400, 100, seed=21)
    A, b, xr = _t(p.A), _t(p.b), _t(p.x_ref)
    taus = [4, 10, 25, 100]
    best, pts = tune_tau(A, b, taus, x_ref=xr, alpha_factor=1.5, storage="fp64", tol=1e-8, seed=40, trials=2)
    assert [q["tau"] for q in pts] == taus
    for q in pts:
        ro, co = contiguous_offsets(400, q["tau"]), contiguous_offsets(100, q["tau"])
        assert q["beta_max"] == pytest.approx(max(O.beta_max(p.A, ro, co)), rel=1e-6)
        assert q["alpha"] == pytest.approx(1.5 / q["beta_max"], rel=1e-15)
        assert q["status"] == R.REBK_OK and q["device_ms"] > 0
        # the tuner's iteration count is the mean of plain solves with the same alpha and seeds
        sol = Solver(A, q["tau"], q["tau"], alpha=q["alpha"], storage=())
        its = [sol.solve(b, tol=1e-8, max_iter=10**7, seed=40 + r, x_ref=xr)["stats"]["iterations"]
               for r in range(2)]
        sol.close()
        assert abs(q["iterations"] - sum(its) // 2) <= 10
    assert best == min(pts, key=lambda q: q["device_ms"])["tau"]
    # beta_max falls as the blocks grow (Section 2.2): the iteration counts follow
    assert pts[0]["beta_max"] > pts[-1]["beta_max"]
    assert pts[0]["iterations"] > pts[-1]["iterations"]


def test_tuner_mixed_precision_and_residual_stop():
    p = product_problem(600, 300, 100, seed=3)
    A, b, xr = _t(p.A), _t(p.b), _t(p.x_ref)
    best, pts = tune_tau(A, b, [16, 64], x_ref=xr, storage="fp32", tol=1e-8, seed=2)
    assert best in (16, 64) and all(q["status"] == R.REBK_OK for q in pts)
    sol = Solver(A, best, best, alpha=0.0, storage=("fp32",))
    out = sol.solve_refined(b, tol=1e-8, seed=2, storage="fp32", x_ref=xr)
    assert out["stats"]["rel_err"] <= 1e-8
    sol.close()
    # without x_ref the stop rule is the residual test of rebk_solve
    best2, pts2 = tune_tau(p.A, b, [32], storage="fp64", tol=1e-9, seed=2)
    assert best2 == 32 and pts2[0]["status"] == R.REBK_OK


def test_tuner_reports_a_candidate_that_misses_the_tolerance():
    """With max_iter far too small no candidate converges: MAX_ITER, best 0,
    every point flagged with time -1."""
    p = gaussian_problem(200, 50, seed=8)
    best, pts = tune_tau(_t(p.A), _t(p.b), [5, 10], x_ref=_t(p.x_ref), tol=1e-12, max_iter=20)
    assert best == 0
    assert all(q["status"] == R.REBK_MAX_ITER and q["device_ms"] == -1.0 for q in pts)
