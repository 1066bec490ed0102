"""Special cases of Algorithm 1 named in the remark that follows it, on the GPU
path against the oracle:

* REK (Zouzias and Freris): single rows and columns, alpha = 1 (Solver.rek);
* RABK (Necoara): z^0 = 0, so every z^k = 0 and the x step is eq. (rabk)
  (Solver.solve_rabk); on a consistent system it reaches A^+ b.

Bars as in the parity tests: block indices bit-exact, FP64 iterates 1e-10."""
import numpy as np
import pytest
from parity import assert_close, assert_converged  # noqa: E402

import oracle as O
from workloads import contiguous_offsets, gaussian_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2001_04179_gb300 import Solver  # noqa: E402
from paper_2001_04179_gb300 import rebk as R  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def test_rek_special_case_matches_oracle_and_converges():
    p = gaussian_problem(120, 30, seed=12)
    sol = Solver.rek(p.A)
    assert sol.alpha == 1.0 and sol.blocks() == (120, 30)
    out = sol.solve(_t(p.b), tol=0.0, max_iter=500, seed=9, record=True, return_z=True)
    ref = O.rebk(p.A, p.b, contiguous_offsets(120, 1), contiguous_offsets(30, 1), 1.0, seed=9, iters=500,
                 record=True)
    assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
    assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
    assert_close(out["z"].cpu().numpy(), ref["z"], 1e-10)
    full = sol.solve(_t(p.b), tol=1e-10, max_iter=10**7, seed=3, x_ref=_t(p.x_ref))
    assert full["status"] == R.REBK_OK
    assert_converged(full["x"].cpu().numpy(), p.x_ref, 1e-10)


@pytest.mark.parametrize("shape", [(200, 60, 8, 6), (50, 140, 5, 12)])
def test_rabk_special_case_matches_oracle_and_reaches_min_norm_solution(shape):
    m, n, tr, tc = shape
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    b = A @ rng.standard_normal(n)  # consistent: RABK's setting
    ro, co = contiguous_offsets(m, tr), contiguous_offsets(n, tc)
    alpha = 1.4 / max(O.beta_max(A, ro, co))
    sol = Solver(A, tr, tc, alpha=alpha, storage=())
    out = sol.solve_rabk(_t(b), tol=0.0, max_iter=300, seed=2, record=True, return_z=True)
    ref = O.rebk(A, b, ro, co, alpha, seed=2, iters=300, z0=np.zeros(m), record=True)
    assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
    assert torch.all(out["z"] == 0)
    assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
    x_ls = O.pinv_solve(A, b)
    full = sol.solve_rabk(_t(b), tol=1e-10, max_iter=10**7, seed=4, x_ref=_t(x_ls))
    assert full["status"] == R.REBK_OK
    assert_converged(full["x"].cpu().numpy(), x_ls, 1e-10)


def _sv2(A):
    s = np.linalg.svd(A, compute_uv=False)
    s = s[s > s[0] * 1e-12]
    return s[0] ** 2, s[-1] ** 2


@pytest.mark.parametrize("kind", ["full_rank", "rank_deficient"])
def test_spectral_estimates_exact_at_the_rank(kind):
    """Golub-Kahan-Lanczos with full reorthogonalisation: after rank(A) steps the
    Krylov space is range(A^T) and the extreme Ritz values are sigma_1^2 and
    sigma_r^2 (against numpy's SVD); the rank-deficient case stops there by
    itself.  The quantities of Remark alpha and Theorems ner / main follow the
    oracle's definitions at the same alpha."""
    if kind == "full_rank":
        p = gaussian_problem(300, 80, seed=6)
        A, r = p.A, 80
    else:
        rng = np.random.default_rng(7)
        A, r = rng.standard_normal((200, 40)) @ rng.standard_normal((40, 150)), 40
    ro, co = contiguous_offsets(A.shape[0], 10), contiguous_offsets(A.shape[1], 10)
    sol = Solver(A, 10, 10, alpha=1.2 / max(O.beta_max(A, ro, co)), storage=())
    sp = sol.spectrum(steps=r + 20, seed=3)
    s1, sr = _sv2(A)
    assert r <= sp["steps"] <= r + 1  # a rank-deficient A may add one null-space direction
    assert sp["sigma1_sq"] == pytest.approx(s1, rel=1e-9)
    assert sp["sigma_r_sq"] == pytest.approx(sr, rel=1e-8)
    F = float(np.sum(A * A))
    assert sp["fro2"] == pytest.approx(F, rel=1e-13)
    assert sp["alpha_mean_opt"] == pytest.approx(2 * F / (s1 + sr), rel=1e-8)
    assert sp["delta_opt"] == pytest.approx((s1 - sr) / (s1 + sr), rel=1e-8)
    a = sol.alpha
    bI, bJ = O.beta_max(A, ro, co)
    assert sp["beta_row"] == pytest.approx(bI, rel=1e-6) and sp["beta_col"] == pytest.approx(bJ, rel=1e-6)
    # Theorem main's eta and Lemma estz's rho, Theorem ner's delta at the handle's alpha
    assert sp["eta"] == pytest.approx(1 - (2 * a - a * a * bI) * sr / F, rel=1e-7)
    assert sp["rho"] == pytest.approx(1 - (2 * a - a * a * bJ) * sr / F, rel=1e-7)
    assert sp["delta"] == pytest.approx(max(abs(1 - a * s1 / F), abs(1 - a * sr / F)), rel=1e-8)


def test_spectral_estimates_bracket_from_inside_with_few_steps():
    p = gaussian_problem(1500, 400, seed=8)
    sol = Solver(p.A, 20, 20, alpha=0.0, storage=())
    s1, sr = _sv2(p.A)
    sp = sol.spectrum(steps=30, seed=1)
    assert sp["steps"] == 30
    assert sr * (1 - 1e-12) <= sp["sigma_r_sq"] and sp["sigma1_sq"] <= s1 * (1 + 1e-12)
    assert sp["sigma1_sq"] >= 0.95 * s1  # the top converges first
    # Remark alpha's step, set on the handle
    a = sol.use_mean_optimal_alpha(steps=400)
    assert a == pytest.approx(2 * np.sum(p.A ** 2) / (s1 + sr), rel=1e-7)
    assert sol.alpha == a


def test_spectral_estimates_of_a_zero_matrix_are_zero():
    sol = Solver(np.zeros((6, 4)), 2, 2, alpha=1.0, storage=())
    sp = sol.spectrum(steps=5)
    assert sp["sigma1_sq"] == 0.0 and sp["steps"] == 0
