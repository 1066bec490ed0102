"""Pins for the oracle's REBK iteration (Algorithm 1 of Du, Si, Sun,
arXiv:2001.04179) against what the paper and the mathematics fix:

* the limit A^+ b for the four kinds of system of Section 1;
* the subspace invariants x^k in range(A^T) (proof of Theorem main) and
  z^k - b in range(A) (proof of Lemma estz);
* the REK special case s = m, t = n, alpha = 1 (remark after Algorithm 1)
  against a separately written single row/column REK;
* the RABK special case z^0 = 0 (remark after Algorithm 1) against the
  weighted-average form of eq. (rabk);
* the exact mean recursions in the proof of Theorem ner;
* the bounds of Theorem ner, Lemma estz and Theorem main;
* the step sizes and iteration counts printed in Tables 1 and 2.
"""
import os

import numpy as np
import pytest

import oracle as O
from workloads import (contiguous_offsets, gaussian_problem, product_problem, small_cases,
                       type1_problem)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _alpha(A, ro, co, c=1.0):
    return c / max(O.beta_max(A, ro, co))


@pytest.mark.parametrize("case", small_cases(seed=0), ids=lambda c: c.name)
@pytest.mark.parametrize("tau", [(1, 1), (3, 4), (7, 5)])
def test_limit_is_pseudoinverse_solution(case, tau):
    ro = contiguous_offsets(case.m, tau[0])
    co = contiguous_offsets(case.n, tau[1])
    alpha = _alpha(case.A, ro, co)
    r = O.rebk(case.A, case.b, ro, co, alpha, seed=11, iters=400000, check_every=1,
               x_ref=case.x_ref, tol=1e-11)
    assert r["iters"] < 400000
    xs = O.pinv_solve(case.A, case.b)
    assert np.linalg.norm(r["x"] - xs) <= 1e-10 * np.linalg.norm(xs)
    # z converges to b_perp = (I - A A^+) b
    bperp = case.b - case.A @ xs
    assert np.linalg.norm(r["z"] - bperp) <= 1e-7 * max(np.linalg.norm(case.b), 1.0)


def test_subspace_invariants():
    """x^k - A^+ b in range(A^T) (so x^k in range(A^T) from x^0 = 0) and
    z^k - b in range(A), checked with SVD projectors on a rank-deficient,
    inconsistent system after a few iterations."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 6)) @ rng.standard_normal((6, 22))
    b = rng.standard_normal(30)
    U, s, Vt = np.linalg.svd(A)
    r = int(np.sum(s > 1e-10 * s[0]))
    PU = U[:, :r] @ U[:, :r].T
    PV = Vt[:r].T @ Vt[:r]
    ro, co = contiguous_offsets(30, 4), contiguous_offsets(22, 3)
    alpha = _alpha(A, ro, co, 1.5)
    for iters in [1, 7, 60]:
        out = O.rebk(A, b, ro, co, alpha, seed=3, iters=iters)
        x, z = out["x"], out["z"]
        assert np.linalg.norm(x - PV @ x) <= 1e-12 * max(np.linalg.norm(x), 1)
        assert np.linalg.norm((z - b) - PU @ (z - b)) <= 1e-12 * np.linalg.norm(b)
        # the iterates did move
        assert np.linalg.norm(x) > 0


def _rek_reference(A, b, seed, stream, iters):
    """REK of Zouzias and Freris as the paper's introduction states it: one
    column j (probability ||A_{:,j}||^2/||A||_F^2) projects z, then one row i
    (probability ||A_{i,:}||^2/||A||_F^2) projects x with b_i - z_i.  Draws
    come from numpy's Philox with the same key/counter layout."""
    m, n = A.shape
    rn = np.array([sum(A[i, c] * A[i, c] for c in range(n)) for i in range(m)])
    cn = np.array([sum(A[r, j] * A[r, j] for r in range(m)) for j in range(n)])
    crow, ccol = np.cumsum(rn), np.cumsum(cn)

    def u(d):
        c = (d - 1) % (1 << 256)
        words = np.array([(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
        w0 = int(np.random.Philox(key=np.array([seed, stream], dtype=np.uint64),
                                  counter=words).random_raw(1)[0])
        return (w0 >> 11) * 2.0 ** -53

    z = b.astype(np.float64).copy()
    x = np.zeros(n)
    picks = []
    for k in range(1, iters + 1):
        j = int(np.searchsorted(ccol, u(2 * (k - 1)) * ccol[-1], side="right"))
        z = z - (A[:, j] @ z) / cn[j] * A[:, j]
        i = int(np.searchsorted(crow, u(2 * (k - 1) + 1) * crow[-1], side="right"))
        x = x - (A[i] @ x - b[i] + z[i]) / rn[i] * A[i]
        picks.append((j, i))
    return x, z, np.array(picks)


def test_reduces_to_rek_at_block_size_one():
    p = gaussian_problem(25, 12, seed=4)
    ro, co = contiguous_offsets(25, 1), contiguous_offsets(12, 1)
    out = O.rebk(p.A, p.b, ro, co, 1.0, seed=21, stream=2, iters=300, record=True)
    x, z, picks = _rek_reference(p.A, p.b, 21, 2, 300)
    assert np.array_equal(out["idx"], picks)
    assert np.linalg.norm(out["x"] - x) <= 1e-12 * np.linalg.norm(x)
    assert np.linalg.norm(out["z"] - z) <= 1e-12 * np.linalg.norm(z)


def test_reduces_to_rabk_when_z0_is_zero():
    """With z^0 = 0 all z^k = 0 and the x step is RABK, eq. (rabk), with
    weights omega_l = ||A_{l,:}||^2 / ||A_{I,:}||_F^2, written as the average
    of single-row projections."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((24, 10))
    b = A @ rng.standard_normal(10)
    ro, co = contiguous_offsets(24, 5), contiguous_offsets(10, 3)
    alpha = 1.3
    out = O.rebk(A, b, ro, co, alpha, seed=5, iters=40, z0=np.zeros(24), record=True)
    assert np.all(out["z"] == 0.0)
    x = np.zeros(10)
    for k in range(40):
        i = out["idx"][k, 1]
        rows = range(ro[i], ro[i + 1])
        blk = sum(A[l] @ A[l] for l in rows)
        step = np.zeros(10)
        for l in rows:
            w = (A[l] @ A[l]) / blk
            step += w * (A[l] @ x - b[l]) / (A[l] @ A[l]) * A[l]
        x = x - alpha * step
    assert np.linalg.norm(out["x"] - x) <= 1e-12 * np.linalg.norm(x)


def test_mean_iterates_follow_closed_form():
    """E[z^k] and E[x^k] from the proof of Theorem ner (exact for any alpha)
    against the average of 20000 independent runs, within 5 standard errors."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((9, 6))
    A[:3] *= 2.0
    b = rng.standard_normal(9)
    ro, co = contiguous_offsets(9, 3), contiguous_offsets(6, 2)
    alpha, k, N = 1.7, 6, 20000
    xs = np.zeros((N, 6))
    zs = np.zeros((N, 9))
    for t in range(N):
        out = O.rebk(A, b, ro, co, alpha, seed=1000 + t, iters=k)
        xs[t], zs[t] = out["x"], out["z"]
    Ex, Ez = O.mean_closed_form(A, b, alpha, k)
    for samples, exact in [(xs, Ex), (zs, Ez)]:
        mean = samples.mean(axis=0)
        se = samples.std(axis=0, ddof=1) / np.sqrt(N)
        assert np.all(np.abs(mean - exact) <= 5 * se + 1e-12), (mean, exact, se)


def test_mean_closed_form_catches_a_wrong_step():
    """The same comparison fails for a run whose step size is off by 10%,
    so the pin above does resolve the update formula."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((9, 6))
    A[:3] *= 2.0
    b = rng.standard_normal(9)
    ro, co = contiguous_offsets(9, 3), contiguous_offsets(6, 2)
    k, N = 6, 20000
    xs = np.array([O.rebk(A, b, ro, co, 1.7 * 1.1, seed=1000 + t, iters=k)["x"] for t in range(N)])
    Ex, _ = O.mean_closed_form(A, b, 1.7, k)
    se = xs.std(axis=0, ddof=1) / np.sqrt(N)
    assert np.any(np.abs(xs.mean(axis=0) - Ex) > 5 * se)


def _mc_errors(A, b, ro, co, alpha, ks, N, z0=None):
    xsol = O.pinv_solve(A, b)
    bperp = b - A @ xsol
    ex = np.zeros((N, len(ks)))
    ez = np.zeros((N, len(ks)))
    mx = np.zeros((len(ks), A.shape[1]))
    for t in range(N):
        z, x, kprev = (b.copy() if z0 is None else z0.copy()), np.zeros(A.shape[1]), 0
        for c, k in enumerate(ks):
            out = O.rebk(A, b, ro, co, alpha, seed=77 + t, iters=k - kprev, k0=kprev, z0=z, x0=x)
            z, x, kprev = out["z"], out["x"], k
            ex[t, c] = np.sum((x - xsol) ** 2)
            ez[t, c] = np.sum((z - bperp) ** 2)
            mx[c] += (x - xsol) / N
    return ex, ez, mx


def test_expected_error_bounds():
    """Lemma estz, Theorem main (any eps > 0) and Theorem ner at
    alpha = 1/beta_max, where their hypotheses hold: seed averages stay
    below the bounds (plus 4 standard errors of the average)."""
    rng = np.random.default_rng(21)
    A = rng.standard_normal((40, 5)) @ rng.standard_normal((5, 16))
    b = rng.standard_normal(40)
    ro, co = contiguous_offsets(40, 5), contiguous_offsets(16, 4)
    alpha = _alpha(A, ro, co, 1.0)
    ks = [5, 20, 60]
    N = 1500
    ex, ez, mx = _mc_errors(A, b, ro, co, alpha, ks, N)
    for c, k in enumerate(ks):
        se_x = ex[:, c].std(ddof=1) / np.sqrt(N)
        se_z = ez[:, c].std(ddof=1) / np.sqrt(N)
        assert ez[:, c].mean() <= O.bound_estz(A, b, alpha, k, ro, co) + 4 * se_z
        for eps in [0.05, 0.5, 2.0]:
            assert ex[:, c].mean() <= O.bound_main(A, b, alpha, k, ro, co, eps=eps) + 4 * se_x
        assert np.linalg.norm(mx[c]) <= O.bound_ner(A, b, alpha, k) + 4 * np.sqrt(ex[:, c].mean() / N)
    # the error does decay
    assert ex[:, -1].mean() < 0.2 * ex[:, 0].mean()


def test_beta_max_range_of_remark_rek9():
    """max 1/|block| <= beta_max <= 1 (Remark rek9), with equality 1 at
    block size one (Remark rek8)."""
    p = gaussian_problem(50, 30, seed=6)
    for tr, tc in [(1, 1), (5, 3), (10, 7)]:
        ro, co = contiguous_offsets(50, tr), contiguous_offsets(30, tc)
        bI, bJ = O.beta_max(p.A, ro, co)
        assert 1.0 / tr - 1e-12 <= bI <= 1.0 + 1e-12
        assert 1.0 / tc - 1e-12 <= bJ <= 1.0 + 1e-12
        if tr == 1:
            assert bI == pytest.approx(1.0, rel=1e-12)


def _load_tables():
    rows = []
    with open(os.path.join(GOLDEN, "tables_1_2.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            t, typ, m, n, r, kap, c, a, it = line.split()
            rows.append(dict(table=t, type=typ, m=int(m), n=int(n), rank=int(r), kappa=float(kap),
                             c=float(c), alpha=float(a), iters=int(it)))
    return rows


@pytest.mark.parametrize("row", _load_tables(), ids=lambda r: f"{r['table']}_{r['m']}x{r['n']}_r{r['rank']}")
def test_tables_1_and_2(row):
    """Regenerated Type I / Type II systems (10 trials, tau = 10): beta_max
    implied by the printed alpha within 10%, and the average iteration count
    to ||x^k - A^+ b|| <= 1e-5 within 30% of the printed one.  The matrices are
    random, so only these loose statistical checks are meaningful."""
    m, n = row["m"], row["n"]
    ro, co = contiguous_offsets(m, 10), contiguous_offsets(n, 10)
    betas, iters = [], []
    for trial in range(10):
        if row["type"] == "I":
            p = type1_problem(m, n, row["rank"], row["kappa"], seed=100 + trial)
        else:
            p = gaussian_problem(m, n, seed=100 + trial)
        beta = max(O.beta_max(p.A, ro, co))
        betas.append(beta)
        alpha = row["c"] / beta
        xs = p.x_ref
        out = O.rebk(p.A, p.b, ro, co, alpha, seed=500 + trial, iters=200000, check_every=1,
                     x_ref=xs, tol=1e-5 / np.linalg.norm(xs))
        iters.append(out["iters"])
    beta_paper = row["c"] / row["alpha"]
    assert abs(np.mean(betas) - beta_paper) <= 0.10 * beta_paper
    assert abs(np.mean(iters) - row["iters"]) <= 0.30 * row["iters"]


def test_correction_form_is_rebk_from_shifted_state():
    """Algorithm 1 on corrections (refinement reading) with the full-precision
    matrix: x + dx and z + dz equal plain Algorithm 1 continued from (x, z) with
    the same draws, dz = -A s and dx = A^T v."""
    p = product_problem(40, 30, 8, seed=9)
    ro, co = contiguous_offsets(40, 6), contiguous_offsets(30, 4)
    alpha = _alpha(p.A, ro, co, 1.5)
    a = O.rebk(p.A, p.b, ro, co, alpha, seed=4, iters=17)
    x, z = a["x"], a["z"]
    cont = O.rebk(p.A, p.b, ro, co, alpha, seed=4, iters=25, k0=17, z0=z, x0=x, record=True)
    f, g = O.dual_residuals(p.A, p.b, z, x)
    nr, nc = O.block_norms(p.A, ro, co)
    c = O.rebk_correction(p.A, f, g, ro, co, (nr, nc), alpha, seed=4, iters=25, k0=17, record=True)
    assert np.array_equal(c["idx"], cont["idx"])
    scale = np.linalg.norm(p.b)
    assert np.linalg.norm(x + c["dx"] - cont["x"]) <= 1e-11 * np.linalg.norm(cont["x"])
    assert np.linalg.norm(z + c["dz"] - cont["z"]) <= 1e-11 * scale
    assert np.linalg.norm(c["dz"] + p.A @ c["s"]) <= 1e-11 * scale
    assert np.linalg.norm(c["dx"] - p.A.T @ c["v"]) <= 1e-11 * max(np.linalg.norm(c["dx"]), 1)


def test_exact_solution_is_a_fixed_point_of_refinement():
    p = product_problem(30, 24, 6, seed=10)
    ro, co = contiguous_offsets(30, 5), contiguous_offsets(24, 4)
    xs = O.pinv_solve(p.A, p.b)
    zs = p.b - p.A @ xs
    f, g = O.dual_residuals(p.A, p.b, zs, xs)
    assert np.linalg.norm(f) <= 1e-12 * np.linalg.norm(p.b)
    assert np.linalg.norm(g) <= 1e-11 * np.linalg.norm(p.b)
    nr, nc = O.block_norms(p.A, ro, co)
    c = O.rebk_correction(O.round_bf16(p.A), f * 0, g * 0, ro, co, (nr, nc), 1.0, seed=1, iters=50)
    for key in ("dz", "dx", "s", "v"):
        assert np.all(c[key] == 0.0)


@pytest.mark.parametrize("prec,red", [("fp32", 1e-4), ("bf16", 1e-2)])
def test_refinement_reaches_pseudoinverse(prec, red):
    """Reduced-precision corrections with FP64 refinement reach A^+ b to
    1e-8 on an inconsistent rank-deficient underdetermined system."""
    p = product_problem(200, 500, 50, seed=1)
    ro, co = contiguous_offsets(p.m, 16), contiguous_offsets(p.n, 16)
    alpha = _alpha(p.A, ro, co, 1.75)
    lo = O.round_fp32(p.A) if prec == "fp32" else O.round_bf16(p.A)
    xs = O.pinv_solve(p.A, p.b)
    assert np.linalg.norm(xs - p.x_ref) <= 1e-10 * np.linalg.norm(xs)
    r = O.refine(p.A, p.b, lo, ro, co, alpha, seed=7, inner_iters=50000, x_ref=xs, tol=1e-8,
                 inner_reduction=red, outer_max=12)
    assert np.linalg.norm(r["x"] - xs) <= 1e-8 * np.linalg.norm(xs)
    # without an error reference: fixed inner length, the error still falls to 1e-8
    r2 = O.refine(p.A, p.b, lo, ro, co, alpha, seed=7, inner_iters=400, outer_max=12)
    assert np.linalg.norm(r2["x"] - xs) <= 1e-8 * np.linalg.norm(xs)


def test_literal_refinement_stagnates_with_bf16():
    """x <- x + REBK(A_bf16, b - A x) keeps an error far above 1e-8 on a
    rank-deficient system: the reduced-precision copy has a different range
    and null space.  This is why the refinement works on (x, z) through the
    duals instead."""
    p = product_problem(200, 500, 50, seed=1)
    ro, co = contiguous_offsets(p.m, 16), contiguous_offsets(p.n, 16)
    alpha = _alpha(p.A, ro, co, 1.75)
    lo = O.round_bf16(p.A)
    xs = O.pinv_solve(p.A, p.b)
    x = np.zeros(p.n)
    errs = []
    for o in range(5):
        out = O.rebk(lo, p.b - p.A @ x, ro, co, alpha, seed=7 + o, iters=2000,
                     norms=O.block_norms(p.A, ro, co))
        x = x + out["x"]
        errs.append(np.linalg.norm(x - xs) / np.linalg.norm(xs))
    assert min(errs) > 1e-5


def test_round_bf16_is_round_to_nearest_even():
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 2**-9, 1.0 + 3 * 2**-9, -2.5, 1e-30, 3.0 + 2**-8])
    got = O.round_bf16(vals)
    # bf16 keeps 8 significant bits: 1 + 2^-8 is a tie -> even (1.0); 1 + 3*2^-9 -> 1 + 2^-7
    assert list(got) == [1.0, 1.0, 1.0, 1.0 + 2**-7, -2.5, got[5], 3.0]
    assert abs(got[5] - 1e-30) <= 2**-8 * 1e-30


# ---------------------------------------------------------------------------
# The bound functions against values the mathematics fixes (no Monte Carlo):
# a 3 x 2 diagonal system whose pseudoinverse solution, b_perp, singular
# values and block spectral norms are known by hand.
#   A = [[3, 0], [0, 1], [0, 0]], b = (1, 2, 5):  A^+ b = (1/3, 2),
#   b_perp = (0, 0, 5), sigma = {3, 1}, ||A||_F^2 = 10, A^T b = (3, 2).
#   Row blocks {0, 1}, {2}: beta^I = 9 / 10 (the zero block is skipped);
#   column blocks {0}, {1}: beta^J = 1.
# ---------------------------------------------------------------------------
_DA = np.array([[3.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
_DB = np.array([1.0, 2.0, 5.0])
_DRO = np.array([0, 2, 3])
_DCO = np.array([0, 1, 2])


def test_bounds_at_k0_equal_the_initial_errors():
    """At k = 0 every bound is the initial error itself: Theorem ner gives
    ||x^0 - A^+ b||, Lemma estz ||z^0 - b_perp||^2 and Theorem main
    ||x^0 - A^+ b||^2 (its tail sum is empty)."""
    x0 = np.array([0.5, -1.0])
    z0 = np.array([4.0, -3.0, 7.0])
    e_x2 = (0.5 - 1.0 / 3.0) ** 2 + (-1.0 - 2.0) ** 2
    e_z2 = 4.0 ** 2 + 3.0 ** 2 + (7.0 - 5.0) ** 2
    for alpha in (0.3, 1.0):
        assert O.bound_ner(_DA, _DB, alpha, 0, z0=z0, x0=x0) == pytest.approx(np.sqrt(e_x2), rel=1e-14)
        assert O.bound_estz(_DA, _DB, alpha, 0, _DRO, _DCO, z0=z0) == pytest.approx(e_z2, rel=1e-14)
        for eps in (0.1, 1.0, 3.0):
            assert O.bound_main(_DA, _DB, alpha, 0, _DRO, _DCO, eps=eps, z0=z0, x0=x0) == \
                pytest.approx(e_x2, rel=1e-14)


def test_bound_rates_on_a_hand_computed_system():
    """delta, eta and rho at alpha = 1 on the diagonal system:
    delta = max |1 - sigma_i^2 / 10| = 0.9, rho = 1 - (2 - 1) / 10 = 0.9,
    eta = 1 - (2 - 0.9) / 10 = 0.89; from x^0 = 0, z^0 = b:
    ||x^0 - A^+ b||^2 = 1/9 + 4, ||z^0 - b_perp||^2 = 5, ||A^T z^0|| = sqrt(13)."""
    assert O.beta_max(_DA, _DRO, _DCO) == pytest.approx((0.9, 1.0), rel=1e-14)
    ex2, ez2 = 1.0 / 9.0 + 4.0, 5.0
    for k in (1, 2, 7):
        ner = 0.9 ** k * (np.sqrt(ex2) + k * np.sqrt(13.0) / 10.0)
        assert O.bound_ner(_DA, _DB, 1.0, k) == pytest.approx(ner, rel=1e-13)
        assert O.bound_estz(_DA, _DB, 1.0, k, _DRO, _DCO) == pytest.approx(0.9 ** k * ez2, rel=1e-13)
    # a smaller step: alpha = 0.5 gives delta = max(|1 - 0.45|, |1 - 0.05|) = 0.95
    assert O.bound_ner(_DA, _DB, 0.5, 3) == pytest.approx(0.95 ** 3 * (np.sqrt(ex2) + 1.5 * np.sqrt(13.0) / 10.0),
                                                          rel=1e-13)


@pytest.mark.parametrize("k,eps", [(1, 0.5), (4, 0.5), (9, 0.05), (6, 2.0)])
def test_bound_main_tail_is_the_geometric_sum(k, eps):
    """Theorem main's second term carries sum_{l<k} rho^{k-l} q^l with
    q = (1 + eps) eta, a geometric sum equal to rho (rho^k - q^k) / (rho - q).
    With alpha = 1 on the diagonal system (eta = 0.89, rho = 0.9,
    beta^I = 0.9, ||z^0 - b_perp||^2 = 5, ||A||_F^2 = 10) the bound is
    q^k (1/9 + 4) + (1 + 1/eps) 0.9 * 5 / 10 * rho (rho^k - q^k) / (rho - q)."""
    rho, eta = 0.9, 0.89
    q = (1.0 + eps) * eta
    tail = rho * (rho ** k - q ** k) / (rho - q)
    want = q ** k * (1.0 / 9.0 + 4.0) + (1.0 + 1.0 / eps) * 0.9 * 5.0 / 10.0 * tail
    assert O.bound_main(_DA, _DB, 1.0, k, _DRO, _DCO, eps=eps) == pytest.approx(want, rel=1e-12)
