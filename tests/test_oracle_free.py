"""Pins for the oracle's partition-free variant (``oracle.rebk_free``): index
sets of tau_c columns and tau_r rows drawn independently with probabilities
proportional to their squared norms, Algorithm 1's step on the drawn
submatrices (a reading of Section 4's variants whose samplings do not depend
on partitions).

* the draw counter layout against numpy's independent Philox4x64-10;
* at tau_r = tau_c = 1 it is the randomized extended Kaczmarz method (the
  separately written REK of test_oracle_rebk);
* the limit A^+ b for the four kinds of system of Section 1, and the subspace
  invariants of Theorem main's proof;
* the expected first step, enumerated exactly over every ordered draw of a
  tiny system, against the mean of many seeded runs (this resolves the
  sampling probabilities and the Frobenius-normalised step, duplicates
  included).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from test_oracle_rebk import _rek_reference
from workloads import small_cases


def _numpy_philox_word0(seed, stream, d, q):
    value = d + (q << 64)
    c = (value - 1) % (1 << 256)  # numpy increments the counter before encrypting
    words = np.array([(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    gen = np.random.Philox(key=np.array([seed, stream], dtype=np.uint64), counter=words)
    return int(gen.random_raw(1)[0])


def test_draw_slots_follow_the_philox_counter_layout():
    for seed, stream, d, q in [(0, 0, 0, 0), (7, 3, 11, 1), (2**40 + 5, 9, 2**33, 127), (1, 0, 5, 511)]:
        want = (_numpy_philox_word0(seed, stream, d, q) >> 11) * 2.0 ** -53
        assert O.uniform_slot(seed, stream, d, q) == want
    assert O.uniform_slot(5, 2, 9, 0) == O.uniform(5, 2, 9)


def test_reduces_to_rek_with_single_draws():
    from workloads import gaussian_problem
    p = gaussian_problem(25, 12, seed=4)
    out = O.rebk_free(p.A, p.b, 1, 1, 1.0, seed=21, stream=2, iters=300, record=True)
    x, z, picks = _rek_reference(p.A, p.b, 21, 2, 300)
    assert np.array_equal(out["idx"], picks)
    assert np.linalg.norm(out["x"] - x) <= 1e-12 * np.linalg.norm(x)
    assert np.linalg.norm(out["z"] - z) <= 1e-12 * np.linalg.norm(z)


@pytest.mark.parametrize("case", small_cases(seed=0), ids=lambda c: c.name)
def test_limit_is_pseudoinverse_solution(case):
    r = O.rebk_free(case.A, case.b, 3, 4, 1.0, seed=11, iters=400000, check_every=1, x_ref=case.x_ref,
                    tol=1e-11)
    assert r["iters"] < 400000
    xs = O.pinv_solve(case.A, case.b)
    assert np.linalg.norm(r["x"] - xs) <= 1e-10 * np.linalg.norm(xs)
    bperp = case.b - case.A @ xs
    assert np.linalg.norm(r["z"] - bperp) <= 1e-7 * max(np.linalg.norm(case.b), 1.0)


def test_subspace_invariants():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 6)) @ rng.standard_normal((6, 22))
    b = rng.standard_normal(30)
    U, s, Vt = np.linalg.svd(A)
    r = int(np.sum(s > 1e-10 * s[0]))
    PU = U[:, :r] @ U[:, :r].T
    PV = Vt[:r].T @ Vt[:r]
    for iters in [1, 7, 60]:
        out = O.rebk_free(A, b, 4, 3, 1.5, seed=3, iters=iters)
        x, z = out["x"], out["z"]
        assert np.linalg.norm(x - PV @ x) <= 1e-12 * max(np.linalg.norm(x), 1)
        assert np.linalg.norm((z - b) - PU @ (z - b)) <= 1e-12 * np.linalg.norm(b)
        assert np.linalg.norm(x) > 0


def _exact_first_step(A, b, tau_r, tau_c, alpha):
    """E[z^1], E[x^1] from z^0 = b, x^0 = 0 by enumerating every ordered draw:
    P(j_1..j_tau) = prod ||A_{:,j_q}||^2 / ||A||_F^2 (likewise rows)."""
    m, n = A.shape
    cn = (A * A).sum(0)
    rn = (A * A).sum(1)
    F = cn.sum()
    Ez, Ex = np.zeros(m), np.zeros(n)
    for J in itertools.product(range(n), repeat=tau_c):
        pJ = np.prod([cn[j] / F for j in J])
        AJ = A[:, list(J)]
        z = b - alpha / (AJ * AJ).sum() * AJ @ (AJ.T @ b)
        Ez += pJ * z
        for I in itertools.product(range(m), repeat=tau_r):
            pI = np.prod([rn[i] / F for i in I])
            AI = A[list(I), :]
            x = -alpha / (AI * AI).sum() * AI.T @ (-b[list(I)] + z[list(I)])
            Ex += pJ * pI * x
    return Ex, Ez


def test_expected_first_step_matches_exact_enumeration():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((4, 3))
    A[:, 0] *= 3.0   # a heavy column: repeated draws are common
    A[1] *= 0.3      # a light row
    b = rng.standard_normal(4)
    alpha, N = 1.3, 40000
    Ex, Ez = _exact_first_step(A, b, 2, 2, alpha)
    xs = np.zeros((N, 3))
    zs = np.zeros((N, 4))
    for t in range(N):
        out = O.rebk_free(A, b, 2, 2, alpha, seed=500 + t, iters=1)
        xs[t], zs[t] = out["x"], out["z"]
    for samples, exact in [(xs, Ex), (zs, Ez)]:
        se = samples.std(axis=0, ddof=1) / np.sqrt(N)
        assert np.all(np.abs(samples.mean(axis=0) - exact) <= 5 * se + 1e-12)
    # the comparison resolves the step: equal weights 1 / tau instead of the
    # Frobenius normalisation move the exact mean far outside the band
    cn = (A * A).sum(0)
    wrong = np.zeros(4)
    F = cn.sum()
    for J in itertools.product(range(3), repeat=2):
        pJ = np.prod([cn[j] / F for j in J])
        wrong += pJ * (b - alpha * sum(A[:, j] * (A[:, j] @ b) / cn[j] for j in J) / 2)
    se = zs.std(axis=0, ddof=1) / np.sqrt(N)
    assert np.any(np.abs(zs.mean(axis=0) - wrong) > 5 * se)
