"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Bars (from the method's arithmetic):
* block indices: bit-exact (integer decisions taken from FP64 tables);
* block norm tables: relative 1e-13 (only summation order differs);
* plain FP64 iterates after the same iterations: relative 1e-10 (the device
  uses FMA and a different reduction order; the iteration is non-expansive,
  so rounding differences of ~1e-16 per step stay far below 1e-10);
* reduced-precision storage copies: bit-exact to the oracle's rounding;
* mixed precision: final ||x - A^+ b|| <= 1e-8 ||A^+ b||, and one refinement
  pass against the oracle's pass on the same rounded matrix within 1e-4
  relative (FP32 arithmetic in the inner sweeps: rounding of ~6e-8 per product,
  amplified by the non-normal pass over a few thousand iterations).
"""
import numpy as np
import pytest
from parity import assert_close, assert_converged  # noqa: E402

import oracle as O
from workloads import (contiguous_offsets, gaussian_problem, product_problem, small_cases,
                       type1_problem)

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
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SHAPES = [
    # m, n, tau_r, tau_c, num_ctas
    (1000, 200, 20, 20, 0),      # the 1000 x 200, tau = 20 workload
    (37, 23, 5, 4, 3),           # ragged last blocks, few CTAs
    (64, 64, 1, 1, 7),           # REK block size
    (50, 120, 7, 9, 16),         # underdetermined, ragged, odd tau
    (300, 41, 16, 8, 152),       # more CTAs than columns per CTA
    (5, 300, 2, 33, 2),
    (1, 17, 1, 4, 1),            # single row
    (19, 1, 3, 1, 4),            # single column
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_tables_indices_and_fp64_iterates_match_oracle(shape):
    m, n, tr, tc, G = shape
    p = gaussian_problem(m, n, seed=m * 7 + n)
    A = p.A.copy()
    if m >= 4:
        A[: m // 4] *= 3.0  # uneven block norms
    ro, co = contiguous_offsets(m, tr), contiguous_offsets(n, tc)
    alpha = 1.1 / max(O.beta_max(A, ro, co)) if (tr > 1 or tc > 1) else 1.0
    sol = Solver(A, tr, tc, alpha=alpha, storage=(), num_ctas=G)
    nr, nc, cr, cc = sol.tables()
    onr, onc = O.block_norms(A, ro, co)
    assert np.allclose(nr, onr, rtol=1e-13, atol=0) and np.allclose(nc, onc, rtol=1e-13, atol=0)
    assert np.allclose(cr, np.cumsum(onr), rtol=1e-13) and np.allclose(cc, np.cumsum(onc), rtol=1e-13)
    iters = 157
    for seed, k0, sid in [(3, 0, 0), (99, 1000, 5)]:
        out = sol.solve(_t(p.b), tol=0.0, max_iter=iters, seed=seed, k0=k0, stream_id=sid, record=True,
                        return_z=True)
        ref = O.rebk(A, p.b, ro, co, alpha, seed=seed, stream=sid, k0=k0, iters=iters, record=True)
        assert out["stats"]["iterations"] == iters
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
        assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
        assert_close(out["z"].cpu().numpy(), ref["z"], 1e-10)


@pytest.mark.parametrize("case", small_cases(seed=0), ids=lambda c: c.name)
def test_four_kinds_of_system_reach_pseudoinverse(case):
    ro, co = contiguous_offsets(case.m, 3), contiguous_offsets(case.n, 4)
    alpha = 1.0 / max(O.beta_max(case.A, ro, co))
    sol = Solver(case.A, 3, 4, alpha=alpha, storage=("fp32", "bf16"))
    xs = O.pinv_solve(case.A, case.b)
    out = sol.solve(_t(case.b), tol=1e-10, max_iter=500000, seed=11, x_ref=_t(xs))
    assert out["status"] == R.REBK_OK
    assert_converged(out["x"].cpu().numpy(), xs, 1e-10)
    # the residual stop rule (no reference solution) also gets there
    out2 = sol.solve(_t(case.b), tol=1e-11, max_iter=500000, seed=12)
    assert out2["status"] == R.REBK_OK
    assert_converged(out2["x"].cpu().numpy(), xs, 1e-8)
    for st in ("fp32", "bf16"):
        out3 = sol.solve_refined(_t(case.b), tol=1e-9, seed=13, storage=st, x_ref=_t(xs))
        assert out3["status"] == R.REBK_OK, out3["stats"]
        assert_converged(out3["x"].cpu().numpy(), xs, 1e-9)


def test_first_iteration_of_stop_rule_matches_oracle():
    """The 1000 x 200 randn workload, tau = 20, alpha = 2.25/beta_max, stop
    at ||x - A^+ b|| <= 1e-10 ||A^+ b|| checked every iteration: the same
    iteration count and iterate as the oracle."""
    p = gaussian_problem(1000, 200, seed=0)
    ro, co = contiguous_offsets(1000, 20), contiguous_offsets(200, 20)
    alpha = 2.25 / max(O.beta_max(p.A, ro, co))
    sol = Solver(p.A, 20, 20, alpha=alpha, storage=(), check_every=1)
    for seed in (1000, 1001, 1002):
        ref = O.rebk(p.A, p.b, ro, co, alpha, seed=seed, iters=100000, check_every=1, x_ref=p.x_ref,
                     tol=1e-10)
        out = sol.solve(_t(p.b), tol=1e-10, max_iter=100000, seed=seed, x_ref=_t(p.x_ref))
        assert out["stats"]["iterations"] == ref["iters"]
        assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
        assert out["stats"]["rel_err"] <= 1e-10


def test_storage_copies_round_like_the_oracle():
    p = product_problem(70, 45, 9, seed=3)
    sol = Solver(p.A, 8, 8, alpha=1.0, storage=("fp32", "bf16"))
    assert np.array_equal(sol.export_storage("fp64"), p.A)
    assert np.array_equal(sol.export_storage("fp32").astype(np.float64), O.round_fp32(p.A))
    bits = sol.export_storage("bf16").astype(np.uint32) << 16
    assert np.array_equal(bits.view(np.float32).astype(np.float64), O.round_bf16(p.A))


PASS_SHAPES = [
    # m, n, rank, tau_r, tau_c, num_ctas
    (120, 90, 30, 8, 8, 0),        # library's CTA choice, shared-memory tiles
    (600, 300, 80, 7, 13, 2),      # two TMA boxes per column tile, unaligned tile starts
    (333, 517, 60, 16, 5, 5),      # ragged blocks, odd column block
    (4000, 64, 20, 8, 32, 2),      # tiles too large for shared memory: global-load path
]


@pytest.mark.parametrize("storage,lo", [("fp32", O.round_fp32), ("bf16", O.round_bf16)])
@pytest.mark.parametrize("shape", PASS_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_one_refinement_pass_matches_oracle_pass(storage, lo, shape):
    """One outer pass (FP64 residuals, K inner iterations on corrections with
    the rounded matrix, FP64 update) against the oracle's pass on the same
    rounded values: the index sequence is identical and the iterate agrees to
    the FP32 arithmetic of the inner sweeps."""
    m, n, rank, tr, tc, G = shape
    p = product_problem(m, n, rank, seed=4)
    ro, co = contiguous_offsets(m, tr), contiguous_offsets(n, tc)
    alpha = 1.5 / max(O.beta_max(p.A, ro, co))
    sol = Solver(p.A, tr, tc, alpha=alpha, storage=(storage,), num_ctas=G)
    K = 200
    out = sol.solve_refined(_t(p.b), tol=0.0, max_iter=K, seed=21, storage=storage, max_outer=1,
                            inner_iters=K, record=True, return_z=True)
    ref = O.refine(p.A, p.b, lo(p.A), ro, co, alpha, seed=21, inner_iters=K, outer_max=1)
    assert out["stats"]["iterations"] == K
    idx_ref = O.rebk_correction(lo(p.A), *O.dual_residuals(p.A, p.b, p.b, np.zeros(n)), ro, co,
                                O.block_norms(p.A, ro, co), alpha, seed=21, iters=K, record=True)["idx"]
    assert np.array_equal(out["idx"].cpu().numpy(), idx_ref)
    # FP32 inner arithmetic: errors of order 1e-6 of the corrections' scale
    # (||x||, and ||b|| for z = b - A s, which cancels down to a small vector)
    assert_close(out["x"].cpu().numpy(), ref["x"], 1e-4)
    assert np.linalg.norm(out["z"].cpu().numpy() - ref["z"]) <= 1e-4 * np.linalg.norm(p.b)


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_mixed_precision_reaches_1e8_on_rank_deficient_system(storage):
    p = product_problem(600, 1500, 150, seed=1)
    ro, co = contiguous_offsets(600, 32), contiguous_offsets(1500, 32)
    alpha = 1.75 / max(O.beta_max(p.A, ro, co))
    sol = Solver(p.A, 32, 32, alpha=alpha, storage=(storage,))
    out = sol.solve_refined(_t(p.b), tol=1e-8, seed=5, storage=storage, x_ref=_t(p.x_ref))
    assert out["status"] == R.REBK_OK
    assert_converged(out["x"].cpu().numpy(), p.x_ref, 1e-8)
    # same inner iteration count as the plain FP64 run, within the pass granularity
    plain = sol.solve(_t(p.b), tol=1e-8, max_iter=10**6, seed=5, x_ref=_t(p.x_ref))
    assert out["stats"]["iterations"] <= 2 * plain["stats"]["iterations"] + 200
    # without a reference solution: residual stop rule
    out2 = sol.solve_refined(_t(p.b), tol=1e-10, seed=6, storage=storage)
    assert out2["status"] == R.REBK_OK
    assert_converged(out2["x"].cpu().numpy(), p.x_ref, 1e-7)


def test_beta_max_matches_oracle():
    p = type1_problem(300, 200, 120, 4.0, seed=2)
    for tr, tc in [(10, 10), (32, 17), (1, 5)]:
        ro, co = contiguous_offsets(300, tr), contiguous_offsets(200, tc)
        sol = Solver(p.A, tr, tc, alpha=1.0, storage=())
        bI, bJ = sol.beta_max()
        oI, oJ = O.beta_max(p.A, ro, co)
        assert bI == pytest.approx(oI, rel=1e-6)
        assert bJ == pytest.approx(oJ, rel=1e-6)
    sol = Solver(p.A, 10, 10, alpha=0.0, storage=())
    assert sol.alpha == pytest.approx(1.75 / max(O.beta_max(p.A, contiguous_offsets(300, 10),
                                                             contiguous_offsets(200, 10))), rel=1e-6)


def test_zero_matrix_and_zero_blocks():
    A = np.zeros((12, 9))
    sol = Solver(A, 3, 3, alpha=1.0, storage=("fp32",))
    b = np.arange(12, dtype=np.float64)
    out = sol.solve(_t(b), tol=1e-10, max_iter=100, seed=1)
    assert np.all(out["x"].cpu().numpy() == 0.0)
    out = sol.solve_refined(_t(b), tol=1e-10, seed=1)
    assert np.all(out["x"].cpu().numpy() == 0.0)
    # zero-norm blocks are never sampled
    rng = np.random.default_rng(3)
    A = rng.standard_normal((20, 12))
    A[4:8] = 0.0
    A[:, 6:9] = 0.0
    sol = Solver(A, 4, 3, alpha=1.0, storage=())
    out = sol.solve(_t(rng.standard_normal(20)), max_iter=400, seed=2, record=True)
    idx = out["idx"].cpu().numpy()
    assert not np.any(idx[:, 1] == 1) and not np.any(idx[:, 0] == 2)


def test_nonfinite_input_reports_divergence():
    p = gaussian_problem(40, 20, seed=1)
    sol = Solver(p.A, 5, 5, alpha=1.0, storage=())
    b = p.b.copy()
    b[3] = np.nan
    out = sol.solve(_t(b), tol=0.0, max_iter=50, seed=1, allow=(R.REBK_DIVERGED,))
    assert out["status"] == R.REBK_DIVERGED


def test_resume_continues_the_random_stream():
    """Two launches of 60 + 90 iterations (k0 = 60, state passed on) equal one
    launch of 150."""
    p = gaussian_problem(90, 40, seed=8)
    sol = Solver(p.A, 10, 8, alpha=2.0, storage=())
    full = sol.solve(_t(p.b), max_iter=150, seed=4, return_z=True)
    a = sol.solve(_t(p.b), max_iter=60, seed=4, return_z=True)
    b2 = sol.solve(_t(p.b), max_iter=90, seed=4, k0=60, x0=a["x"].clone(), z0=a["z"].clone(), return_z=True)
    assert_close(b2["x"].cpu().numpy(), full["x"].cpu().numpy(), 1e-13)
    assert_close(b2["z"].cpu().numpy(), full["z"].cpu().numpy(), 1e-13)


def test_bounded_waits_give_up_and_leave_the_context_usable():
    """Failure detection without a fault: device-wide waits for arrivals that never
    come end by their own limit with REBK_BARRIER_TIMEOUT, and the next solve runs."""
    import ctypes
    lib = R.load()
    codes = (ctypes.c_int32 * 2)()
    ms = ctypes.c_double()
    st = lib.rebk_selftest_waits(5_000_000, ctypes.cast(codes, ctypes.c_void_p), ctypes.byref(ms))
    assert st == R.REBK_BARRIER_TIMEOUT
    assert list(codes) == [R.REBK_BARRIER_TIMEOUT, R.REBK_BARRIER_TIMEOUT]
    assert 10.0 <= ms.value < 2000.0  # two waits of 5 ms each, then the kernel returned
    p = gaussian_problem(200, 60, seed=2)
    sol = Solver(p.A, 10, 10, alpha=0.0, storage=())
    out = sol.solve(_t(p.b), tol=1e-10, max_iter=10**6, seed=1, x_ref=_t(p.x_ref))
    assert out["status"] == R.REBK_OK
    assert_converged(out["x"].cpu().numpy(), p.x_ref, 1e-10)
