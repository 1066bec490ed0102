"""Algorithm 1 with arbitrary partitions (Section 2: any row blocks I_1..I_s
partitioning [m] and column blocks J_1..J_t partitioning [n]) through the C
ABI's rebk_partition, against the oracle run on the same offsets.

Partitions here are ragged on purpose: blocks of a single row or column, one
block much larger than the others, starts off every 16-byte boundary (the
unaligned tile paths) and a partition whose starts are all multiples of 8 but
whose sizes differ (the aligned tile paths).  Bars as in test_gpu_parity:
tables 1e-13, block indices bit-exact, plain FP64 iterates 1e-10 entry by
entry, one mixed-precision pass 1e-4."""
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


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def ragged(size, seed, big, small=(1, 2, 3), mid=(5, 40), align=1):
    """Offsets 0 < ... < size: one block of `big`, a few of the sizes in
    `small`, the rest uniform in `mid` (multiples of `align` when align > 1,
    except that the last block takes what is left)."""
    rng = np.random.default_rng(seed)
    sizes = [big] + list(small)
    while sum(sizes) < size:
        sizes.append(int(rng.integers(mid[0], mid[1] + 1)) // align * align or align)
    rng.shuffle(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)])
    off = off[off < size]
    return np.append(off, size).astype(np.int64)


CASES = [
    # name, m, n, row offsets, column offsets, CTAs
    ("ragged", 700, 333, ragged(700, 1, 300), ragged(333, 2, 200), 0),
    ("ragged_tma", 640, 500, ragged(640, 3, 150), ragged(500, 4, 120, small=(1, 7)), 0),
    ("aligned_starts", 512, 480, ragged(512, 5, 96, small=(8, 16), align=8),
     ragged(480, 6, 64, small=(8,), mid=(8, 48), align=8), 0),
    ("few_ctas", 90, 70, np.array([0, 1, 2, 50, 51, 90]), np.array([0, 1, 40, 41, 69, 70]), 3),
]


def _check_partition(ro, co, m, n):
    assert ro[0] == 0 and ro[-1] == m and np.all(np.diff(ro) > 0)
    assert co[0] == 0 and co[-1] == n and np.all(np.diff(co) > 0)


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_partitioned_tables_indices_and_fp64_iterates(case):
    name, m, n, ro, co, G = case
    _check_partition(ro, co, m, n)
    p = gaussian_problem(m, n, seed=m + n)
    alpha = 1.5 / max(O.beta_max(p.A, ro, co))
    sol = Solver(p.A, alpha=alpha, storage=(), num_ctas=G, row_off=ro, col_off=co)
    gro, gco = sol.partition()
    assert np.array_equal(gro, ro) and np.array_equal(gco, co)
    assert (sol.tau_row, sol.tau_col) == (int(np.max(np.diff(ro))), int(np.max(np.diff(co))))
    nr, nc, cr, cc = sol.tables()
    onr, onc, ocr, occ = O.tables(p.A, ro, co)
    for a, b in ((nr, onr), (nc, onc), (cr, ocr), (cc, occ)):
        assert np.max(np.abs(a - b) / np.abs(b)) <= 1e-13
    for K in (1, 37, 400):
        out = sol.solve(_t(p.b), tol=0.0, max_iter=K, seed=31, record=True, return_z=True)
        ref = O.rebk(p.A, p.b, ro, co, alpha, seed=31, iters=K, record=True)
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
        assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
        assert_close(out["z"].cpu().numpy(), ref["z"], 1e-10)


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: c[0])
def test_partitioned_beta_max_and_limit(case):
    name, m, n, ro, co, G = case
    p = gaussian_problem(m, n, seed=m + 2 * n)
    sol = Solver(p.A, alpha=0.0, storage=(), num_ctas=G, row_off=ro, col_off=co)
    bi, bj = sol.beta_max()
    obi, obj = O.beta_max(p.A, ro, co)
    assert bi == pytest.approx(obi, rel=1e-6) and bj == pytest.approx(obj, rel=1e-6)
    assert sol.alpha == pytest.approx(1.75 / max(obi, obj), rel=1e-6)
    out = sol.solve(_t(p.b), tol=1e-10, max_iter=2_000_000, seed=3, x_ref=_t(p.x_ref))
    assert out["status"] == R.REBK_OK
    assert_converged(out["x"].cpu().numpy(), p.x_ref, 1e-10)


@pytest.mark.parametrize("storage,lo", [("fp32", O.round_fp32), ("bf16", O.round_bf16)])
@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: c[0])
def test_partitioned_refinement_pass_matches_oracle_pass(storage, lo, case):
    name, m, n, ro, co, G = case
    p = product_problem(m, n, min(m, n) // 3, seed=8)
    alpha = 1.5 / max(O.beta_max(p.A, ro, co))
    sol = Solver(p.A, alpha=alpha, storage=(storage,), num_ctas=G, row_off=ro, col_off=co)
    K = 200
    out = sol.solve_refined(_t(p.b), tol=0.0, max_iter=K, seed=21, storage=storage, max_outer=1,
                            inner_iters=K, record=True, return_z=True)
    ref = O.refine(p.A, p.b, lo(p.A), ro, co, alpha, seed=21, inner_iters=K, outer_max=1)
    idx_ref = O.rebk_correction(lo(p.A), *O.dual_residuals(p.A, p.b, p.b, np.zeros(n)), ro, co,
                                O.block_norms(p.A, ro, co), alpha, seed=21, iters=K, record=True)["idx"]
    assert np.array_equal(out["idx"].cpu().numpy(), idx_ref)
    assert_close(out["x"].cpu().numpy(), ref["x"], 1e-4)
    assert np.linalg.norm(out["z"].cpu().numpy() - ref["z"]) <= 1e-4 * np.linalg.norm(p.b)
    full = sol.solve_refined(_t(p.b), tol=1e-8, seed=5, storage=storage, x_ref=_t(p.x_ref))
    assert full["status"] == R.REBK_OK
    assert_converged(full["x"].cpu().numpy(), p.x_ref, 1e-8)


def test_one_sided_partition_and_contiguous_equivalence():
    """Offsets on one side only (the other side contiguous blocks of tau), and
    offsets that spell out the contiguous partition give the contiguous
    solver's draws and iterates."""
    p = gaussian_problem(300, 120, seed=9)
    co = np.arange(0, 121, 10, dtype=np.int64)
    a = Solver(p.A, 16, 10, alpha=1.0, storage=())
    b = Solver(p.A, 16, 99, alpha=1.0, storage=(), col_off=co)
    ra = a.solve(_t(p.b), max_iter=300, seed=2, record=True)
    rb = b.solve(_t(p.b), max_iter=300, seed=2, record=True)
    assert np.array_equal(ra["idx"].cpu().numpy(), rb["idx"].cpu().numpy())
    assert_close(rb["x"].cpu().numpy(), ra["x"].cpu().numpy(), 1e-12)
    ro = np.array([0, 1, 2, 3, 200, 300], dtype=np.int64)
    c = Solver(p.A, 0, 12, alpha=1.0, storage=(), row_off=ro)
    rc = c.solve(_t(p.b), max_iter=300, seed=2, record=True, return_z=True)
    ref = O.rebk(p.A, p.b, ro, np.arange(0, 121, 12), 1.0, seed=2, iters=300, record=True)
    assert np.array_equal(rc["idx"].cpu().numpy(), ref["idx"])
    assert_close(rc["x"].cpu().numpy(), ref["x"], 1e-10)
    assert_close(rc["z"].cpu().numpy(), ref["z"], 1e-10)
