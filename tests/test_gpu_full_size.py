"""Full-size parity at the workloads' own sizes, in the launch configurations the
benchmark times.  First the 8000 x 20000 rank-2000 workload (A = G1 G2, b = A x* +
N(0, 0.01^2), seed 0): tau = 128
for rows and columns, the library's CTA count (one per SM), TMA-staged FP32 tiles
for the mixed path.

* block indices bit-exact and plain FP64 iterates within 1e-10 of the oracle
  after 60 iterations, and again 10^6 iterations into the random stream;
* one mixed-precision pass (FP64 residuals, 100 FP32 inner iterations on the
  FP32-rounded matrix, FP64 update) against the oracle's pass, bar 1e-4 as in the
  small-size tests;
* whole solves to 1e-8: the plain FP64 path stops at the iteration the oracle
  recorded for this workload (tests/golden/precision_anchor.txt, written by the
  oracle alone), the mixed path within 5% of it, both within 1e-8 of A^+ b.
The step size is the oracle's recorded alpha, passed to both sides.  Then the
512-system batch, the 65536 x 16384 sparse matrix and the 8192 -> 512 -> 512 ->
8192 warm-start network (see each test)."""
import os

import numpy as np
import pytest
from parity import assert_close, assert_converged  # noqa: E402

import oracle as O
from workloads import contiguous_offsets, product_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2001_04179_gb300 import Solver  # noqa: E402
from paper_2001_04179_gb300 import rebk as R  # noqa: E402

DEV = torch.device("cuda:0")
M, N, RANK, TAU = 8000, 20000, 2000, 128
HERE = os.path.dirname(os.path.abspath(__file__))


def _anchor():
    out = {}
    for line in open(os.path.join(HERE, "golden", "precision_anchor.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        out[k] = float(v)
    return out


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.fixture(scope="module")
def setup():
    def mm(a, b):  # input generation only: the product on the device, in FP64
        return (torch.from_numpy(np.ascontiguousarray(a)).to(DEV) @
                torch.from_numpy(np.ascontiguousarray(b)).to(DEV)).cpu().numpy()

    p = product_problem(M, N, RANK, seed=0, noise=0.01, matmul=mm)
    anchor = _anchor()
    alpha = anchor["alpha"]
    A_dev = torch.from_numpy(p.A).to(DEV)
    sol = Solver(A_dev, TAU, TAU, alpha=alpha, storage=("fp32",))
    yield p, anchor, alpha, sol
    sol.close()


def test_full_size_indices_and_fp64_iterates(setup):
    p, _, alpha, sol = setup
    ro, co = contiguous_offsets(M, TAU), contiguous_offsets(N, TAU)
    b = torch.from_numpy(p.b).to(DEV)
    for k0, iters in [(0, 60), (1_000_000, 20)]:
        out = sol.solve(b, tol=0.0, max_iter=iters, seed=7, k0=k0, record=True, return_z=True)
        ref = O.rebk(p.A, p.b, ro, co, alpha, seed=7, k0=k0, iters=iters, record=True)
        assert out["stats"]["iterations"] == iters
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
        assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
        assert_close(out["z"].cpu().numpy(), ref["z"], 1e-10)


def test_full_size_mixed_pass_matches_oracle_pass(setup):
    p, _, alpha, sol = setup
    ro, co = contiguous_offsets(M, TAU), contiguous_offsets(N, TAU)
    K = 100
    out = sol.solve_refined(torch.from_numpy(p.b).to(DEV), tol=0.0, max_iter=K, seed=21, storage="fp32",
                            max_outer=1, inner_iters=K, record=True, return_z=True)
    assert out["stats"]["iterations"] == K
    ref = O.refine(p.A, p.b, O.round_fp32(p.A), ro, co, alpha, seed=21, inner_iters=K, outer_max=1)
    assert_close(out["x"].cpu().numpy(), ref["x"], 1e-4)
    assert np.linalg.norm(out["z"].cpu().numpy() - ref["z"]) <= 1e-4 * np.linalg.norm(p.b)


def test_full_size_solves_stop_where_the_oracle_stops(setup):
    p, anchor, _, sol = setup
    b, xr = torch.from_numpy(p.b).to(DEV), torch.from_numpy(p.x_ref).to(DEV)
    target = int(anchor["iterations_to_1e-8"])
    plain = sol.solve(b, tol=1e-8, max_iter=100000, seed=1000, x_ref=xr)
    assert plain["status"] == R.REBK_OK
    assert abs(plain["stats"]["iterations"] - target) <= 10  # one test interval
    assert_converged(plain["x"].cpu().numpy(), p.x_ref, 1e-8)
    mixed = sol.solve_refined(b, tol=1e-8, seed=1000, storage="fp32", x_ref=xr)
    assert mixed["status"] == R.REBK_OK
    assert mixed["stats"]["iterations"] <= 1.05 * target
    assert_converged(mixed["x"].cpu().numpy(), p.x_ref, 1e-8)


def test_full_size_multi_rhs_pass_matches_oracle_per_member(setup):
    """Several right-hand sides at once at full size, in the benchmark's launch
    (groups of 8, one CTA per SM, products on tensor cores): the workload's b and 7
    more of the same law after one pass of 100 iterations, each against the
    oracle's pass on its own right-hand side, block indices bit-exact."""
    p, _, alpha, sol = setup
    ro, co = contiguous_offsets(M, TAU), contiguous_offsets(N, TAU)
    assert sol.multi_group("fp32") == 8
    rng = np.random.default_rng(11)
    B = np.array([p.b] + [p.A @ rng.standard_normal(N) + 0.01 * rng.standard_normal(M) for _ in range(7)])
    K = 100
    out = sol.solve_multi(torch.from_numpy(B).to(DEV), tol=0.0, max_iter=K, seed=21, storage="fp32", max_outer=1,
                          inner_iters=K, record=True)
    assert out["stats"]["iterations"] == K
    lo = O.round_fp32(p.A)
    idx_ref = O.rebk_correction(lo, *O.dual_residuals(p.A, B[0], B[0], np.zeros(N)), ro, co,
                                O.block_norms(p.A, ro, co), alpha, seed=21, iters=K, record=True)["idx"]
    assert np.array_equal(out["idx"][: 2 * K].view(-1, 2).cpu().numpy(), idx_ref)
    X = out["X"].cpu().numpy()
    for j in range(len(B)):
        ref = O.refine(p.A, B[j], lo, ro, co, alpha, seed=21, inner_iters=K, outer_max=1)
        assert_close(X[j], ref["x"], 1e-4)


# ---------------------------------------------------------------------------
# Batched systems at full size: 512 systems, m ~ U[200, 6000], n ~ U[50, 2000],
# 8 right-hand sides each, tau 16 (the benchmark's batch).
# ---------------------------------------------------------------------------

def test_full_size_batch_pass_matches_oracle_on_sampled_systems():
    """One pass (K inner iterations) of the whole 512-system batch; sampled
    systems and right-hand sides against the oracle's pass on the FP32-rounded
    matrix (bar 1e-4, as at small size).  alpha = 1 for every system: admissible
    for any matrix (beta_max <= 1), so no spectral norm is needed on either side."""
    from paper_2001_04179_gb300 import BatchSolver
    from workloads import batched_problems
    ps = batched_problems(512, seed=0, nrhs=8)
    bs = BatchSolver([p.A for p in ps], nrhs=8, tau=16, alpha=np.ones(len(ps)), max_outer=1)
    B = bs.stack_rhs([p.b for p in ps], bs.m)
    K = 50
    out = bs.solve(B, X_ref=None, tol=0.0, max_iter=K, inner_iters=K, seed=5, record_iters=K, return_z=True)
    assert out["stats"]["iterations"] == K * len(ps)
    xs = bs.split_x(out["x"])
    Z = out["z"].cpu().numpy()
    idx = out["idx"].cpu().numpy()
    big = int(np.argmax([p.m * p.n for p in ps]))
    for sid in sorted({0, 1, 100, 255, 383, 511, big}):
        p = ps[sid]
        ro, co = contiguous_offsets(p.m, 16), contiguous_offsets(p.n, 16)
        _, _, cr, cc = O.tables(p.A, ro, co)
        want = np.array([[O.pick(cc, O.uniform(5, sid, 2 * k)), O.pick(cr, O.uniform(5, sid, 2 * k + 1))]
                         for k in range(K)], dtype=np.int32)
        assert np.array_equal(idx[sid], want), sid
        if sid not in (0, 255, 511, big):
            continue
        lo = O.round_fp32(p.A)
        zs = Z[bs.mrow[sid]:bs.mrow[sid + 1]]
        for r in (0, 7):
            ref = O.refine(p.A, p.b[:, r], lo, ro, co, 1.0, seed=5, inner_iters=K, outer_max=1, stream=sid)
            assert_close(xs[sid][:, r], ref["x"], 1e-4, str((sid, r)))
            dz = zs[:, r] - ref["z"]
            assert np.linalg.norm(dz) <= 1e-4 * np.linalg.norm(p.b[:, r]), (sid, r)
    bs.close()


# ---------------------------------------------------------------------------
# Sparse at full size: 65536 x 16384, 96 nonzeros per row, tau 256.
# ---------------------------------------------------------------------------

def test_full_size_sparse_indices_and_iterates():
    """Plain FP64 sparse path against the oracle's CSR form of Algorithm 1 (the
    dense form would need 8.6 GB): bit-exact blocks and iterates within 1e-10,
    also 10^6 iterations into the random stream."""
    from paper_2001_04179_gb300 import SparseSolver
    from workloads import sparse_problem
    p = sparse_problem(65536, 16384, 96, seed=0, noise=0.01, decades=1.0, x_ref=None)
    sol = SparseSolver(p.m, p.n, p.indptr, p.indices, p.data, 256, 256)
    alpha = sol.alpha
    ro, co = contiguous_offsets(p.m, 256), contiguous_offsets(p.n, 256)
    b = torch.from_numpy(p.b).to(DEV)
    for k0, iters in [(0, 30), (1_000_000, 10)]:
        out = sol.solve(b, tol=0.0, max_iter=iters, seed=7, k0=k0, record=True, return_z=True)
        ref = O.rebk_sparse(p.m, p.n, p.indptr, p.indices, p.data, p.b, ro, co, alpha, seed=7, iters=iters,
                            k0=k0, record=True)
        assert np.array_equal(out["idx"].cpu().numpy(), ref["idx"])
        assert_close(out["x"].cpu().numpy(), ref["x"], 1e-10)
        assert_close(out["z"].cpu().numpy(), ref["z"], 1e-10)
    sol.close()


# ---------------------------------------------------------------------------
# Warm-start network at full size: 8192 -> 512 -> 512 -> 8192 on an 8192 x 2048 A.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("loss", ["x", "y_rel"])
def test_full_size_network_matches_oracle_network(loss):
    """Forward pass and gradients of the BF16 network at the warm-start workload's
    size against the FP64 oracle network on the same BF16-rounded weights and
    inputs (bars as at small size: 2e-2 forward and loss, 8e-2 gradients)."""
    from paper_2001_04179_gb300 import WarmStartNet
    from workloads import spectrum_problem
    p = spectrum_problem(8192, 2048, seed=0)
    Bsz, H = 64, 512
    rng = np.random.default_rng(1)
    W = [w.astype(np.float32) for w in O.mlp_init([8192, H, H, 8192], seed=3)]
    net = WarmStartNet(p.A, hidden=H, batch_capacity=Bsz, init_weights=W)
    Bm = rng.standard_normal((Bsz, 8192))
    bf = lambda a: O.round_bf16(np.asarray(a, dtype=np.float64))  # noqa: E731
    Wq = [bf(w) for w in W]
    if loss == "x":
        T = rng.standard_normal((Bsz, 2048))
        scale = 1.0
    else:
        T = rng.standard_normal((Bsz, 8192))
        scale = 0.37
        net.set_loss("y_rel", scale)
    Y = net.forward(torch.from_numpy(Bm).to(DEV)).cpu().numpy()
    y_ref, _ = O.mlp_forward(Wq, bf(Bm).T, out_scale=scale)
    assert _rel(Y, y_ref.T) <= 2e-2
    lval, grads = net.gradients(torch.from_numpy(Bm).to(DEV), torch.from_numpy(T).to(DEV))
    A_or_none = bf(p.A) if loss == "x" else None
    l_ref = O.mlp_loss(Wq, A_or_none, bf(Bm).T, T.T, loss, scale)
    assert lval == pytest.approx(l_ref, rel=2e-2)
    g_ref = O.mlp_backward(Wq, A_or_none, bf(Bm).T, T.T, loss=loss, out_scale=scale)
    for g, gr in zip(grads, g_ref):
        assert _rel(g, gr) <= 8e-2
    net.close()
