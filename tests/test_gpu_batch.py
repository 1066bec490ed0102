"""Batched systems (rebk_batch_*) against the FP64 oracle.

Bars: every system's block draws bit-exact against the oracle's Philox stream
and table search (key (seed, system index)); one refinement pass per system
and right-hand side against the oracle's pass on the FP32-rounded matrix
within 1e-4 (x, as a norm and entry by entry) and 1e-4 ||b|| (z), the same
bars as the single-system mixed path; full solves reach ||x - A^+ b|| <= 1e-8 ||A^+ b|| for every RHS of
every converged system, and systems reported converged really are."""
import numpy as np
import pytest

import oracle as O
from workloads import batched_problems, contiguous_offsets

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from parity import assert_close  # noqa: E402
from paper_2001_04179_gb300 import BatchSolver  # noqa: E402
from paper_2001_04179_gb300 import rebk as R  # noqa: E402


def _alphas(ps, tau):
    out = []
    for p in ps:
        ro, co = contiguous_offsets(p.m, tau), contiguous_offsets(p.n, tau)
        out.append(1.5 / max(O.beta_max(p.A, ro, co)))
    return np.array(out)


def oracle_draws(A, tau, seed, system, iters):
    """(j_k, i_k) for k = 1..iters from the oracle's tables and Philox stream."""
    ro, co = contiguous_offsets(A.shape[0], tau), contiguous_offsets(A.shape[1], tau)
    _, _, cr, cc = O.tables(A, ro, co)
    out = np.zeros((iters, 2), dtype=np.int32)
    for k in range(iters):
        out[k, 0] = O.pick(cc, O.uniform(seed, system, 2 * k))
        out[k, 1] = O.pick(cr, O.uniform(seed, system, 2 * k + 1))
    return out


@pytest.mark.parametrize("nrhs,tau,path", [(8, 16, 0), (8, 16, 1), (3, 7, 0), (1, 32, 0), (2, 32, 1), (8, 64, 0),
                                           (4, 128, 0)])
def test_one_pass_matches_oracle_per_system(nrhs, tau, path):
    """Both column-step tile shapes for blocks of 16 / 32 columns, the wide-block
    layout (64, 128) and ragged blocks (7)."""
    ps = batched_problems(5, seed=11, scale_down=12, nrhs=nrhs)
    alphas = _alphas(ps, tau)
    bs = BatchSolver([p.A for p in ps], nrhs=nrhs, tau=tau, alpha=alphas, max_outer=1, col_path=path)
    B = bs.stack_rhs([p.b for p in ps], bs.m)
    K = 120
    out = bs.solve(B, X_ref=None, tol=0.0, max_iter=K, inner_iters=K, seed=5, record_iters=K, return_z=True)
    assert out["stats"]["iterations"] == K * len(ps)
    xs = bs.split_x(out["x"])
    Z = out["z"].cpu().numpy()
    idx = out["idx"].cpu().numpy()
    for sid, p in enumerate(ps):
        # the batch kernel's own sampler: every draw of every system, bit-exact
        assert np.array_equal(idx[sid], oracle_draws(p.A, tau, 5, sid, K)), sid
        ro, co = contiguous_offsets(p.m, tau), contiguous_offsets(p.n, tau)
        lo = O.round_fp32(p.A)
        zs = Z[bs.mrow[sid]:bs.mrow[sid + 1]]
        b = p.b.reshape(p.m, nrhs)
        for r in range(nrhs):
            ref = O.refine(p.A, b[:, r], lo, ro, co, alphas[sid], seed=5, inner_iters=K, outer_max=1,
                           stream=sid)
            assert_close(xs[sid][:, r], ref["x"], 1e-4, str((sid, r)))
            dz = zs[:, r] - ref["z"]
            assert np.linalg.norm(dz) <= 1e-4 * np.linalg.norm(b[:, r]), (sid, r)
            assert np.max(np.abs(dz)) <= 1e-4 * np.max(np.abs(b[:, r])), (sid, r)


@pytest.mark.parametrize("cluster,joint_frac,tau,path", [(2, 1e-9, 16, 0), (4, 1e-9, 16, 1), (4, 1e-9, 7, 0),
                                                          (8, 1e-9, 64, 0), (4, 8.0, 16, 0), (0, 0.0, 16, 0)])
def test_cluster_pass_matches_oracle_per_system(cluster, joint_frac, tau, path):
    """Systems run on a whole thread-block cluster (rows and columns split over
    its CTAs, the block products added up through distributed shared memory):
    the same draws and the same pass as one CTA per system.  joint_frac 1e-9
    puts every system on a cluster; 8 only the largest, the rest one per CTA.
    cluster 0 (library choice): the longest systems on clusters of 4 in a launch
    of their own beside the main one."""
    nrhs = 8
    ps = batched_problems(9, seed=13, scale_down=8, nrhs=nrhs)
    alphas = _alphas(ps, tau)
    bs = BatchSolver([p.A for p in ps], nrhs=nrhs, tau=tau, alpha=alphas, max_outer=1, col_path=path,
                     cluster=cluster, joint_frac=joint_frac)
    B = bs.stack_rhs([p.b for p in ps], bs.m)
    K = 100
    out = bs.solve(B, X_ref=None, tol=0.0, max_iter=K, inner_iters=K, seed=5, record_iters=K, return_z=True)
    st = out["stats"]
    assert st["iterations"] == K * len(ps)
    if cluster == 0:
        assert st["top_cluster"] == 4 and 1 <= st["top_joint"] < len(ps)
    else:
        assert st["cluster"] == cluster and st["top_joint"] == 0
        assert 1 <= st["joint"] <= len(ps)
        if joint_frac < 1e-6:
            assert st["joint"] == len(ps)
    xs = bs.split_x(out["x"])
    Z = out["z"].cpu().numpy()
    idx = out["idx"].cpu().numpy()
    for sid, p in enumerate(ps):
        assert np.array_equal(idx[sid], oracle_draws(p.A, tau, 5, sid, K)), sid
        ro, co = contiguous_offsets(p.m, tau), contiguous_offsets(p.n, tau)
        lo = O.round_fp32(p.A)
        zs = Z[bs.mrow[sid]:bs.mrow[sid + 1]]
        b = p.b.reshape(p.m, nrhs)
        for r in range(nrhs):
            ref = O.refine(p.A, b[:, r], lo, ro, co, alphas[sid], seed=5, inner_iters=K, outer_max=1,
                           stream=sid)
            assert_close(xs[sid][:, r], ref["x"], 1e-4, str((sid, r)))
            dz = zs[:, r] - ref["z"]
            assert np.linalg.norm(dz) <= 1e-4 * np.linalg.norm(b[:, r]), (sid, r)
            assert np.max(np.abs(dz)) <= 1e-4 * np.max(np.abs(b[:, r])), (sid, r)


@pytest.mark.parametrize("cluster", [2, 4])
def test_cluster_solves_reach_pseudoinverse_solutions(cluster):
    """The stopping test summed over the cluster's CTAs: every RHS of every
    system at 1e-8, and a second solve (planned from the first one's
    iteration counts) as well."""
    ps = batched_problems(10, seed=3, scale_down=10, nrhs=8)
    bs = BatchSolver([p.A for p in ps], nrhs=8, tau=16, cluster=cluster, joint_frac=0.3)
    B = bs.stack_rhs([p.b for p in ps], bs.m)
    Xr = bs.stack_rhs([p.x_ref for p in ps], bs.n)
    for seed in (9, 10):
        out = bs.solve(B, X_ref=Xr, tol=1e-8, max_iter=400000, seed=seed)
        st = out["stats"]
        assert st["cluster"] == cluster and st["joint"] >= 1
        assert st["converged"] == len(ps)
        assert np.all(out["status"] == R.REBK_OK)
        xs = bs.split_x(out["x"])
        for sid, p in enumerate(ps):
            for r in range(8):
                err = np.linalg.norm(xs[sid][:, r] - p.x_ref[:, r]) / np.linalg.norm(p.x_ref[:, r])
                assert err <= 1e-8, (sid, r, err)


def test_batch_reaches_pseudoinverse_solutions():
    ps = batched_problems(12, seed=3, scale_down=10, nrhs=8)
    bs = BatchSolver([p.A for p in ps], nrhs=8, tau=16)
    B = bs.stack_rhs([p.b for p in ps], bs.m)
    Xr = bs.stack_rhs([p.x_ref for p in ps], bs.n)
    out = bs.solve(B, X_ref=Xr, tol=1e-8, max_iter=400000, seed=9)
    st = out["stats"]
    assert st["graph"] == 1
    assert st["converged"] == len(ps)
    assert np.all(out["status"] == R.REBK_OK)
    xs = bs.split_x(out["x"])
    for sid, p in enumerate(ps):
        for r in range(8):
            err = np.linalg.norm(xs[sid][:, r] - p.x_ref[:, r]) / np.linalg.norm(p.x_ref[:, r])
            assert err <= 1e-8, (sid, r, err)


def test_iteration_cap_reports_unconverged_systems():
    """A nearly square Gaussian system (kappa in the hundreds) cannot reach
    1e-8 within a small cap: it is reported as MAX_ITER, the others as OK."""
    rng = np.random.default_rng(4)
    As, bs_, xs_ = [], [], []
    for m, n in [(120, 40), (100, 98), (90, 30)]:
        A = rng.standard_normal((m, n))
        X = rng.standard_normal((n, 2))
        B = A @ X
        As.append(A)
        bs_.append(B)
        xs_.append(np.linalg.lstsq(A, B, rcond=None)[0])
    bs = BatchSolver(As, nrhs=2, tau=8)
    out = bs.solve(bs.stack_rhs(bs_, bs.m), X_ref=bs.stack_rhs(xs_, bs.n), tol=1e-8, max_iter=3000, seed=1)
    assert list(out["status"]) == [R.REBK_OK, R.REBK_MAX_ITER, R.REBK_OK]
    assert out["stats"]["converged"] == 2


def test_autotuned_block_size():
    ps = batched_problems(6, seed=21, scale_down=10, nrhs=4)
    bs = BatchSolver([p.A for p in ps], nrhs=4, tau=0)
    B = bs.stack_rhs([p.b for p in ps], bs.m)
    Xr = bs.stack_rhs([p.x_ref for p in ps], bs.n)
    out = bs.solve(B, X_ref=Xr, tol=1e-8, max_iter=400000, seed=2)
    assert out["stats"]["tau"] in (16, 32, 64, 128, 256)
    assert out["stats"]["col_path"] in (0, 1)
    assert out["stats"]["col_path"] == 0 or out["stats"]["tau"] in (16, 32)
    assert out["stats"]["converged"] == len(ps)


def test_systems_sharing_a_matrix_match_separate_copies():
    """Equal pointers with equal shapes are stored once; the iterates are those
    of separate copies (same data, same per-system block sequences) up to the
    summation order of the FP64 sweeps' atomic adds."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((150, 60))
    Xs = rng.standard_normal((60, 8 * 4))
    Bm = A @ Xs
    blocks = [Bm[:, 8 * i:8 * i + 8] for i in range(4)]
    shared = BatchSolver([A] * 4, nrhs=8, tau=16, alpha=[1.0] * 4, max_outer=1)
    copies = BatchSolver([A.copy() for _ in range(4)], nrhs=8, tau=16, alpha=[1.0] * 4, max_outer=1)
    B = shared.stack_rhs(blocks, shared.m)
    a = shared.solve(B, X_ref=None, tol=0.0, max_iter=0, inner_iters=300, seed=2)["x"].cpu().numpy()
    b = copies.solve(B, X_ref=None, tol=0.0, max_iter=0, inner_iters=300, seed=2)["x"].cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_batched_warm_start_converges_in_fewer_iterations():
    """X0 = x_ls + 1e-3 perturbation in range(A^T), Z0 = b - A X0: every system
    still reaches 1e-8, with fewer inner iterations than from x = 0, z = b."""
    ps = batched_problems(6, seed=13, scale_down=10, nrhs=8)
    bs = BatchSolver([p.A for p in ps], nrhs=8, tau=16)
    B = bs.stack_rhs([p.b for p in ps], bs.m)
    Xr = bs.stack_rhs([p.x_ref for p in ps], bs.n)
    rng = np.random.default_rng(5)
    x0s, z0s = [], []
    for p in ps:
        pert = p.A.T @ rng.standard_normal((p.A.shape[0], 8))
        pert *= 1e-3 * np.linalg.norm(p.x_ref) / max(np.linalg.norm(pert), 1e-300)
        x0 = p.x_ref + pert
        x0s.append(x0)
        z0s.append(p.b - p.A @ x0)
    X0 = bs.stack_rhs(x0s, bs.n)
    Z0 = bs.stack_rhs(z0s, bs.m)
    cold = bs.solve(B, X_ref=Xr, tol=1e-8, max_iter=400000, seed=9)
    warm = bs.solve(B, X_ref=Xr, tol=1e-8, max_iter=400000, seed=9, X0=X0, Z0=Z0)
    assert cold["stats"]["converged"] == len(ps) and warm["stats"]["converged"] == len(ps)
    xs = bs.split_x(warm["x"])
    for sid, p in enumerate(ps):
        for r in range(8):
            err = np.linalg.norm(xs[sid][:, r] - p.x_ref[:, r]) / np.linalg.norm(p.x_ref[:, r])
            assert err <= 1e-8, (sid, r, err)
    assert warm["stats"]["iterations"] < 0.8 * cold["stats"]["iterations"]
