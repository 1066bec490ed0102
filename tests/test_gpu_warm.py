"""Learned warm start (rebk_mlp_*, rebk_warm_start) against the FP64 oracle
network and against the cold start.

Bars: the network runs BF16 operands with FP32 accumulation; compared with the
oracle's FP64 forward / backward on the same BF16-rounded weights and inputs,
the BF16 rounding of each layer's activation (2^-9 relative) over three
layers bounds the forward error near 5e-3 relative (bar 2e-2) and the
gradients, which also pass through BF16-rounded back-propagated signals, near
2e-2 (bar 8e-2)."""
import numpy as np
import pytest

import oracle as O
from workloads import contiguous_offsets, spectrum_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2001_04179_gb300 import Solver, WarmStartNet  # noqa: E402
from paper_2001_04179_gb300 import rebk as R  # noqa: E402

DEV = torch.device("cuda:0")


def _bf16(a):
    return O.round_bf16(np.asarray(a, dtype=np.float64))


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_forward_and_gradients_match_oracle_network():
    rng = np.random.default_rng(0)
    m, n, H, B = 96, 40, 64, 24
    A = rng.standard_normal((m, n)) / np.sqrt(m)
    W = [w.astype(np.float32) for w in O.mlp_init([m, H, H, m], seed=3)]
    net = WarmStartNet(A, hidden=H, batch_capacity=B, init_weights=W)
    Bm = rng.standard_normal((B, m))
    Xls = rng.standard_normal((B, n))
    Wq = [_bf16(w) for w in W]
    Y = net.forward(_t(Bm)).cpu().numpy()
    y_ref, _ = O.mlp_forward(Wq, _bf16(Bm).T)
    assert _rel(Y, y_ref.T) <= 2e-2
    loss, grads = net.gradients(_t(Bm), _t(Xls))
    loss_ref = O.mlp_loss(Wq, _bf16(A), _bf16(Bm).T, Xls.T)
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    g_ref = O.mlp_backward(Wq, _bf16(A), _bf16(Bm).T, Xls.T)
    for g, gr in zip(grads, g_ref):
        assert _rel(g, gr) <= 8e-2


def test_training_lowers_the_loss():
    p = spectrum_problem(256, 64, seed=1, latent=6, nrhs=512)
    net = WarmStartNet(p.A, hidden=128, batch_capacity=128, seed=2)
    Bm, Xs = p.b.T, p.x_ref.T
    first = None
    for epoch in range(60):
        for s in range(0, 512, 128):
            loss = net.train_step(_t(Bm[s:s + 128]), _t(Xs[s:s + 128]), lr=2e-3)
            first = loss if first is None else first
    assert loss < 0.05 * first


def test_warm_start_cuts_iterations_and_keeps_the_limit():
    """A network trained on solver-generated (b, x_ls) pairs of one A: the
    warm-started mixed solve reaches the same 1e-8 relative error in fewer
    iterations than the cold start, and x0 = A^T y lies in range(A^T)."""
    m, n = 512, 128
    p = spectrum_problem(m, n, seed=4, latent=8, nrhs=640)
    tau = 16
    ro, co = contiguous_offsets(m, tau), contiguous_offsets(n, tau)
    alpha = 1.75 / max(O.beta_max(p.A, ro, co))
    sol = Solver(p.A, tau, tau, alpha=alpha, storage=("fp32",))
    # training targets from the solver itself (mixed precision, 1e-9)
    X = np.zeros((640, n))
    for i in range(512):
        X[i] = sol.solve_refined(_t(p.b[:, i]), tol=1e-9, seed=100 + i, x_ref=_t(p.x_ref[:, i]))["x"].cpu().numpy()
    assert _rel(X[:512].T, p.x_ref[:, :512]) <= 1e-8
    net = WarmStartNet(p.A, hidden=256, batch_capacity=128, seed=5)
    for epoch in range(150):
        for s in range(0, 512, 128):
            net.train_step(_t(p.b[:, s:s + 128].T), _t(X[s:s + 128]), lr=1e-3)
    cold, warm = [], []
    for i in range(512, 640):
        b, xr = _t(p.b[:, i]), _t(p.x_ref[:, i])
        c = sol.solve_refined(b, tol=1e-8, seed=7, x_ref=xr)
        x0, z0 = net.warm_start(sol, b)
        w = sol.solve_refined(b, tol=1e-8, seed=7, x_ref=xr, x0=x0, z0=z0)
        assert c["status"] == R.REBK_OK and w["status"] == R.REBK_OK
        assert w["stats"]["rel_err"] <= 1e-8
        cold.append(c["stats"]["iterations"])
        warm.append(w["stats"]["iterations"])
    assert np.mean(warm) < 0.85 * np.mean(cold), (np.mean(warm), np.mean(cold))


def test_y_space_loss_and_output_scale_match_oracle_network():
    rng = np.random.default_rng(1)
    m, n, H, B = 96, 40, 64, 24
    A = rng.standard_normal((m, n)) / np.sqrt(m)
    W = [w.astype(np.float32) for w in O.mlp_init([m, H, H, m], seed=4)]
    net = WarmStartNet(A, hidden=H, batch_capacity=B, init_weights=W)
    s = 7.5
    net.set_loss("y_rel", s)
    Bm = rng.standard_normal((B, m))
    Ys = rng.standard_normal((B, m)) * 20.0
    Wq = [_bf16(w) for w in W]
    Y = net.forward(_t(Bm)).cpu().numpy()
    y_ref, _ = O.mlp_forward(Wq, _bf16(Bm).T, out_scale=s)
    assert _rel(Y, y_ref.T) <= 2e-2
    loss, grads = net.gradients(_t(Bm), _t(Ys))
    assert loss == pytest.approx(O.mlp_loss(Wq, None, _bf16(Bm).T, Ys.T, "y_rel", s), rel=2e-2)
    g_ref = O.mlp_backward(Wq, None, _bf16(Bm).T, Ys.T, loss="y_rel", out_scale=s)
    for g, gr in zip(grads, g_ref):
        assert _rel(g, gr) <= 8e-2
    with pytest.raises(R.RebkError):
        net.set_loss("y_rel", 0.0)


def test_y_space_training_on_batched_solver_targets_cuts_iterations():
    """The recipe of the 8192 x 2048 study at a small size: x_ls from batched
    systems sharing A, y* = (A^T)^+ x_ls from batched systems sharing A^T,
    training with the y-space loss; warm mixed solves (FP32 and BF16) reach
    1e-8 in fewer iterations than cold ones."""
    from paper_2001_04179_gb300 import BatchSolver
    m, n, ntr, nev = 1024, 256, 512, 32
    p = spectrum_problem(m, n, seed=6, latent=8, nrhs=ntr + nev)
    tau = 32
    ro, co = contiguous_offsets(m, tau), contiguous_offsets(n, tau)
    alpha = 1.75 / max(O.beta_max(p.A, ro, co))
    ns = ntr // 8
    At = np.ascontiguousarray(p.A.T)
    bsA = BatchSolver([p.A] * ns, nrhs=8, tau=tau, alpha=[alpha] * ns, max_outer=2)
    Bsys = _t(np.concatenate([p.b[:, 8 * i:8 * i + 8] for i in range(ns)], axis=0))
    Xs = bsA.solve(Bsys, X_ref=None, tol=0.0, max_iter=0, inner_iters=20000, seed=3)["x"]
    Xtr = Xs.view(ns, n, 8).permute(0, 2, 1).reshape(ntr, n).cpu().numpy()
    assert _rel(Xtr.T, p.x_ref[:, :ntr]) <= 1e-8
    bsT = BatchSolver([At] * ns, nrhs=8, tau=tau, alpha=[alpha] * ns, max_outer=2)
    Ys = bsT.solve(Xs, X_ref=None, tol=0.0, max_iter=0, inner_iters=20000, seed=4)["x"]
    Ytr = Ys.view(ns, m, 8).permute(0, 2, 1).reshape(ntr, m).contiguous()
    # y* is the minimum-norm solution of A^T y = x_ls
    assert _rel(At @ Ytr.cpu().numpy().T, Xtr.T) <= 1e-7
    net = WarmStartNet(p.A, hidden=256, batch_capacity=128, seed=5)
    Btr = _t(p.b[:, :ntr].T)
    scale = 0.1 * float(np.sqrt(np.mean(np.sum(Ytr.cpu().numpy() ** 2, 1)) / np.mean(np.sum(p.b[:, :ntr] ** 2, 0))))
    net.set_loss("y_rel", scale)
    losses = net.fit(Btr, Ytr, steps=1500, lr=1e-3, batch=128)
    assert np.mean(losses[-10:]) < 0.02 * losses[0]
    sol = Solver(p.A, tau, tau, alpha=alpha, storage=("fp32", "bf16"))
    for st in ("fp32", "bf16"):
        cold, warm = [], []
        for i in range(ntr, ntr + nev):
            b, xr = _t(p.b[:, i]), _t(p.x_ref[:, i])
            c = sol.solve_refined(b, tol=1e-8, seed=7, storage=st, x_ref=xr)
            x0, z0 = net.warm_start(sol, b)
            w = sol.solve_refined(b, tol=1e-8, seed=7, storage=st, x_ref=xr, x0=x0, z0=z0)
            assert c["status"] == R.REBK_OK and w["status"] == R.REBK_OK
            assert w["stats"]["rel_err"] <= 1e-8
            cold.append(c["stats"]["iterations"])
            warm.append(w["stats"]["iterations"])
        if st == "fp32":
            assert np.mean(warm) < 0.85 * np.mean(cold), (st, np.mean(warm), np.mean(cold))
        else:  # BF16: bounded by the refinement's stagnation rule, no runaway pass
            assert np.mean(warm) < 2.0 * np.mean(cold), (st, np.mean(warm), np.mean(cold))


def test_batched_warm_start_matches_single_right_hand_sides():
    rng = np.random.default_rng(3)
    m, n = 200, 60
    A = rng.standard_normal((m, n))
    net = WarmStartNet(A, hidden=64, batch_capacity=16, seed=2)
    sol = Solver(A, 8, 8, alpha=0.0, storage=("fp32",))
    count, g = 40, 8  # three network batches (16, 16, 8)
    Bg = rng.standard_normal((count // g * m, g))
    X0, Z0 = net.warm_start_batch(sol, _t(Bg), count, group=g)
    X0, Z0 = X0.cpu().numpy(), Z0.cpu().numpy()
    for j in range(count):
        blk, col = divmod(j, g)
        b = Bg[blk * m:(blk + 1) * m, col]
        x0, z0 = net.warm_start(sol, _t(b))
        assert _rel(X0[blk * n:(blk + 1) * n, col], x0.cpu().numpy()) <= 1e-12
        assert _rel(Z0[blk * m:(blk + 1) * m, col], z0.cpu().numpy()) <= 1e-12
    with pytest.raises(R.RebkError):
        net.warm_start_batch(sol, _t(Bg), count - 1, group=g)
