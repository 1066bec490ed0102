"""Pins for the FP64 warm-start network of the oracle.  The network maps a
right-hand side b to y and the solve starts from x^0 = A^T y, which lies in
range(A^T) as Theorem main requires; the loss is ||A^T y - A^+ b||^2."""
import numpy as np
import pytest

import oracle as O


def _setup(seed=0, sizes=(8, 6, 5, 8), B=3):
    rng = np.random.default_rng(seed)
    W = O.mlp_init(list(sizes), seed)
    A = rng.standard_normal((sizes[0], 4))
    Bm = rng.standard_normal((sizes[0], B))
    X = rng.standard_normal((4, B))
    return W, A, Bm, X


def test_gradients_match_finite_differences():
    W, A, Bm, X = _setup()
    grads = O.mlp_backward(W, A, Bm, X)
    h = 1e-6
    for l, Wl in enumerate(W):
        for (i, j) in [(0, 0), (1, 2), (Wl.shape[0] - 1, Wl.shape[1] - 1), (2, 1)]:
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (O.mlp_loss(Wp, A, Bm, X) - O.mlp_loss(Wm, A, Bm, X)) / (2 * h)
            assert grads[l][i, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_single_linear_layer_has_closed_form_gradient():
    """With one layer y = W b (no activation), dL/dW = (2/B) A (A^T W Bm - X) Bm^T."""
    rng = np.random.default_rng(4)
    W = [rng.standard_normal((7, 7))]
    A = rng.standard_normal((7, 3))
    Bm = rng.standard_normal((7, 5))
    X = rng.standard_normal((3, 5))
    g = O.mlp_backward(W, A, Bm, X)[0]
    exact = (2.0 / 5) * A @ (A.T @ W[0] @ Bm - X) @ Bm.T
    assert np.allclose(g, exact, rtol=1e-13, atol=1e-13)


def test_relu_masks_and_forward():
    W = [np.array([[1.0, -1.0], [2.0, 0.5]]), np.array([[1.0, 1.0]])]
    b = np.array([[1.0], [3.0]])
    y, (pres, acts) = O.mlp_forward(W, b)
    # layer 1: [1-3, 2+1.5] = [-2, 3.5] -> relu [0, 3.5]; layer 2: 3.5
    assert np.allclose(pres[0][:, 0], [-2.0, 3.5])
    assert np.allclose(acts[1][:, 0], [0.0, 3.5])
    assert y[0, 0] == 3.5


def test_warm_start_lies_in_range_of_At():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((10, 4)) @ rng.standard_normal((4, 7))
    W = O.mlp_init([10, 8, 10], 3)
    y, _ = O.mlp_forward(W, rng.standard_normal((10, 2)))
    x0 = A.T @ y
    U, s, Vt = np.linalg.svd(A)
    PV = Vt[:4].T @ Vt[:4]
    assert np.allclose(PV @ x0, x0, atol=1e-12)


@pytest.mark.parametrize("loss,scale", [("x", 2.5), ("y_rel", 1.0), ("y_rel", 3.7)])
def test_scaled_and_y_space_gradients_match_finite_differences(loss, scale):
    W, A, Bm, X = _setup(seed=5)
    rng = np.random.default_rng(6)
    T = X if loss == "x" else rng.standard_normal((Bm.shape[0], Bm.shape[1]))
    grads = O.mlp_backward(W, A, Bm, T, loss=loss, out_scale=scale)
    h = 1e-6
    for l, Wl in enumerate(W):
        for (i, j) in [(0, 0), (1, 2), (Wl.shape[0] - 1, Wl.shape[1] - 1)]:
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (O.mlp_loss(Wp, A, Bm, T, loss, scale) - O.mlp_loss(Wm, A, Bm, T, loss, scale)) / (2 * h)
            assert grads[l][i, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_single_layer_y_space_gradient_has_closed_form():
    """One layer y = s W b: dL/dW = (2 s / B) sum_b (s W b_b - t_b) b_b^T / ||t_b||^2."""
    rng = np.random.default_rng(8)
    W = [rng.standard_normal((6, 6))]
    Bm = rng.standard_normal((6, 4))
    T = rng.standard_normal((6, 4))
    s = 1.9
    g = O.mlp_backward(W, None, Bm, T, loss="y_rel", out_scale=s)[0]
    exact = np.zeros((6, 6))
    for b in range(4):
        exact += (s * W[0] @ Bm[:, b] - T[:, b])[:, None] * Bm[:, b][None, :] / np.dot(T[:, b], T[:, b])
    exact *= 2 * s / 4
    assert np.allclose(g, exact, rtol=1e-13, atol=1e-13)
    assert O.mlp_loss(W, None, Bm, T, "y_rel", s) == pytest.approx(
        np.mean([np.sum((s * W[0] @ Bm[:, b] - T[:, b]) ** 2) / np.dot(T[:, b], T[:, b]) for b in range(4)]),
        rel=1e-13)


def test_y_space_target_gives_the_least_squares_start():
    """y* = (A^T)^+ x_ls satisfies A^T y* = x_ls when x_ls is in range(A^T), so
    the y-space loss at zero means x^0 = x_ls."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((12, 3)) @ rng.standard_normal((3, 7))
    b = rng.standard_normal(12)
    x_ls = O.pinv_solve(A, b)
    y_star = O.pinv_solve(A.T, x_ls)
    assert np.allclose(A.T @ y_star, x_ls, atol=1e-10)
