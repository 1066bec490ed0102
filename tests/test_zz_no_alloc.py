"""rebk_solve_noalloc: the solve entry point for callers that must not call
cudaMalloc (a host that routes every device allocation through its own
allocator, or a serving loop that must not take the driver's allocation
locks).  It works in a fixed-size device array inside the library, so its
results must equal those of the allocating entry point -- checked here on
calls in a row, so that later calls also show the scratch array's left-over
contents from earlier ones do not leak in: a second call on the same problem,
one whose A is a column slice of a wider matrix (leading dimension > n), and
one with a different shape and block sizes (its tables sit at other offsets
of the reused array).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle as O
from workloads import contiguous_offsets, gaussian_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2001_04179_gb300 import Solver  # noqa: E402
from paper_2001_04179_gb300 import rebk as R  # noqa: E402

DEV = torch.device("cuda:0")
_P = ctypes.c_void_p


def _noalloc(lib):
    fn = lib.rebk_solve_noalloc
    fn.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                   ctypes.c_double, _P, _P, _P, ctypes.c_int64, ctypes.c_uint64, _P]
    fn.restype = ctypes.c_int
    return fn


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _call(fn, lib, A_dev, lda, tau_r, tau_c, alpha, b, iters, seed, stream):
    m, n = A_dev.shape
    b_dev = torch.from_numpy(b).to(DEV)
    x = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
    z = torch.full((m,), float("nan"), dtype=torch.float64, device=DEV)
    st = fn(_P(A_dev.data_ptr()), m, n, lda, tau_r, tau_c, alpha, _P(b_dev.data_ptr()), _P(x.data_ptr()),
            _P(z.data_ptr()), iters, seed, _P(stream.cuda_stream))
    assert st == R.REBK_OK, lib.rebk_last_error().decode()
    return b_dev, x.cpu().numpy(), z.cpu().numpy()


def _check_against_solver(sol, b_dev, x, z, iters, seed):
    ref = sol.solve(b_dev, tol=0.0, max_iter=iters, seed=seed, return_z=True)
    xr, zr = ref["x"].cpu().numpy(), ref["z"].cpu().numpy()
    # same iterates up to the device's reduction order (FP64 parity bar), as a
    # norm and entry by entry
    assert _rel(x, xr) <= 1e-10
    assert _rel(z, zr) <= 1e-10
    assert np.max(np.abs(x - xr)) <= 1e-10 * np.max(np.abs(xr))
    assert np.max(np.abs(z - zr)) <= 1e-10 * np.max(np.abs(zr))


def test_noalloc_matches_allocating_solve_on_two_calls():
    lib = R.load()
    fn = _noalloc(lib)
    p = gaussian_problem(1000, 200, seed=0)
    ro, co = contiguous_offsets(1000, 20), contiguous_offsets(200, 20)
    alpha = 2.25 / max(O.beta_max(p.A, ro, co))
    A_dev = torch.from_numpy(p.A).to(DEV)
    sol = Solver(p.A, 20, 20, alpha=alpha, storage=())
    rng = np.random.default_rng(1)
    stream = torch.cuda.current_stream()
    for call, (seed, iters) in enumerate([(1000, 400), (77, 250)]):
        b = p.b if call == 0 else p.b + 0.1 * rng.standard_normal(p.m)
        b_dev, x, z = _call(fn, lib, A_dev, p.n, 20, 20, alpha, b, iters, seed, stream)
        _check_against_solver(sol, b_dev, x, z, iters, seed)


def test_noalloc_strided_matrix_and_a_second_shape():
    lib = R.load()
    fn = _noalloc(lib)
    stream = torch.cuda.current_stream()
    # A as a column slice of a wider matrix: leading dimension 300 > n = 200
    p = gaussian_problem(1000, 200, seed=4)
    wide = np.zeros((1000, 300))
    wide[:, 50:250] = p.A
    W_dev = torch.from_numpy(wide).to(DEV)
    A_view = W_dev[:, 50:250]
    ro, co = contiguous_offsets(1000, 20), contiguous_offsets(200, 20)
    alpha = 2.0 / max(O.beta_max(p.A, ro, co))
    sol = Solver(p.A, 20, 20, alpha=alpha, storage=())
    b_dev, x, z = _call(fn, lib, A_view, 300, 20, 20, alpha, p.b, 300, 5, stream)
    _check_against_solver(sol, b_dev, x, z, 300, 5)
    # then a smaller problem with other block sizes (ragged last blocks)
    q = gaussian_problem(333, 97, seed=6)
    ro, co = contiguous_offsets(333, 13), contiguous_offsets(97, 7)
    alpha = 1.75 / max(O.beta_max(q.A, ro, co))
    sol = Solver(q.A, 13, 7, alpha=alpha, storage=())
    Aq = torch.from_numpy(q.A).to(DEV)
    b_dev, x, z = _call(fn, lib, Aq, q.n, 13, 7, alpha, q.b, 500, 11, stream)
    _check_against_solver(sol, b_dev, x, z, 500, 11)


def test_noalloc_rejects_problems_larger_than_its_array():
    lib = R.load()
    fn = _noalloc(lib)
    m, n = 4096, 4096  # padded copy alone is 128 MiB > 32 MiB
    dummy = torch.zeros(8, dtype=torch.float64, device=DEV)
    ptr = _P(dummy.data_ptr())
    st = fn(ptr, m, n, n, 64, 64, 1.0, ptr, ptr, ptr, 10, 0, None)
    assert st == R.REBK_EUNSUPPORTED
    assert "scratch" in lib.rebk_last_error().decode()
    # sizes whose byte counts would overflow are rejected before any arithmetic on them
    big = 1 << 61
    st = fn(ptr, big, 4, 4, 2, 2, 1.0, ptr, ptr, ptr, 10, 0, None)
    assert st == R.REBK_EUNSUPPORTED
    st = fn(ptr, 4, big, big, 2, 2, 1.0, ptr, ptr, ptr, 10, 0, None)
    assert st == R.REBK_EUNSUPPORTED
    st = fn(ptr, 8, 4, 4, 2, 2, 0.0, ptr, ptr, ptr, 10, 0, None)  # alpha must be > 0
    assert st == R.REBK_EINVAL
