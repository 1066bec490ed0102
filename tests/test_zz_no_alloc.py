"""rebk_solve_noalloc: the solve entry point for callers that must not call
cudaMalloc (for example while a CUDA graph is being captured, or inside a host
that owns every device allocation).  It works in a fixed-size device array
inside the library, so its results must equal those of the allocating entry
point -- checked here on two calls in a row, so that the second call also
shows the scratch array's left-over contents from the first do not leak in.
This file is collected last on purpose."""
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
        b_dev = torch.from_numpy(b).to(DEV)
        x = torch.full((p.n,), float("nan"), dtype=torch.float64, device=DEV)
        z = torch.full((p.m,), float("nan"), dtype=torch.float64, device=DEV)
        st = fn(_P(A_dev.data_ptr()), p.m, p.n, p.n, 20, 20, alpha, _P(b_dev.data_ptr()), _P(x.data_ptr()),
                _P(z.data_ptr()), iters, seed, _P(stream.cuda_stream))
        assert st == R.REBK_OK, lib.rebk_last_error().decode()
        ref = sol.solve(b_dev, tol=0.0, max_iter=iters, seed=seed, return_z=True)
        # same iterates up to the device's reduction order (FP64 parity bar)
        assert _rel(x.cpu().numpy(), ref["x"].cpu().numpy()) <= 1e-10
        assert _rel(z.cpu().numpy(), ref["z"].cpu().numpy()) <= 1e-10


def test_noalloc_rejects_problems_larger_than_its_array():
    lib = R.load()
    fn = _noalloc(lib)
    m, n = 4096, 4096  # padded copy alone is 128 MiB > 32 MiB
    dummy = torch.zeros(8, dtype=torch.float64, device=DEV)
    ptr = _P(dummy.data_ptr())
    st = fn(ptr, m, n, n, 64, 64, 1.0, ptr, ptr, ptr, 10, 0, None)
    assert st == R.REBK_EUNSUPPORTED
    assert "scratch" in lib.rebk_last_error().decode()
    st = fn(ptr, 8, 4, 4, 2, 2, 0.0, ptr, ptr, ptr, 10, 0, None)  # alpha must be > 0
    assert st == R.REBK_EINVAL
