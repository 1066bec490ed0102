"""Full-size parity on the 8000 x 20000 rank-2000 workload (A = G1 G2, b = A x* +
N(0, 0.01^2), seed 0), in the launch configuration the benchmark times: tau = 128
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
The step size is the oracle's recorded alpha, passed to both sides."""
import os

import numpy as np
import pytest

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
        assert _rel(out["x"].cpu().numpy(), ref["x"]) <= 1e-10
        assert _rel(out["z"].cpu().numpy(), ref["z"]) <= 1e-10


def test_full_size_mixed_pass_matches_oracle_pass(setup):
    p, _, alpha, sol = setup
    ro, co = contiguous_offsets(M, TAU), contiguous_offsets(N, TAU)
    K = 100
    out = sol.solve_refined(torch.from_numpy(p.b).to(DEV), tol=0.0, max_iter=K, seed=21, storage="fp32",
                            max_outer=1, inner_iters=K, record=True, return_z=True)
    assert out["stats"]["iterations"] == K
    ref = O.refine(p.A, p.b, O.round_fp32(p.A), ro, co, alpha, seed=21, inner_iters=K, outer_max=1)
    assert _rel(out["x"].cpu().numpy(), ref["x"]) <= 1e-4
    assert np.linalg.norm(out["z"].cpu().numpy() - ref["z"]) <= 1e-4 * np.linalg.norm(p.b)


def test_full_size_solves_stop_where_the_oracle_stops(setup):
    p, anchor, _, sol = setup
    b, xr = torch.from_numpy(p.b).to(DEV), torch.from_numpy(p.x_ref).to(DEV)
    target = int(anchor["iterations_to_1e-8"])
    plain = sol.solve(b, tol=1e-8, max_iter=100000, seed=1000, x_ref=xr)
    assert plain["status"] == R.REBK_OK
    assert abs(plain["stats"]["iterations"] - target) <= 10  # one test interval
    assert _rel(plain["x"].cpu().numpy(), p.x_ref) <= 1e-8
    mixed = sol.solve_refined(b, tol=1e-8, seed=1000, storage="fp32", x_ref=xr)
    assert mixed["status"] == R.REBK_OK
    assert mixed["stats"]["iterations"] <= 1.05 * target
    assert _rel(mixed["x"].cpu().numpy(), p.x_ref) <= 1e-8
