"""The warm-start network's BF16 GEMM (rebk_gemm_bf16: tcgen05 tensor cores,
TMA-staged tiles, accumulator in tensor memory) against the FP64 product of
the same BF16 values.

Bar: every entry within 1e-5 of sum_k |A_ik| |B_jk| (FP32 accumulation of K
products: rounding of about 2^-24 per add, summed in some order) plus 1e-30.
Shapes cover the network's products (M = 256 batch rows, K = 8192 inputs:
split over K; M = 8192, K = 256: many tiles), ragged tails in M, N and K (K
off a multiple of the 64-wide slice), a single row, and leading dimensions
above K; K not a multiple of 8 takes the mma.sync path."""
import ctypes

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2001_04179_gb300 import rebk as R  # noqa: E402

DEV = torch.device("cuda:0")


def _bf16_bits(x):
    f = O.round_bf16(x).astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16), O.round_bf16(x)


SHAPES = [
    # M, N, K, lda pad, ldb pad, expected path
    (256, 512, 8192, 0, 0, 1),
    (8192, 512, 256, 0, 0, 1),
    (256, 8192, 512, 0, 0, 1),
    (300, 200, 72, 8, 16, 1),
    (1, 130, 136, 0, 0, 1),
    (129, 257, 1000, 24, 0, 1),
    (40, 33, 13, 3, 5, 0),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s[:3])))
def test_gemm_matches_fp64_product(shape):
    M, N, K, pa, pb, path_want = shape
    rng = np.random.default_rng(M + 7 * N + 13 * K)
    lda, ldb = K + pa, K + pb
    A = rng.standard_normal((M, lda))
    B = rng.standard_normal((N, ldb)) * 0.5
    Ab, Av = _bf16_bits(A)
    Bb, Bv = _bf16_bits(B)
    Ad = torch.from_numpy(Ab.view(np.int16)).to(DEV)
    Bd = torch.from_numpy(Bb.view(np.int16)).to(DEV)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device=DEV)
    path = ctypes.c_int32(-1)
    alpha = 0.75
    st = R.load().rebk_gemm_bf16(M, N, K, ctypes.c_void_p(Ad.data_ptr()), lda, ctypes.c_void_p(Bd.data_ptr()), ldb,
                                 alpha, ctypes.c_void_p(C.data_ptr()), N, None, ctypes.byref(path))
    assert st == R.REBK_OK, R.load().rebk_last_error().decode()
    assert path.value == path_want
    ref = alpha * (Av[:, :K] @ Bv[:, :K].T)
    scale = alpha * (np.abs(Av[:, :K]) @ np.abs(Bv[:, :K]).T)
    got = C.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-30)
