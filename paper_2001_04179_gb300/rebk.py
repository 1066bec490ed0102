"""ctypes binding of librebk.so (include/rebk.h).  Argument marshalling only.

Device memory comes from torch tensors (``data_ptr()``); every step of the
method runs in the library's CUDA kernels.  There is no CPU path: if the
library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

from . import build as _build

REBK_OK, REBK_EINVAL, REBK_ENOMEM, REBK_ECUDA = 0, 1, 2, 3
REBK_MAX_ITER, REBK_DIVERGED, REBK_BARRIER_TIMEOUT, REBK_EUNSUPPORTED = 4, 5, 6, 7
REBK_FP64, REBK_FP32, REBK_BF16 = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "MAX_ITER", 5: "DIVERGED",
                6: "BARRIER_TIMEOUT", 7: "EUNSUPPORTED"}
STORAGE = {"fp64": REBK_FP64, "fp32": REBK_FP32, "bf16": REBK_BF16}


class RebkOptions(ctypes.Structure):
    _fields_ = [("tau_row", ctypes.c_int64), ("tau_col", ctypes.c_int64),
                ("storage_mask", ctypes.c_int32), ("num_ctas", ctypes.c_int32),
                ("check_every", ctypes.c_int64), ("stream", ctypes.c_void_p)]


class RebkStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("outer", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rel_err", ctypes.c_double), ("resid_f", ctypes.c_double),
                ("resid_g", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("sweep_ms", ctypes.c_double),
                ("launches", ctypes.c_int64), ("grid_launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class RebkSolveExt(ctypes.Structure):
    _fields_ = [("x_ref", ctypes.c_void_p), ("x0", ctypes.c_void_p), ("z0", ctypes.c_void_p),
                ("z_out", ctypes.c_void_p), ("idx_out", ctypes.c_void_p), ("k0", ctypes.c_int64),
                ("stream_id", ctypes.c_uint64)]


class RebkRefineOpts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("inner_iters", ctypes.c_int64), ("inner_reduction", ctypes.c_double)]


class RebkMultiOpts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("group", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("inner_iters", ctypes.c_int64), ("inner_reduction", ctypes.c_double),
                ("idx_out", ctypes.c_void_p), ("stream_id", ctypes.c_uint64)]


class RebkTunePoint(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_int64), ("beta_max", ctypes.c_double), ("alpha", ctypes.c_double),
                ("iterations", ctypes.c_int64), ("device_ms", ctypes.c_double), ("status", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class RebkSpectrum(ctypes.Structure):
    _fields_ = [("sigma1_sq", ctypes.c_double), ("sigma_r_sq", ctypes.c_double), ("fro2", ctypes.c_double),
                ("alpha_mean_opt", ctypes.c_double), ("delta_opt", ctypes.c_double), ("alpha", ctypes.c_double),
                ("delta", ctypes.c_double), ("eta", ctypes.c_double), ("rho", ctypes.c_double),
                ("beta_row", ctypes.c_double), ("beta_col", ctypes.c_double), ("steps", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class RebkBatchOptions(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("inner_reduction", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("col_path", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("joint_frac", ctypes.c_double)]


class RebkBatchStats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int32), ("outer", ctypes.c_int32), ("iterations", ctypes.c_int64),
                ("max_iterations", ctypes.c_int64), ("device_ms", ctypes.c_double),
                ("inner_ms", ctypes.c_double), ("sweep_ms", ctypes.c_double), ("launches", ctypes.c_int64),
                ("tau", ctypes.c_int32), ("graph", ctypes.c_int32), ("col_path", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("joint", ctypes.c_int32), ("top_cluster", ctypes.c_int32),
                ("top_joint", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class RebkPartition(ctypes.Structure):
    _fields_ = [("row_off", ctypes.c_void_p), ("s", ctypes.c_int64), ("col_off", ctypes.c_void_p),
                ("t", ctypes.c_int64)]


class RebkPeaks(ctypes.Structure):
    _fields_ = [("fp64_tflops", ctypes.c_double), ("fp64_ms", ctypes.c_double), ("sm_mhz", ctypes.c_double),
                ("l2_gbs", ctypes.c_double), ("l2_ms", ctypes.c_double), ("l2_bytes", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class RebkSparseOptions(ctypes.Structure):
    _fields_ = [("num_ctas", ctypes.c_int32), ("check_every", ctypes.c_int32), ("power_iters", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None

_P = ctypes.c_void_p
_SIGNATURES = {
    "rebk_create": ([ctypes.POINTER(_P), _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                     ctypes.POINTER(RebkPartition), ctypes.c_double, ctypes.POINTER(RebkOptions)], ctypes.c_int),
    "rebk_get_partition": ([_P, _P, _P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
                           ctypes.c_int),
    "rebk_destroy": ([_P], None),
    "rebk_solve": ([_P, _P, _P, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                    ctypes.POINTER(RebkStats)], ctypes.c_int),
    "rebk_solve_ex": ([_P, _P, _P, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                       ctypes.POINTER(RebkSolveExt), ctypes.POINTER(RebkStats)], ctypes.c_int),
    "rebk_solve_refined": ([_P, _P, _P, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                            ctypes.POINTER(RebkRefineOpts), ctypes.POINTER(RebkSolveExt),
                            ctypes.POINTER(RebkStats)], ctypes.c_int),
    "rebk_solve_free": ([_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, _P, _P, ctypes.c_double,
                         ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(RebkSolveExt), ctypes.POINTER(RebkStats)],
                        ctypes.c_int),
    "rebk_solve_multi": ([_P, ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_double,
                          ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(RebkMultiOpts), _P, ctypes.c_int64, _P,
                          ctypes.POINTER(RebkStats)], ctypes.c_int),
    "rebk_multi_group": ([_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "rebk_beta_max": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "rebk_get_alpha": ([_P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "rebk_set_alpha": ([_P, ctypes.c_double], ctypes.c_int),
    "rebk_spectral_estimates": ([_P, ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(RebkSpectrum)], ctypes.c_int),
    "rebk_tune_tau": ([_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _P, _P, _P, ctypes.c_int32,
                       ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                       ctypes.c_int32, ctypes.POINTER(RebkOptions), _P, ctypes.POINTER(ctypes.c_int64)],
                      ctypes.c_int),
    "rebk_get_blocks": ([_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "rebk_get_tables": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "rebk_export_storage": ([_P, ctypes.c_int32, _P], ctypes.c_int),
    "rebk_batch_create": ([ctypes.POINTER(_P), ctypes.c_int32, _P, _P, _P, ctypes.c_int, _P,
                           ctypes.POINTER(RebkBatchOptions)], ctypes.c_int),
    "rebk_batch_destroy": ([_P], None),
    "rebk_batch_solve": ([_P, _P, _P, _P, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                          _P, ctypes.POINTER(RebkBatchStats)], ctypes.c_int),
    "rebk_batch_solve_ex": ([_P, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_uint64, _P, ctypes.POINTER(RebkBatchStats)], ctypes.c_int),
    "rebk_batch_info": ([_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "rebk_batch_record": ([_P, _P, ctypes.c_int64, _P], ctypes.c_int),
    "rebk_solve_noalloc": ([_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                            ctypes.c_double, _P, _P, _P, ctypes.c_int64, ctypes.c_uint64, _P], ctypes.c_int),
    "rebk_mlp_create": ([ctypes.POINTER(_P), _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                         ctypes.c_int64, _P, ctypes.c_uint64, _P], ctypes.c_int),
    "rebk_mlp_destroy": ([_P], None),
    "rebk_mlp_forward": ([_P, _P, ctypes.c_int64, _P], ctypes.c_int),
    "rebk_mlp_gradients": ([_P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "rebk_mlp_train_step": ([_P, _P, _P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
                            ctypes.c_int),
    "rebk_mlp_get_weights": ([_P, _P], ctypes.c_int),
    "rebk_mlp_set_loss": ([_P, ctypes.c_int32, ctypes.c_double], ctypes.c_int),
    "rebk_mlp_shape": ([_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "rebk_warm_start": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "rebk_warm_start_batch": ([_P, _P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P], ctypes.c_int),
    "rebk_sparse_create": ([ctypes.POINTER(_P), ctypes.c_int64, ctypes.c_int64, _P, _P, _P, ctypes.c_int64,
                            ctypes.c_int64, ctypes.c_double, ctypes.POINTER(RebkSparseOptions)], ctypes.c_int),
    "rebk_sparse_destroy": ([_P], None),
    "rebk_sparse_solve": ([_P, _P, _P, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                           ctypes.POINTER(RebkSolveExt), ctypes.POINTER(RebkStats)], ctypes.c_int),
    "rebk_sparse_solve_refined": ([_P, _P, _P, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.POINTER(RebkRefineOpts), ctypes.POINTER(RebkSolveExt),
                                   ctypes.POINTER(RebkStats)], ctypes.c_int),
    "rebk_sparse_info": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "rebk_selftest_waits": ([ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "rebk_gemm_bf16": ([ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.c_int64,
                        ctypes.c_float, _P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "rebk_device_peaks": ([ctypes.POINTER(RebkPeaks), _P], ctypes.c_int),
    "rebk_last_error": ([], ctypes.c_char_p),
    "rebk_version": ([], ctypes.c_char_p),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load librebk.so (building it first if needed).  Raises if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"librebk.so not found at {path}; build it with "
                                   "paper_2001_04179_gb300/build.py")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


class RebkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, allow=(REBK_OK,)) -> int:
    if status not in allow:
        raise RebkError(status, load().rebk_last_error().decode())
    return status
