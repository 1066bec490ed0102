"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/*.h declares.  No compute call is made here."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(rebk_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["rebk_create", "rebk_solve", "rebk_solve_ex", "rebk_solve_refined",
                     "rebk_destroy", "rebk_beta_max", "rebk_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.rebk_version().decode().startswith("rebk-gb300")
    assert isinstance(lib.rebk_last_error().decode(), str)  # thread-local; earlier tests may have set it


def test_invalid_arguments_are_rejected_before_any_launch():
    """rebk_create validates its arguments on the host: these fail with
    EINVAL without touching a GPU."""
    import ctypes
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    h = ctypes.c_void_p()
    A = (ctypes.c_double * 4)(1, 2, 3, 4)
    opt = R.RebkOptions(1, 1, 0, 0, 0, None)
    assert lib.rebk_create(None, A, 2, 2, 2, 0, None, 1.0, ctypes.byref(opt)) == R.REBK_EINVAL
    assert lib.rebk_create(ctypes.byref(h), None, 2, 2, 2, 0, None, 1.0, ctypes.byref(opt)) == R.REBK_EINVAL
    assert lib.rebk_create(ctypes.byref(h), A, 0, 2, 2, 0, None, 1.0, ctypes.byref(opt)) == R.REBK_EINVAL
    assert lib.rebk_create(ctypes.byref(h), A, 2, 2, 1, 0, None, 1.0, ctypes.byref(opt)) == R.REBK_EINVAL
    bad = R.RebkOptions(-1, 1, 0, 0, 0, None)
    assert lib.rebk_create(ctypes.byref(h), A, 2, 2, 2, 0, None, 1.0, ctypes.byref(bad)) == R.REBK_EINVAL
    big = R.RebkOptions(1000, 1000, 0, 0, 0, None)
    # tau is clamped to m, n first: 2 x 2 with tau 1000 is fine in principle; a
    # tau above the kernel limit on a large matrix is EUNSUPPORTED
    assert "must" in lib.rebk_last_error().decode() or lib.rebk_last_error().decode() != ""
    assert lib.rebk_solve(None, None, None, 0.0, 1, 0, None) == R.REBK_EINVAL
    lib.rebk_destroy(None)


def test_package_has_no_cpu_fallback():
    """The package's Python sources never import the oracle."""
    pkg = os.path.join(ROOT, "paper_2001_04179_gb300")
    for path in glob.glob(os.path.join(pkg, "*.py")):
        src = open(path).read()
        assert "import oracle" not in src and "from oracle" not in src, path


def test_network_loss_selection_rejects_bad_arguments_on_the_host():
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    assert lib.rebk_mlp_set_loss(None, 0, 1.0) == R.REBK_EINVAL
    assert lib.rebk_batch_solve_ex(None, None, None, None, None, None, 0.0, 0, 0, 0, None, None) == R.REBK_EINVAL


def test_step_size_and_tuner_reject_bad_arguments_on_the_host():
    """rebk_set_alpha and rebk_tune_tau check their arguments before any CUDA call."""
    import ctypes
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    assert lib.rebk_set_alpha(None, 1.0) == R.REBK_EINVAL
    assert lib.rebk_spectral_estimates(None, 10, 0, None) == R.REBK_EINVAL
    assert lib.rebk_sparse_solve_refined(None, None, None, 1e-8, 10, 0, None, None, None) == R.REBK_EINVAL
    A = (ctypes.c_double * 4)(1, 2, 3, 4)
    b = (ctypes.c_double * 2)(1, 1)
    taus = (ctypes.c_int64 * 2)(1, 2)
    pts = (R.RebkTunePoint * 2)()
    best = ctypes.c_int64(7)
    P = lambda a: ctypes.cast(a, ctypes.c_void_p)

    def tune(A_=A, m=2, n=2, taus_=taus, count=2, storage=0, tol=1e-6, max_iter=10, trials=1):
        return lib.rebk_tune_tau(P(A_) if A_ is not None else None, m, n, n, 0, P(b),
                                 None, P(taus_) if taus_ is not None else None, count, 1.75, storage,
                                 tol, max_iter, 0, trials, None, P(pts), ctypes.byref(best))

    assert tune(A_=None) == R.REBK_EINVAL
    assert tune(taus_=None) == R.REBK_EINVAL
    assert tune(count=0) == R.REBK_EINVAL
    assert tune(m=0) == R.REBK_EINVAL
    assert tune(storage=9) == R.REBK_EINVAL
    assert tune(tol=0.0) == R.REBK_EINVAL
    assert tune(max_iter=0) == R.REBK_EINVAL
    assert tune(trials=0) == R.REBK_EINVAL
    assert best.value == 0
    zero = (ctypes.c_int64 * 2)(0, 2)
    assert tune(taus_=zero) == R.REBK_EINVAL
    assert "tau" in lib.rebk_last_error().decode()


def test_block_size_above_the_kernel_limit_is_unsupported_before_any_cuda_call():
    """tau is clamped to m and n first; what remains above 512 is rejected on the host."""
    import ctypes
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    h = ctypes.c_void_p()
    A = (ctypes.c_double * 4)(1, 2, 3, 4)   # never read: the call returns before any copy
    opt = R.RebkOptions(600, 8, 0, 0, 0, None)
    assert lib.rebk_create(ctypes.byref(h), A, 1000, 1000, 1000, 0, None, 1.0, ctypes.byref(opt)) == R.REBK_EUNSUPPORTED
    assert "tau" in lib.rebk_last_error().decode()
    assert not h.value


def test_header_is_plain_c():
    """The boundary header compiles as C99 (no C++ or torch types) and as C++."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:  # pragma: no cover
        pytest.skip("gcc not available")
    hdr = os.path.join(ROOT, "include", "rebk.h")
    subprocess.run([gcc, "-std=c99", "-fsyntax-only", "-Wall", "-Wextra", "-Werror", "-x", "c", hdr], check=True)
    gxx = shutil.which("g++")
    if gxx:
        subprocess.run([gxx, "-std=c++17", "-fsyntax-only", "-Wall", "-Werror", "-x", "c++", hdr], check=True)


def test_wait_selftest_rejects_bad_arguments_on_the_host():
    import ctypes
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    codes = (ctypes.c_int32 * 2)()
    assert lib.rebk_selftest_waits(10**6, None, None) == R.REBK_EINVAL
    assert lib.rebk_selftest_waits(10, ctypes.cast(codes, ctypes.c_void_p), None) == R.REBK_EINVAL
    assert lib.rebk_selftest_waits(10**10, ctypes.cast(codes, ctypes.c_void_p), None) == R.REBK_EINVAL


def test_partition_offsets_are_checked_before_any_cuda_call():
    """rebk_create's partition (Section 2's I_1..I_s, J_1..J_t) must run from 0 to
    m (n) strictly increasing, with blocks of at most 512; anything else is
    rejected on the host."""
    import ctypes
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    A = (ctypes.c_double * 4)(1, 2, 3, 4)   # never read: the call returns before any copy
    opt = R.RebkOptions(4, 4, 0, 0, 0, None)

    def create(row, col, m=100, n=50):
        h = ctypes.c_void_p()
        ro = None if row is None else (ctypes.c_int64 * len(row))(*row)
        co = None if col is None else (ctypes.c_int64 * len(col))(*col)
        part = R.RebkPartition(None if ro is None else ctypes.cast(ro, ctypes.c_void_p).value,
                               0 if row is None else len(row) - 1,
                               None if co is None else ctypes.cast(co, ctypes.c_void_p).value,
                               0 if col is None else len(col) - 1)
        st = lib.rebk_create(ctypes.byref(h), A, m, n, n, 0, ctypes.byref(part), 1.0, ctypes.byref(opt))
        assert not h.value
        return st

    assert create([1, 50, 100], None) == R.REBK_EINVAL          # does not start at 0
    assert create([0, 50, 99], None) == R.REBK_EINVAL           # does not end at m
    assert create([0, 50, 50, 100], None) == R.REBK_EINVAL      # an empty block
    assert create([0, 60, 40, 100], None) == R.REBK_EINVAL      # decreasing
    assert create(None, [0, 25]) == R.REBK_EINVAL               # ends short of n
    assert create(None, [0, 50, 60]) == R.REBK_EINVAL           # past n
    assert "column partition" in lib.rebk_last_error().decode()
    assert create([0, 600, 1000], None, m=1000) == R.REBK_EUNSUPPORTED  # a block above 512
    assert "512" in lib.rebk_last_error().decode()


def test_multi_right_hand_side_entry_points_reject_bad_arguments_on_the_host():
    """rebk_solve_multi and rebk_multi_group check the handle before any CUDA call."""
    import ctypes
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    opt = R.RebkMultiOpts(R.REBK_FP32, 0, 0, 0, 0, 0.0, None, 0)
    stats = R.RebkStats()
    assert lib.rebk_solve_multi(None, 1, None, 1, None, 1, 1e-8, 10, 0, ctypes.byref(opt), None, 0, None,
                                ctypes.byref(stats)) == R.REBK_EINVAL
    assert "NULL" in lib.rebk_last_error().decode()
    g = ctypes.c_int32(0)
    assert lib.rebk_multi_group(None, R.REBK_FP32, ctypes.byref(g)) == R.REBK_EINVAL


def test_batch_cluster_options_are_checked_on_the_host():
    """rebk_batch_create rejects a cluster size other than 0, 1, 2, 4, 8 and a
    negative joint_frac before any CUDA call."""
    import ctypes
    from paper_2001_04179_gb300 import rebk as R
    lib = R.load()
    m = (ctypes.c_int64 * 1)(4)
    n = (ctypes.c_int64 * 1)(3)
    A = (ctypes.c_double * 12)()
    ptrs = (ctypes.c_void_p * 1)(ctypes.cast(A, ctypes.c_void_p).value)
    h = ctypes.c_void_p()

    def create(cluster, joint_frac):
        opt = R.RebkBatchOptions(16, 8, 0, 0, 0.0, None, 0, cluster, joint_frac)
        return lib.rebk_batch_create(ctypes.byref(h), 1, ctypes.cast(m, ctypes.c_void_p),
                                     ctypes.cast(n, ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p), 0, None,
                                     ctypes.byref(opt))

    assert create(3, 0.0) == R.REBK_EINVAL
    assert "cluster" in lib.rebk_last_error().decode()
    assert create(16, 0.0) == R.REBK_EINVAL
    assert create(2, -1.0) == R.REBK_EINVAL
    assert "joint_frac" in lib.rebk_last_error().decode()
    assert create(2, float("nan")) == R.REBK_EINVAL
    assert not h.value
