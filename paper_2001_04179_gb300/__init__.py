"""GB300-native (sm_103a) randomized extended block Kaczmarz (REBK) solver.

Du, Si, Sun, "Randomized extended block Kaczmarz for solving least squares",
arXiv:2001.04179.  The method runs in librebk.so (C ABI in include/rebk.h);
this package only marshals arguments, with torch for device memory.
"""
from .rebk import load, library_path, RebkError  # noqa: F401
from .solver import BatchSolver, Solver, SparseSolver, WarmStartNet, tune_tau  # noqa: F401

__all__ = ["load", "library_path", "RebkError", "Solver", "SparseSolver", "BatchSolver", "WarmStartNet", "tune_tau"]
