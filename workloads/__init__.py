"""Seeded synthetic inputs shaped like the REBK paper's workloads.

This package is shared by the oracle tests and by the CUDA path.  It holds
none of the REBK method's arithmetic: only how test matrices, right-hand
sides and their known minimum-norm least-squares solutions are built.
"""
from .generators import *  # noqa: F401,F403
