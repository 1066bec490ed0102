"""Writes precision_anchor.txt: what the FP64 oracle does on the 8000 x 20000,
rank-2000 workload (A = G1 G2, b = A x* + N(0, 0.01^2), seed 0; blocks of
tau = 128; alpha = 1.75 / beta_max).

Calls only the oracle (and the seeded generators).  The recorded values are:
beta_max from the exact block spectral norms, alpha, and the iteration count
at which Algorithm 1 (Philox seed 1000, stream 0) first reaches
||x - A^+ b|| <= 1e-8 ||A^+ b|| when tested every 10 iterations, plus the
oracle's own time per iteration on this machine (single thread).

Usage: python tests/golden/make_precision_anchor.py  (about 10 minutes)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from workloads import contiguous_offsets, product_problem  # noqa: E402

M, N, R, TAU, SEED, SOLVE_SEED, CHECK, TOL = 8000, 20000, 2000, 128, 0, 1000, 10, 1e-8


def main():
    t0 = time.time()
    p = product_problem(M, N, R, seed=SEED, noise=0.01)
    ro, co = contiguous_offsets(M, TAU), contiguous_offsets(N, TAU)
    bI, bJ = O.beta_max(p.A, ro, co)
    alpha = 1.75 / max(bI, bJ)
    t1 = time.time()
    out = O.rebk(p.A, p.b, ro, co, alpha, seed=SOLVE_SEED, iters=400000, check_every=CHECK,
                 x_ref=p.x_ref, tol=TOL)
    t2 = time.time()
    rel = np.linalg.norm(out["x"] - p.x_ref) / np.linalg.norm(p.x_ref)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "precision_anchor.txt")
    with open(path, "w") as fh:
        fh.write("# Written by tests/golden/make_precision_anchor.py (oracle only).\n")
        fh.write(f"# workload: A = G1 G2, {M} x {N}, rank {R}, seed {SEED}; tau = {TAU}; "
                 f"Philox seed {SOLVE_SEED}, stream 0; test every {CHECK} iterations\n")
        fh.write(f"beta_row {bI!r}\nbeta_col {bJ!r}\nalpha {alpha!r}\n")
        fh.write(f"iterations_to_1e-8 {out['iters']}\nfinal_rel_err {float(rel)!r}\n")
        fh.write(f"oracle_seconds_per_iteration {(t2 - t1) / out['iters']!r}\n")
        fh.write(f"setup_seconds {t1 - t0!r}\n")
    print(open(path).read())


if __name__ == "__main__":
    main()
