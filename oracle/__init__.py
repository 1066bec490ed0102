"""Plain, slow FP64 CPU oracle for randomized extended block Kaczmarz (REBK).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package.  The solver
library (paper_2001_04179_gb300) never imports, links or runs it, and the two
share no code; the only module both use is ``workloads`` (seeded inputs).

Functions whose result the paper and mathematics pin (see tests/):
  philox / uniform / pick     -- numpy's Philox, chi-square on frequencies
  block_norms / cdf           -- direct sums, numpy
  rebk                        -- pseudoinverse limit, subspace invariants,
                                 REK and RABK special cases, closed-form mean
                                 recursion, expected-error bounds, Tables 1-2
  rebk_correction / refine    -- equals rebk from the shifted state; limit A^+ b
  rebk_sparse                 -- equals rebk on the dense form (same picks)
  beta_max                    -- Tables 1-2 step sizes, bounds of Remark rek9
  mlp_*                       -- finite differences, linear special case
"""
from .oracle import *  # noqa: F401,F403
