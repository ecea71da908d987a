"""FP64 CPU oracle for the SPDE sampler (test infrastructure only).

Plain, slow, obviously correct statements of what the sampling path
computes, used to check the CUDA library.  Only the tests, the smoke check
and the CPU-baseline leg of the benchmark may import this package; the
library never calls it and shares no code with it.

Modules:
  philox   -- Philox4x32-10 and the Box-Muller white-noise mapping (Sec. 4.2)
  mixed    -- RT0 x P0 mixed system assembled by quadrature, sparse direct
              and DCT closed-form solves, exact discrete covariance (Sec. 4)
  clip     -- tet/hex intersection volumes by convex hulls, coupling matrix G
              (Sec. 5.1-5.2)
  project  -- L2 projection W_h^{-1} G and the lognormal map (Eq. proj_op)
  vcycle   -- plain restatement of the multigrid preconditioner operator
"""
