"""Plain, slow FP64 CPU oracle for the MCD pressure-Poisson hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package: only the tests, `__graft_entry__.smoke()` and
the CPU-baseline leg of `bench.py` use it.  It shares no code with the CUDA
library (no kernels, headers, helpers or tables); the seeded generators in
`paper_2404_17542_gb300.inputs` are the only module both sides read.

Modules (each function cites the passage of arXiv 2404.17542 it restates):
  mask     DP masking (Sec. 2.2, Eq. (1)), arrangement (Sec. 2.3, Eqs. (2)-(9))
           and moving-boundary role reassignment (Sec. 2.4)
  mls      chi=1 quadratic MLS stencil weights (Sec. 3.2, Eqs. (12)-(17))
  solve    sparse assembly of the pressure-Poisson system (Eq. (21)) and a
           textbook BiCGSTAB (Sec. 3.3)
  flow     projection-method driver pieces (Sec. 3.3, Eqs. (20)-(23))
  ale      the moving-boundary step: ALE interpolation (Eq. (19), Appendix A),
           boundary velocities and rigid accelerations (Eqs. (24)-(29)), the
           fluid force (Eqs. (30)-(31)) and the whole step in the order of
           Sec. 3.3 (moving_step)
  sdf      discrete signed-distance bodies and their MLS interpolation
           (Sec. 2.5)
  cnn      FP64 forward/backward of the small convolutional network used as
           the learned warm start (an addition: the paper has no network)

Parity status: every function is pinned by a `-m "not gpu"` test against a
closed form, a brute-force recount, a dense library solve or an invariant,
except where the module header says "parity unpinned".
"""
