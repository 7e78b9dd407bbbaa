"""liftblas for GB300: fused map/reduce kernels (asum, dot, scal, gemv) of
Steuwer, Fensch and Dubach, "Patterns and Rewrite Rules for Systematic Code
Generation" (arXiv 1502.02389), as hand-written sm_103a CUDA behind a C-ABI.

Modules:
  lift      -- ctypes binding of include/lift.h (same names as the C entry points)
  build     -- compiles csrc/*.cu into liftblas.so in this directory
  synth     -- seeded synthetic inputs of the benchmark workloads
"""
