"""CPU oracle for the fused map/reduce hot path of Steuwer, Fensch and Dubach,
"Patterns and Rewrite Rules for Systematic Code Generation" (arXiv 1502.02389).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library (no headers, no
helpers, no tables); the two meet only through seeded inputs that a separate
generator module produces.

Contents
--------
patterns  -- FP64 interpreter and type checker of the high-level (Table 1) and
             OpenCL-level (Table 2) patterns, plus an fp32-rounded mode.
rules     -- the rewrite rules of Fig. 3 (algorithmic) and Fig. 4 (lowering).
blas      -- scal, asum, dot and gemv exactly as Fig. 5 writes them, and the
             parity tolerance.
lowlevel  -- the printed low-level expressions (Fig. 2b, Fig. 8, Fig. 9) and
             the parametrised low-level expression of each kernel variant.
mixed     -- exact decoding of bf16 and fp8-e4m3 stored values and the
             mixed-precision asum/dot definitions.
mlp       -- FP64 forward, backward and Adam step of the variant cost model.
finance   -- the BlackScholes map of Fig. 6 (Black-Scholes model, FP64).
"""
