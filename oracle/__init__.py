"""Plain, slow FP64 CPU oracle of the block-preconditioned Krylov solve.

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check in
__graft_entry__ and the CPU-baseline leg of bench.py may import this package.
The product path (the CUDA library and its Python binding) never calls it and
shares no code with it.

Modules
  physics  -- TPFA residual G(x) (Eq. Fm, Eq. Fe), its analytic Jacobian
              (Eq. AXR, Eq. App..Eq. rhouT) and the Schur approximation
              S~_T (Eq. Se)
  amg      -- classical AMG: strength, PMIS C/F split, classical
              interpolation, Galerkin product, l1-Jacobi / Chebyshev
              smoothing, V-cycle (Sec. 3, Sec. 4 solver settings)
  krylov   -- the five-step block preconditioner (Sec. 3.2) and flexible
              GMRES with restarts (Sec. 4 solver settings)

Everything is float64, single threaded, written for checking by eye rather
than for speed. Functions whose result has no independent pin say
"parity unpinned" in their docstring.
"""
