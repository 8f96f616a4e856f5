"""Plain, slow FP64 CPU oracle of the block-preconditioned Krylov solve.

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check in
__graft_entry__ and the CPU-baseline leg of bench.py may import this package.
The product path (the CUDA library and its Python binding) never calls it and
shares no code with it.

Modules
  physics  -- TPFA residual G(x) (Eq. Fm, Eq. Fe) for water or the Bennison
              heavy oil, its analytic Jacobian (Eq. AXR, Eq. App..Eq. rhouT)
              and the Schur approximations S~_T (Eq. Se), S~_ATT, S~_diag
              (Sec. 3.3)
  amg      -- classical AMG: strength, PMIS C/F split, classical and
              extended+i interpolation with truncation, Galerkin product,
              l1-Jacobi / Chebyshev smoothing, V-cycle with a dense LU on the
              coarsest level (Sec. 3, Sec. 4 solver settings)
  krylov   -- the five-step block preconditioner (Sec. 3.2), flexible GMRES
              with restarts (Sec. 4 solver settings), the Table-4 condition
              numbers
  newton   -- Newton with backtracking line search for one backward-Euler
              step (Sec. 3, Sec. 4)
  learned  -- features, MLP, exact Schur columns and the corrected S~_T of
              the learned Schur correction (no counterpart in the paper)

Everything is float64, single threaded, written for checking by eye rather
than for speed. Functions whose result has no independent pin say
"parity unpinned" in their docstring.
"""
