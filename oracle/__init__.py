"""CPU FP64 oracle for the fast random-walk Kalman filter -- TEST INFRASTRUCTURE.

This package is the independent, plain and slow reference that the CUDA path is
checked against.  It is test infrastructure only: the tests, the smoke check
and the benchmark's CPU-baseline leg may import it; the library never does.
It shares no code with the CUDA path (the seeded input generators in `synth`
are the one common dependency and hold none of the method's arithmetic).

Contents (each function cites the passage it follows):
  matern      -- Matern covariance kernel, Sec. 2.2.1 Eq. maternfamily
  covariance  -- dense Gamma, exact Gamma x by direct sums and by circulant
                 embedding on regular grids (Sec. 2.2.1)
  kalman      -- O1: the textbook Kalman filter with F = I (Alg. standard and
                 the random-walk assumption of Sec. 2.1); O2: the exact
                 cross-covariance recursion for a fixed H, evaluated on sampled
                 rows (same Kalman algebra, tracking Sigma H^T); O1t: O1 with
                 the rank control of Alg. lowrankaddition step 4 (rank cap and
                 relative truncation) applied densely; O1e: the extended filter
                 of Sec. 4.2 (Alg. extkalman) with the Box-Cox map of Eq.
                 nonlinear
  ghep        -- Eq. ghep solved exactly (the definition) and by the randomized
                 algorithm of App. B (Alg. randomizedghepuncert)
  uq          -- variance, relative entropy and conditional realizations
                 (Sec. 3) computed densely from a covariance matrix, and the
                 paper's low-rank representation (Eq. sigmakk) recovered
                 densely from a covariance

Parity status: every function is pinned by a test in tests/test_oracle_*.py
against a closed form, an independent algebraic identity, a library routine or
brute force (see each test's docstring).  No function is "parity unpinned".
"""
