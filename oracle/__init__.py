"""CPU FP64 oracle for the block alpha-circulant nested-Chebyshev solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the method computes, written from the paper (Tabeart,
Gurol, Pearson, Weaver: "Block alpha-circulant preconditioners for all-at-once
diffusion-based covariance operators").  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import it.  The CUDA library never calls it, shares no code with it, and it
imports nothing from the CUDA package.

Everything is numpy float64 / complex128.  Each function cites the section,
equation, theorem or algorithm of the paper it restates.  Where the paper is
silent or inconsistent the reading taken is stated beside the code:

* Kronecker factorisation (Eq. 4): the forward transform U* uses
  exp(-2 pi i (t-1)(j-1)/ell) and frequency j pairs with the shift
  lambda_j = alpha^(1/ell) exp(-2 pi i (j-1)/ell).  As printed, U and Lambda
  carry the same sign and do not reproduce C_alpha; conjugating Lambda does.
  The set of shifts is the same, so Fig. 1 and the printed roots still hold.
* The Chebyshev recurrence (Section 3) is not printed, only its polynomial
  (proof of Proposition 1); the textbook three-term recurrence is used.
* The outer solver is right-preconditioned flexible GMRES (the paper's outer
  solver is Chebyshev semi-iteration, Section 5); stopping uses the paper's
  relative residual ||b - A x|| / ||b|| with x_0 = 0 (Section 5).

Pins: every function here is checked by ``tests/test_oracle_*.py`` against
closed forms, the paper's printed numbers (``tests/golden/``), brute-force
dense solves or invariants.  No function is left "parity unpinned".

Modules:
  operator   -- A = I + K (Neumann finite volume), the paper's Dirichlet
                operator (Eq. 17, Appendix A), Gershgorin bound.
  allatonce  -- the all-at-once matrix (Eq. 1), C_alpha and P_alpha (Eq. 2).
  spectral   -- shifts, scalings, Fourier matrix, Chebyshev polynomial and the
                convergence results (Theorems 1, 3, 4; Proposition 1;
                Corollary 1; Algorithm 1).
  chebyshev  -- textbook Chebyshev semi-iteration on B_j = A - lambda_j I.
  precond    -- P_NC^{-1} (Eq. 5 with inner CI), exact P_alpha^{-1}, and the
                best-case P_alpha^{-1} through the spatial DCT (constant
                diffusivities, Section 2.2).
  saddle     -- P_SP (Section 4): CG on the real shifts, block-diagonally
                preconditioned MINRES on the saddle-point systems, and the
                aggregation multigrid V-cycle that applies the SPD blocks.
  gmres      -- right-preconditioned flexible GMRES (MGS, Givens).
  outer_ci   -- the paper's outer Chebyshev semi-iteration over Corollary 1's
                interval (Section 5).
  solve      -- FGMRES on Eq. 1 with P_NC^{-1}, assembled from the above.
  exact      -- the solution of Eq. 1 by sequential solves; plain CG.
"""
