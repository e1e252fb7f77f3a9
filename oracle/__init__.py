"""Plain FP64 CPU oracle of the bootstrap AMG method for Markov chains.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
statement of what the CUDA library computes, written from the paper
(Brannick, Kahl, Sokolovic, "An adaptively constructed algebraic multigrid
preconditioner for irreducible Markov chains").  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the library never does, and this package never imports the
library.  Each function cites the section / equation / algorithm it follows.

Modules
  rng         SplitMix64 counter-based generator (initial test vectors, MIS
              priorities)
  operators   B = I - A, transpose, structural sparse products (Section 2, 3)
  coarsening  geometric and greedy-MIS C/F splitting, interpolation sets J_i
  smoothing   weighted Jacobi, lexicographic and multicolour Gauss-Seidel
  interp      least-squares interpolation P and constrained restriction Q
              (eq. ls_interpolation, eq. ls_weights, Section 5), with an
              optional Tikhonov term towards equal weights (not in the paper)
  coarsest    generalized singular triplets and pseudo-inverse on the
              coarsest level (eq. generalized_eigenvalue)
  setup       Algorithm 1 (bamg_mle), the first and later bootstrap cycles
  solve       V-cycle (eq. error_propagator_twogrid), right FGMRES, the
              paper's left-preconditioned GMRES (eq. prec_residual),
              unpreconditioned GMRES(m), reference stationary vectors
"""
