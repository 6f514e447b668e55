"""Plain FP64 CPU oracle for LOBPCG on the 7-point 3-D Dirichlet Laplacian.

TEST INFRASTRUCTURE ONLY.  This package is a slow, obviously-correct restatement
of the method of Knyazev, Argentati, Lashuk and Ovtchinnikov, "Block Locally
Optimal Preconditioned Eigenvalue Xolvers (BLOPEX) in hypre and PETSc"
(Section 2.2, "The Detailed Description of the LOBPCG Algorithm"), plus the
geometric-multigrid V-cycle that stands in for the paper's hypre/PETSc
preconditioners.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never imports, links or calls anything here, and this package
shares no code with it.

Everything is numpy/scipy in float64.  Library primitives (matrix products,
Cholesky, the dense symmetric-definite eigensolver) serve as single steps; no
blocking, fusion or reordering beyond what the paper's algorithm states.

Modules
  rng        -- SplitMix64 counter generator for the random initial block.
  laplace    -- the 7-point operator, its closed-form eigenpairs (Section 4.1).
  multigrid  -- the V-cycle preconditioner T (weighted Jacobi, full weighting,
                trilinear prolongation, exact coarsest solve).
  dense      -- scale-invariant Cholesky (Section 2.2) and the Rayleigh-Ritz
                generalized eigensolve (Section 2.2).
  lobpcg     -- the block LOBPCG iteration with soft locking (Sections 2.2, 2.3).

Parity status per function is stated in each module header; the V-cycle values
beyond the pins listed in ``multigrid`` are "parity unpinned" (the paper does
not define this preconditioner; its definition is this project's reading).
"""

from . import rng, laplace, multigrid, dense, lobpcg  # noqa: F401
