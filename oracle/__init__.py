"""Plain, slow FP64 CPU oracle of the matrix-free multigrid elasticity solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import it: only the
test suite, the package-level smoke check and the benchmark's CPU-baseline leg
do.  It shares no code with the CUDA library; the only module both sides use is
the seeded input generator ``paper_2001_04789_gb300.microstructure``, which
holds none of the method's arithmetic.

Every function follows the paper (Runnels et al., "Massively parallel finite
difference elasticity using block-structured adaptive mesh refinement with a
geometric multigrid solver") step by step and cites the passage it follows.
Where the paper is silent the reading taken is stated in the docstring.

Modules:
  stencil    -- the discrete operator D_H, boundary-operator rows, RHS, block diagonal
  multigrid  -- hierarchy, transfers, red-black smoother, bottom solve, V-cycle, solve
  amr        -- composite (reflux-free) two-level cycle
"""
