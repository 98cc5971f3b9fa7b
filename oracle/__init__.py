"""FP64 CPU oracle for the EMIN-AMG V-cycle / FGMRES path (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only the tests, the `smoke()` check in
`__graft_entry__.py` and the CPU-baseline leg of `bench.py` may import it.  The
product path (the C++ setup, the CUDA kernels and their Python binding)
shares no code with it, and it imports nothing from the product.

It is a plain, slow restatement of the method, step by step in the paper's
order (Alg. 1-4, Section 4.3 for EMIN, Section 5.2 for Braess-Sarazin,
Section 5.1 for Vanka, Section 5 for ILU(1)),
written with numpy / scipy.sparse primitives and Python loops over graph
vertices.  Where the paper is silent or garbled, the reading taken is stated
in the docstring of the function that implements the step.

Parity status per function (the pins are in tests/test_oracle_*.py and
tests/test_synth.py):
  * filter_lump, find_coarse_pressures (with the min-distance reading of
    update_heuristics), pressure_pattern, find_velocity_cpoints,
    velocity_pattern, emin_step, the Galerkin products, gauss_seidel,
    bs_sweep, coarse_solve, vcycle, fgmres: pinned (closed forms, the
    paper's worked special cases, invariants, dense brute force, Table 1).
  * vanka.py (Vanka relaxation, Section 5.1): pinned (block definition,
    exact local solves, colored sweep = block-by-block sweep, dense solves,
    Table 1's Vanka(1,1) counts); the coarsest-level Vanka relaxation of
    Section 6.1 (Params.coarse = "vanka"): pinned (pre + post steps from zero on
    a one-level hierarchy, dense solves with it).
  * ilu.py (ILU(1) relaxation, Section 5): pinned (L U = A on the kept
    pattern, the level-of-fill rule, exactness without fill, the zero-pivot
    reading on a 3x3 saddle matrix, the error-propagation spectrum, dense
    solves, Table 1's and Table 5's ILU(1)(1,1) counts).
  * find_extra_dist3_cpoints: pinned on hand-built graphs whose conversions
    are worked out by hand (one C-point at distance 3; two C-points at distance
    3 with the point on either side of the quarter-length threshold and beyond
    the segment's end), and it fires on the perturbed-coordinate meshes of the
    setup-parity tests, where the library's choices equal the oracle's.
  * emin_step: pinned by its optimality (the CG step is the exact line
    minimum of the energy along -Proj(A P0); the GMRES step's projected
    residual is orthogonal to Proj(A R0)), with a projection built in the test
    from null-space bases.
"""
from .hierarchy import Params, Hierarchy, setup_hierarchy  # noqa: F401
from .solve import bs_sweep, vcycle, fgmres, apply_A  # noqa: F401
