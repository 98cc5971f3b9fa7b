"""Seeded synthetic inputs shared by the CUDA path and the oracle.

Holds the splitmix64 generator and the Q2-Q1 problem generator (the block
system of Section 2, its coordinates and right-hand sides); none of the
multigrid method's arithmetic lives here.
"""
from .rng import splitmix64, uniform_pm1, uniform01, exponential  # noqa: F401
from .serving import MESHES, REYNOLDS, serving_stream, homogeneous_rhs  # noqa: F401
from .q2q1 import (Problem, make_problem, stokes_pinned_2d, stokes_lid_2d,  # noqa: F401
                   oseen_recirculating_2d, stokes_lid_3d, element_matrices, recirculating_wind,
                   with_perturbed_coordinates)
from .navier_stokes import picard_lid_cavity, lid_cavity_problem  # noqa: F401
