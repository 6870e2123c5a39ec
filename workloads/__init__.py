"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Holds meshes, coefficient fields, the finest-level stiffness matrix and
right-hand sides, and nothing of the multigrid method itself.
"""
from .configs import (Problem, checkerboard_square, helmholtz_square,  # noqa: F401
                      lognormal_square, lshape_anisotropic, poisson_square,
                      square_with_coefficients, training_square)
from .meshes import MeshHierarchy, MeshLevel  # noqa: F401
