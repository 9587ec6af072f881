"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds only input generation (microstructure coefficients on the grid, their separable
terms where the geometry gives them, random tensors for operator tests).  It contains none of the
homogenisation method's arithmetic, imports neither ``oracle`` nor the product package, and is the
only code both sides use.
"""
from .microstructures import (  # noqa: F401
    BASE_SEED, grid_points, square_inclusion, smoothed_cube, smoothed_sphere, laminate, lognormal_grf, random_tt,
    random_field,
)
