"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and bench.py.

This package holds geometry and random numbers only: surface meshes (vertex and
triangle arrays), seeded coefficient vectors and seeded incidence directions.  It
contains none of the NESA/EFIE arithmetic (no basis functions, no Green's function,
no quadrature, no tree), so that the oracle and the CUDA path stay independent.
"""
from .meshes import icosphere, geodesic_ellipsoid, plate, aircraft  # noqa: F401
from .vectors import random_coefficients, plane_wave_directions  # noqa: F401
from .configs import CONFIGS, get_config  # noqa: F401
