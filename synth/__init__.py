"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds only input generation (point sets and normals, the
Helmholtz single- and double-layer collocation matrices, random probe
vectors).  It contains none of the
compression method's arithmetic and imports neither the oracle nor the
CUDA package.
"""
from .inputs import (  # noqa: F401
    fibonacci_sphere,
    random_sphere,
    random_ellipsoid,
    random_cube_surface,
    mean_nn_distance,
    helmholtz_matrix,
    sphere_normals,
    ellipsoid_normals,
    dlp_matrix,
    planted_separable_matrix,
    random_complex_vectors,
    SEED,
)
