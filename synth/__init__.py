"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This package holds no arithmetic of the solver: it only samples closed curves
(node coordinates, outward normals, quadrature weights, curvature) and draws
the random workload parameters.  Both the CUDA path and the oracle consume
its output.
"""

from .curves import (  # noqa: F401
    Curve,
    disk,
    star,
    fourier_star,
    fourier_star_at,
    random_star_batch,
    workload,
    WORKLOADS,
)
