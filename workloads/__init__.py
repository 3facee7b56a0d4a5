"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds none of the method's arithmetic: it only builds triangle
meshes (vertex coordinates and triangle index lists), the time-step size and
step count of each workload, the parameters of the incident pulse, and seeded
random current histories.  Everything that evaluates the method (basis
functions, kernels, integrals, fields) lives either in ``oracle/`` or in the
CUDA library, each written independently.
"""
from .meshes import icosphere, cube_jittered, cylinder_cone, ellipsoid_uv, octa_ellipsoid, mean_edge_length
from .configs import Pulse, Workload, workload, pulse_star, random_history, WORKLOADS

__all__ = [
    "icosphere", "cube_jittered", "cylinder_cone", "ellipsoid_uv", "octa_ellipsoid",
    "mean_edge_length", "Pulse", "Workload", "workload", "pulse_star", "random_history",
    "WORKLOADS",
]
