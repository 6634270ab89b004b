"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This package holds no arithmetic of the method: it only lays out structured P1 meshes
(triangles and tetrahedra, or quadrilaterals and hexahedra) of a box domain Omega with its
interaction layer, with an optional seeded vertex jitter, their higher-order nodes, and
describes the workloads (horizon, mollifier width,
refinement levels, kernel, manufactured solution) the tests and the benchmark run.
"""
from .mesh import HEX27, Mesh, hex_mesh, p2_mesh, q2_hex_mesh, q2_mesh, quad_mesh, s20_hex_mesh, s2_mesh, structured_mesh, splitmix64_unit  # noqa: F401
from .configs import WORKLOADS, Workload, workload_mesh  # noqa: F401
