"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module builds meshes (triangle soups), sphere packings and random densities.
It holds none of the boundary-integral arithmetic: quadrature points, weights and
normals are computed separately by ``oracle.quadrature`` (CPU) and by the
library's ``kifmm_quadrature_points`` kernel (GPU).
"""
from .geometry import (  # noqa: F401
    Mesh,
    cube_surface,
    geodesic_sphere,
    sphere_pack,
    pack_mesh,
    cube_n_for_triangles,
    geodesic_freq_for_triangles,
)
from .workloads import (  # noqa: F401
    WORKLOADS,
    batch_instances,
    serve_requests,
    workload,
    uniform_density,
)
