"""Seeded synthetic inputs for the DOLINC stage: meshes and initial cell averages.

This package only builds inputs (node coordinates, face/cell connectivity and
cell-averaged initial fields).  It holds none of the method's arithmetic:
geometry used by the scheme (volumes, centroids, interpolation weights, growth
rates) is computed independently by the oracle and by the CUDA library.

Both the oracle tests and the GPU path take their inputs from here.
"""
from .meshes import (tri_mesh, strip_mesh, tet_mesh, hexprism_mesh, hex_mesh,
                     mesh_summary)
from .fields import (cell_average, sine2d, gaussian3d, isentropic_vortex,
                     vortex_params, fourier_modes, riemann_quadrants,
                     prim_to_cons)
from .workloads import workload, WORKLOADS, STENCIL_OF_ORDER

__all__ = [
    "tri_mesh", "strip_mesh", "tet_mesh", "hexprism_mesh", "hex_mesh",
    "mesh_summary", "cell_average", "sine2d", "gaussian3d", "isentropic_vortex",
    "vortex_params", "fourier_modes", "riemann_quadrants", "prim_to_cons",
    "workload", "WORKLOADS", "STENCIL_OF_ORDER",
]
