"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This package holds no arithmetic of the sampling method itself: it only
generates target tet meshes and request streams from seeds.  The random
numbers it draws (vertex jitter, request parameters) come from NumPy's PCG64,
not from the Philox generator the method uses for white noise.
"""
from .mesh import kuhn_mesh, box_mesh, lprism_mesh, MeshSpec  # noqa: F401
from .cylinder import quarter_cylinder_mesh, polygon_prism_volume, radial_nodes  # noqa: F401
from .spe10 import cartesian_kuhn_mesh, spe10_mesh, SPE10_BOUNDING_BOX, SPE10_CELLS, SPE10_DOMAIN  # noqa: F401
