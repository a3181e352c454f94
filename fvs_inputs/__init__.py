"""Seeded synthetic inputs (meshes, wall data, UQ samples) shared by the tests,
the benchmark and the oracle.  Holds no finite-volume arithmetic."""
from .mesh import box_mesh, casting_mesh, strip_mesh, voxel_mesh, zones_inner_box  # noqa: F401
from . import cases  # noqa: F401
