"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This package only *makes inputs*: procedural triangle meshes, area-uniform
surface samples, uniformly random rigid poses, scenes of many environments and
Xavier-initialised network parameters.  It holds none of the contact-detection
arithmetic (no crop selection, no network forward, no collision test); both
the oracle and the GPU library receive what it produces as plain arrays.

The paper trains and tests on scanned meshes (Google Scanned Objects, YCB,
EGAD; Sec. IV-A) that are not available here; the procedural shapes below
stand in for them (non-convex unions of boxes and ellipsoids, an L-bracket and
a torus).
"""

from .shapes import (Mesh, box_mesh, ellipsoid_mesh, torus_mesh, l_bracket,
                     random_union, sample_surface, ShapeLibrary, make_library,
                     tiny_library, convex_elements)
from .poses import (random_quaternions, random_poses, quat_multiply,
                    compose_relative_tiny)
from .weights import LAYER_DIMS, xavier_weights, voxel_weights
from .scenes import uneven_scene, sweep_pairs, client_batch
from .drop import drop_scene, drop_initial_state

__all__ = [
    "Mesh", "box_mesh", "ellipsoid_mesh", "torus_mesh", "l_bracket",
    "random_union", "sample_surface", "ShapeLibrary", "make_library",
    "tiny_library", "random_quaternions", "random_poses", "quat_multiply",
    "compose_relative_tiny", "LAYER_DIMS", "xavier_weights", "voxel_weights", "uneven_scene",
    "sweep_pairs", "client_batch", "drop_scene", "drop_initial_state", "convex_elements",
]
