"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package generates *inputs only*: query points, network weights from a
geometric initialisation, a procedural watertight mesh, a cloth grid and
per-network query counts.  It holds none of the query arithmetic (no SDF
evaluation, no gradient, no projection), so the oracle and the CUDA path can
both draw from it without sharing any of the method's computation.

Every generator is a pure function of its seed built on a counter-based
splitmix64 stream (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), so the same seed yields the same bits on x86 and
Arm hosts.
"""

from .rng import Stream, splitmix64
from .weights import Arch, geometric_init, layer_shapes, n_params, unpack, ff_matrix, fourier_relu_init
from .points import (uniform_cube, ellipsoid_shell, body_scale_points,
                     uniform_cube_points)
from .mesh import icosphere, displaced_icosphere, box_mesh, value_noise
from .cloth import cloth_grid, spring_list
from .counts import grouped_counts
from .training import training_points
from .poses import rigid_transforms

__all__ = [
    "Stream", "splitmix64", "Arch", "geometric_init", "layer_shapes", "ff_matrix",
    "fourier_relu_init",
    "n_params", "unpack", "uniform_cube", "ellipsoid_shell",
    "body_scale_points", "uniform_cube_points", "icosphere",
    "displaced_icosphere", "box_mesh", "value_noise", "cloth_grid",
    "spring_list", "grouped_counts", "training_points", "rigid_transforms",
]
