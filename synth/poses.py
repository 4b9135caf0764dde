"""Rigid body poses for scenes of several bodies (Sec. 4.2)."""

import numpy as np

from .rng import Stream


def rigid_transforms(n, seed=77, max_shift=0.5):
    """n row-major 4x4 rigid transforms [R | t; 0 0 0 1], float32 [n, 4, 4].

    R comes from a uniformly random unit quaternion (four standard normals,
    normalised; Shoemake, Graphics Gems III, 1992), t uniform in
    [-max_shift, max_shift]^3.
    """
    s = Stream(seed, tag=401)
    q = s.normal(4 * n).reshape(n, 4)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    T = np.zeros((n, 4, 4))
    T[:, 0, 0] = 1 - 2 * (y * y + z * z)
    T[:, 0, 1] = 2 * (x * y - w * z)
    T[:, 0, 2] = 2 * (x * z + w * y)
    T[:, 1, 0] = 2 * (x * y + w * z)
    T[:, 1, 1] = 1 - 2 * (x * x + z * z)
    T[:, 1, 2] = 2 * (y * z - w * x)
    T[:, 2, 0] = 2 * (x * z - w * y)
    T[:, 2, 1] = 2 * (y * z + w * x)
    T[:, 2, 2] = 1 - 2 * (x * x + y * y)
    T[:, :3, 3] = s.uniform(3 * n, -max_shift, max_shift).reshape(n, 3)
    T[:, 3, 3] = 1.0
    return T.astype(np.float32)
