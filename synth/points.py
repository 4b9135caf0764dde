"""Seeded query-point sets, returned as float32 [n, 4] (x, y, z, 0).

The fourth component pads each point to 16 bytes so a point is one aligned
vector load on the device.
"""

import numpy as np

from .rng import Stream


def _pad4(xyz):
    out = np.zeros((xyz.shape[0], 4), dtype=np.float32)
    out[:, :3] = xyz
    return out


def uniform_cube(n, seed, half=1.0):
    """n points uniform in [-half, half]^3 as float64 [n, 3]."""
    s = Stream(seed, tag=101)
    return s.uniform(3 * n, -half, half).reshape(n, 3)


def ellipsoid_shell(n, seed, axes=(0.3, 0.5, 0.2), sigma=0.01):
    """n points x = diag(axes) u + N(0, sigma^2 I), u uniform on the unit sphere.

    The direction u is a normalised Gaussian vector, so the samples are
    uniform in direction, not in surface area; the offset makes a thin shell
    of points on both sides of the ellipsoid.
    """
    s = Stream(seed, tag=102)
    g = s.normal(3 * n).reshape(n, 3)
    u = g / np.linalg.norm(g, axis=1, keepdims=True)
    x = u * np.asarray(axes)[None, :]
    return x + s.normal(3 * n, std=sigma).reshape(n, 3)


def uniform_cube_points(n, seed=1):
    """Tiny workload: n points uniform in [-1, 1]^3 (float32 [n, 4])."""
    return _pad4(uniform_cube(n, seed))


def body_scale_points(n, seed=1, frac_surface=0.9):
    """Body-scale workload: 90% on a noisy ellipsoid shell, 10% uniform.

    The surface share is floor-free: n_surf = round(frac_surface * n).  The two
    groups are interleaved by a seeded permutation so every tile of points
    mixes near-surface and far points, as a cloth draped over a body would.
    """
    n_surf = int(round(frac_surface * n))
    xyz = np.concatenate([ellipsoid_shell(n_surf, seed),
                          uniform_cube(n - n_surf, seed)])
    s = Stream(seed, tag=103)
    perm = np.argsort(s.u64(n), kind="stable")
    return _pad4(xyz[perm])
