"""Seeded training-point sampler for fitting a network to a mesh (Sec. 3.1).

80% of the points are near the surface (area-uniform on the triangles plus an
isotropic Gaussian offset of std `sigma`), 20% uniform in [-1, 1]^3; the paper
samples near-surface and uniform points at this ratio with a margin of a few
millimetres.  Returns float32 [n, 4] (w = 0).
"""

import numpy as np

from .rng import Stream


def training_points(V, F, n, seed, near_frac=0.8, sigma=0.01):
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F)
    s = Stream(seed, tag=401)
    n_near = int(round(near_frac * n))
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    cdf = np.cumsum(area) / area.sum()
    tri = np.searchsorted(cdf, s.uniform(n_near), side="right")
    tri = np.minimum(tri, len(F) - 1)
    r1, r2 = s.uniform(n_near), s.uniform(n_near)
    sq = np.sqrt(r1)                          # uniform barycentric sampling
    w0, w1, w2 = 1.0 - sq, sq * (1.0 - r2), sq * r2
    p = w0[:, None] * a[tri] + w1[:, None] * b[tri] + w2[:, None] * c[tri]
    p = p + s.normal(3 * n_near, std=sigma).reshape(n_near, 3)
    u = s.uniform(3 * (n - n_near), -1.0, 1.0).reshape(n - n_near, 3)
    out = np.zeros((n, 4), dtype=np.float32)
    out[:, :3] = np.concatenate([p, u])
    return out
