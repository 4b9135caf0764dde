"""Procedural watertight triangle meshes (vertices float64 [V,3], faces int32 [F,3]).

All faces are oriented counter-clockwise seen from outside, so the winding
number of an interior point is +1.

* ``icosphere(level)``: the regular icosahedron subdivided ``level`` times
  (every triangle split into four, new vertices pushed to the unit sphere):
  20 * 4**level faces, 10 * 4**level + 2 vertices.
* ``displaced_icosphere``: icosphere vertices moved radially to
  r(u) = radius + amp * n(u), with n a seeded 3-octave value noise.  Radial
  displacement of a star-shaped mesh keeps it watertight and non-self-
  intersecting as long as r(u) > 0.
* ``box_mesh``: the 12-triangle surface of an axis-aligned box.
"""

import numpy as np

from .rng import splitmix64


def _orient_outward(V, F, centre=(0.0, 0.0, 0.0)):
    """Flip faces whose normal points towards ``centre`` (star-shaped meshes)."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    inward = np.einsum("ij,ij->i", n, (a + b + c) / 3.0 - np.asarray(centre)) < 0
    F = F.copy()
    F[inward] = F[inward][:, [0, 2, 1]]
    return F


def icosphere(level, radius=1.0):
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]],
                 dtype=np.int64)
    F = _orient_outward(V, F)
    for _ in range(level):
        verts = list(V)
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        newF = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            newF += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        V = np.array(verts)
        F = np.array(newF, dtype=np.int64)
    return V * radius, F.astype(np.int32)


def _lattice(seed, octave, ix, iy, iz):
    """Hash of integer lattice coordinates to a value uniform in [-1, 1)."""
    off = np.int64(1 << 20)
    k = ((ix + off).astype(np.uint64) << np.uint64(42)) \
        ^ ((iy + off).astype(np.uint64) << np.uint64(21)) \
        ^ (iz + off).astype(np.uint64)
    with np.errstate(over="ignore"):
        k = k + np.uint64((int(seed) * 0x51ED27 + octave * 0x2545F491) & 0xFFFFFFFFFFFFFFFF)
    h = splitmix64(splitmix64(k))
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def value_noise(x, seed, octaves=3, base_freq=2.0, lacunarity=2.0, gain=0.5):
    """Fractal value noise at points x [n,3], normalised by the sum of gains.

    Each octave interpolates hashed lattice values trilinearly with smoothstep
    weights s(t) = t^2 (3 - 2t).
    """
    x = np.asarray(x, dtype=np.float64)
    total = np.zeros(x.shape[0])
    amp, freq, norm = 1.0, base_freq, 0.0
    for o in range(octaves):
        q = x * freq
        i0 = np.floor(q).astype(np.int64)
        t = q - i0
        w = t * t * (3.0 - 2.0 * t)
        acc = np.zeros(x.shape[0])
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    v = _lattice(seed, o, i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz)
                    wx = w[:, 0] if dx else 1.0 - w[:, 0]
                    wy = w[:, 1] if dy else 1.0 - w[:, 1]
                    wz = w[:, 2] if dz else 1.0 - w[:, 2]
                    acc += v * wx * wy * wz
        total += amp * acc
        norm += amp
        amp *= gain
        freq *= lacunarity
    return total / norm


def displaced_icosphere(level=5, seed=7, radius=0.5, amp=0.05):
    V, F = icosphere(level)
    r = radius + amp * value_noise(V, seed)
    return V * r[:, None], F


def box_mesh(half=(0.3, 0.2, 0.1), centre=(0.0, 0.0, 0.0)):
    h = np.asarray(half, dtype=np.float64)
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1)
                        for sz in (-1, 1)], dtype=np.float64)
    V = corners * h + np.asarray(centre)
    # corner index = 4*(sx>0) + 2*(sy>0) + (sz>0)
    quads = [(0, 1, 3, 2), (4, 6, 7, 5),     # x = -h, x = +h
             (0, 4, 5, 1), (2, 3, 7, 6),     # y = -h, y = +h
             (0, 2, 6, 4), (1, 5, 7, 3)]     # z = -h, z = +h
    F = []
    for a, b, c, d in quads:
        F += [[a, b, c], [a, c, d]]
    F = _orient_outward(V, np.array(F, dtype=np.int64), centre)
    return V, F.astype(np.int32)
