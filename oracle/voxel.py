"""FP64 reference for the voxel SDF baseline (the comparison system of
Sec. 4.3, Table 1): a signed distance sampled on a regular grid, looked up by
trilinear interpolation.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definitions followed (the paper names the baseline and its grid resolution,
N = 256, but not its interpolation; the readings are this build's):

* grid: n^3 nodes over the box [lo, hi], node (i, j, k) at
  lo + (i, j, k) h with h = (hi - lo) / (n - 1), value grid[k, j, i];
* inside the box, f(p) is the trilinear interpolant of the 8 nodes of the
  cell holding p (the last cell for points on the upper faces), and grad f
  its gradient, differentiated per axis;
* outside the box, f(p) = f(q) + |p - q| with q the nearest point of the box,
  and grad f = grad f(q) along the axes where p is inside the box's slab, plus
  (p - q) / |p - q|;
* the normal, the test and the contact point are those of the network query
  (Eq. 2, Sec. 3.2, Eq. 3): N = grad f / |grad f| (zero where |grad f| <
  1e-20), collision where f < eps, p + (eps - f) N.
"""

import numpy as np

DEGENERATE_NORM = 1e-20


def query(grid, lo, hi, p):
    """(f, grad f) at points p [n, 3+] from a grid [n_z, n_y, n_x] = [n, n, n]."""
    grid = np.asarray(grid, dtype=np.float64)
    n = grid.shape[0]
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    h = (hi - lo) / (n - 1)
    p = np.asarray(p, dtype=np.float64)[:, :3]
    q = np.clip(p, lo, hi)
    outside = p - q
    d = np.linalg.norm(outside, axis=1)
    u = (q - lo) / h
    c = np.minimum(np.floor(u).astype(np.int64), n - 2)
    t = u - c
    f = np.zeros(p.shape[0])
    g = np.zeros((p.shape[0], 3))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                v = grid[c[:, 2] + dz, c[:, 1] + dy, c[:, 0] + dx]
                wx = t[:, 0] if dx else 1.0 - t[:, 0]
                wy = t[:, 1] if dy else 1.0 - t[:, 1]
                wz = t[:, 2] if dz else 1.0 - t[:, 2]
                f += v * wx * wy * wz
                sx = 1.0 if dx else -1.0
                sy = 1.0 if dy else -1.0
                sz = 1.0 if dz else -1.0
                g[:, 0] += v * sx * wy * wz / h[0]
                g[:, 1] += v * wx * sy * wz / h[1]
                g[:, 2] += v * wx * wy * sz / h[2]
    g[outside != 0.0] = 0.0              # f(q) does not change along a clamped axis
    out = d > 0.0
    f[out] += d[out]
    g[out] += outside[out] / d[out, None]
    return f, g


def collide(grid, lo, hi, p, eps):
    """(f, N, hit, x') of the collision query answered from the grid."""
    f, g = query(grid, lo, hi, p)
    nrm = np.linalg.norm(g, axis=1, keepdims=True)
    N = np.where(nrm < DEGENERATE_NORM, 0.0, g / np.where(nrm < DEGENERATE_NORM, 1.0, nrm))
    hit = f < eps
    x = np.asarray(p, dtype=np.float64)[:, :3].copy()
    x[hit] += (eps - f[hit])[:, None] * N[hit]
    return f, N, hit, x
