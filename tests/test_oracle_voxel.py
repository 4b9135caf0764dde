"""Pins of ``oracle.voxel`` (trilinear lookup of a signed-distance grid, the
comparison system of Sec. 4.3): each pin is chosen so that a plausible
mistake (a swapped axis, a wrong corner weight, a sign or scale slip in the
gradient, the outside-the-box rule) fails one of them."""

import numpy as np

import synth
from oracle import voxel

LO, HI = np.array([-1.0, -0.8, -1.2]), np.array([1.0, 1.2, 0.9])   # unequal spacing per axis


def nodes(n, lo=LO, hi=HI):
    h = (hi - lo) / (n - 1)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return lo[0] + h[0] * i, lo[1] + h[1] * j, lo[2] + h[2] * k      # each [n_z, n_y, n_x]


def test_affine_fields_are_reproduced_exactly():
    """Trilinear interpolation reproduces every affine function and its
    gradient; distinct coefficients per axis catch a transposed axis."""
    a, b = np.array([0.3, -1.7, 2.9]), 0.25
    x, y, z = nodes(9)
    grid = a[0] * x + a[1] * y + a[2] * z + b
    p = synth.uniform_cube(500, 3) * np.array([0.99, 0.99, 0.9]) + np.array([0.0, 0.2, -0.15])
    f, g = voxel.query(grid, LO, HI, p)
    np.testing.assert_allclose(f, p @ a + b, atol=1e-12)
    np.testing.assert_allclose(g, np.broadcast_to(a, g.shape), atol=1e-11)


def test_node_values_and_bilinear_faces():
    s = synth.Stream(4)
    grid = s.normal(7 ** 3).reshape(7, 7, 7)
    x, y, z = nodes(7)
    p = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    f, _ = voxel.query(grid, LO, HI, p)
    np.testing.assert_allclose(f, grid.ravel(), atol=1e-12)
    # the midpoint of a cell is the mean of its 8 corners
    h = (HI - LO) / 6
    m = LO + h * np.array([2.5, 1.5, 3.5])
    fm, _ = voxel.query(grid, LO, HI, m[None, :])
    np.testing.assert_allclose(fm[0], grid[3:5, 1:3, 2:4].mean(), atol=1e-12)


def test_gradient_matches_central_differences_inside_cells():
    s = synth.Stream(5)
    grid = s.normal(6 ** 3).reshape(6, 6, 6)
    h = (HI - LO) / 5
    cell = (s.u64(3 * 200) % np.uint64(5)).astype(np.float64).reshape(200, 3)
    frac = 0.1 + 0.8 * s.uniform(3 * 200).reshape(200, 3)      # away from the cell faces
    p = LO + h * (cell + frac)
    _, g = voxel.query(grid, LO, HI, p)
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1e-6 * h[a]
        fp, _ = voxel.query(grid, LO, HI, p + e)
        fm, _ = voxel.query(grid, LO, HI, p - e)
        np.testing.assert_allclose(g[:, a], (fp - fm) / (2 * e[a]), rtol=1e-6, atol=1e-6)


def test_outside_the_box():
    """f = f(nearest box point) + distance; the gradient gains the outward direction."""
    a = np.array([0.3, -1.7, 2.9])
    x, y, z = nodes(5)
    grid = a[0] * x + a[1] * y + a[2] * z
    q = np.array([HI[0], 0.1, -0.3])                       # on the +x face
    p = q + np.array([0.4, 0.0, 0.0])
    f, g = voxel.query(grid, LO, HI, p[None, :])
    np.testing.assert_allclose(f[0], q @ a + 0.4, atol=1e-12)
    np.testing.assert_allclose(g[0], [1.0, a[1], a[2]], atol=1e-11)
    p2 = np.array([HI[0] + 0.3, HI[1] + 0.4, 0.0])        # beyond an edge: distance 0.5
    f2, g2 = voxel.query(grid, LO, HI, p2[None, :])
    q2 = np.array([HI[0], HI[1], 0.0])
    np.testing.assert_allclose(f2[0], q2 @ a + 0.5, atol=1e-12)
    np.testing.assert_allclose(g2[0], [0.6, 0.8, a[2]], atol=1e-11)


def test_sphere_grid_error_within_the_interpolation_bound():
    """A sphere SDF |p| - r sampled at spacing h: trilinear interpolation
    errs by at most h^2/8 times the largest second derivative along an axis
    (1/|p| for the distance function) summed over the three axes."""
    lo, hi = -np.ones(3), np.ones(3)
    n = 41
    x, y, z = nodes(n, lo, hi)
    grid = np.sqrt(x ** 2 + y ** 2 + z ** 2) - 0.5
    p = synth.uniform_cube(3000, 8)
    r = np.linalg.norm(p, axis=1)
    sel = r > 0.3
    f, g = voxel.query(grid, lo, hi, p[sel])
    h = 2.0 / (n - 1)
    bound = 3 * h * h / 8 / (r[sel] - np.sqrt(3) * h)
    assert np.all(np.abs(f - (r[sel] - 0.5)) <= bound)


def test_collide_lands_on_eps_for_a_plane():
    """For an affine field the projected point lies exactly on f = eps."""
    a = np.array([0.0, 0.6, 0.8])                        # unit normal
    x, y, z = nodes(5)
    grid = a[0] * x + a[1] * y + a[2] * z - 0.1
    p = synth.uniform_cube(400, 9) * 0.5
    eps = 0.002
    f, N, hit, xp = voxel.collide(grid, LO, HI, p, eps)
    np.testing.assert_allclose(N, np.broadcast_to(a, N.shape), atol=1e-12)
    np.testing.assert_array_equal(hit, f < eps)
    f2, _ = voxel.query(grid, LO, HI, xp[hit])
    np.testing.assert_allclose(f2, eps, atol=1e-12)
    np.testing.assert_array_equal(xp[~hit], p[~hit])
